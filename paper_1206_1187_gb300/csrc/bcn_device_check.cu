// bcn_device_check.cu -- a kernel written only against include/bcn_device.cuh,
// the way a user's simulation would call the device-side generator, exposed
// through the C ABI so the header is checked against the oracle like every
// other path.
#include "bcn_device.cuh"
#include "bcn_internal.h"

namespace {

// Thread t of T takes variates [t*n/T, (t+1)*n/T) of the call, with its own
// generator positioned there; FP64, FP32 and (when `st` is not null) the raw
// state of each variate go to their arrays, each from its own copy of the
// generator.
__global__ void device_api_kernel(uint64_t start, uint64_t offset, uint64_t n, double* f64,
                                  float* f32, uint64_t* st) {
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t a = (uint64_t)((unsigned __int128)n * t / T);
  const uint64_t b = (uint64_t)((unsigned __int128)n * (t + 1) / T);
  if (a >= b) return;
  bcn_device::Stream g = bcn_device::make_stream(start, offset, a);
  bcn_device::Stream h = g, k = g;
  for (uint64_t i = a; i < b; ++i) {
    f64[i] = bcn_device::next_f64(g);
    f32[i] = bcn_device::next_f32(h);
    if (st) st[i] = bcn_device::next_state(k);
  }
}

// Thread t of T consumes variates [t*n/T, (t+1)*n/T) in registers: the
// wrap-around sum of their bit patterns (one integer add each, so the FP64
// pipe stays free) is its only output (sums[t]).  FP64: one next_f64 call per
// variate.  FP32: runs of kRunF32 from f32_run, the remainder by next_f32.
constexpr int kRunF32 = 32;
template <bool F32>
__global__ void device_api_checksum_kernel(uint64_t start, uint64_t offset, uint64_t n,
                                           uint64_t* sums) {
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t a = (uint64_t)((unsigned __int128)n * t / T);
  const uint64_t b = (uint64_t)((unsigned __int128)n * (t + 1) / T);
  uint64_t s = 0, i = a;
  if constexpr (F32) {
    for (; i + kRunF32 <= b; i += kRunF32) {
      float v[kRunF32];
      bcn_device::f32_run<kRunF32>(start, offset, i, v);
#pragma unroll
      for (int k = 0; k < kRunF32; ++k) s += __float_as_uint(v[k]);
    }
    bcn_device::Stream g = bcn_device::make_stream(start, offset, i);
    for (; i < b; ++i) s += __float_as_uint(bcn_device::next_f32(g));
  } else {
    bcn_device::Stream g = bcn_device::make_stream(start, offset, a);
    for (; i < b; ++i) s += (uint64_t)__double_as_longlong(bcn_device::next_f64(g));
  }
  sums[t] = s;
}

// Thread t of T writes FP32 variates [t*n/T, (t+1)*n/T) of the call: runs of
// kRunF32 from f32_run, the remainder by next_f32.
__global__ void device_api_f32_runs_kernel(uint64_t start, uint64_t offset, uint64_t n,
                                           float* out) {
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t a = (uint64_t)((unsigned __int128)n * t / T);
  const uint64_t b = (uint64_t)((unsigned __int128)n * (t + 1) / T);
  uint64_t i = a;
  for (; i + kRunF32 <= b; i += kRunF32) {
    float v[kRunF32];
    bcn_device::f32_run<kRunF32>(start, offset, i, v);
#pragma unroll
    for (int k = 0; k < kRunF32; ++k) out[i + k] = v[k];
  }
  bcn_device::Stream g = bcn_device::make_stream(start, offset, i);
  for (; i < b; ++i) out[i] = bcn_device::next_f32(g);
}

}  // namespace

using namespace bcn;

extern "C" rng_status rng_device_api_checksum(uint64_t start_index, uint64_t offset,
                                              uint64_t n, rng_dtype dt, uint64_t* sums,
                                              uint32_t threads, void* cuda_stream) {
  if (start_index < kSeedMin || start_index > kSeedMax)
    return set_error(RNG_ERANGE, "start index outside [3^33+100, 2^53]");
  if (dt != RNG_F64 && dt != RNG_F32)
    return set_error(RNG_EINVAL, "dtype %d: the checksum takes RNG_F64 or RNG_F32", (int)dt);
  if (threads == 0 || threads % 128 != 0)
    return set_error(RNG_EINVAL, "threads %u must be a positive multiple of 128", threads);
  if (!sums || (uintptr_t)sums % 8) return set_error(RNG_EINVAL, "sums NULL or misaligned");
  const cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
  if (dt == RNG_F32)
    device_api_checksum_kernel<true><<<threads / 128, 128, 0, cs>>>(start_index, offset, n, sums);
  else
    device_api_checksum_kernel<false><<<threads / 128, 128, 0, cs>>>(start_index, offset, n, sums);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "device API checksum launch");
  return RNG_OK;
}

extern "C" rng_status rng_device_api_f32_runs(uint64_t start_index, uint64_t offset,
                                              uint64_t n, float* out, uint32_t threads,
                                              void* cuda_stream) {
  if (start_index < kSeedMin || start_index > kSeedMax)
    return set_error(RNG_ERANGE, "start index outside [3^33+100, 2^53]");
  if (threads == 0 || threads % 128 != 0)
    return set_error(RNG_EINVAL, "threads %u must be a positive multiple of 128", threads);
  if (n == 0) return RNG_OK;
  if (!out || (uintptr_t)out % 4) return set_error(RNG_EINVAL, "output NULL or misaligned");
  device_api_f32_runs_kernel<<<threads / 128, 128, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      start_index, offset, n, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "device API FP32 runs launch");
  return RNG_OK;
}

extern "C" rng_status rng_device_api_check(uint64_t start_index, uint64_t offset, uint64_t n,
                                           double* out_f64, float* out_f32,
                                           uint64_t* out_state, uint32_t threads,
                                           void* cuda_stream) {
  if (start_index < kSeedMin || start_index > kSeedMax)
    return set_error(RNG_ERANGE, "start index outside [3^33+100, 2^53]");
  if (n == 0) return RNG_OK;
  if (!out_f64 || !out_f32 || (uintptr_t)out_f64 % 8 || (uintptr_t)out_f32 % 4 ||
      (uintptr_t)out_state % 8)
    return set_error(RNG_EINVAL, "outputs NULL or misaligned");
  if (threads == 0) threads = 1;
  const uint32_t block = threads < 128 ? threads : 128;
  const uint32_t grid = (threads + block - 1) / block;
  device_api_kernel<<<grid, block, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      start_index, offset, n, out_f64, out_f32, out_state);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "device API check launch");
  return RNG_OK;
}
