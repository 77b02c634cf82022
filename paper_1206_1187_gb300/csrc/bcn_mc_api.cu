// bcn_mc_api.cu -- host side of the fused Monte-Carlo consumer: argument
// checks and the launch.  The kernel is in bcn_mc.cu.
#include "bcn_math.cuh"
#include "bcn_mc.cuh"

using namespace bcn;

extern "C" {

rng_status rng_consume_mc(uint64_t start_index, uint64_t block0, uint64_t nblocks, uint64_t len,
                          uint64_t* hits_total, uint64_t* hits, double* sum, double* sumsq,
                          void* cuda_stream, const rng_tune* tune) {
  if (start_index < kSeedMin || start_index > kSeedMax)
    return set_error(RNG_ERANGE, "start index outside [3^33+100, 2^53]");
  if (len == 0 || len % 2 != 0) return set_error(RNG_EINVAL, "len must be even and > 0");
  if (len > RNG_MAX_N) return set_error(RNG_ERANGE, "len exceeds RNG_MAX_N");
  if (nblocks == 0) return RNG_OK;
  if (!hits_total || !sum || !sumsq) return set_error(RNG_EINVAL, "hits_total, sum and sumsq are required");
  if (((uintptr_t)hits_total | (uintptr_t)sum | (uintptr_t)sumsq | (uintptr_t)hits) % 8 != 0)
    return set_error(RNG_EINVAL, "outputs must be 8-byte aligned");
  if (nblocks > UINT64_MAX / len || block0 > UINT64_MAX / len - nblocks)
    return set_error(RNG_ERANGE, "block range overflows");
  if (len / 2 > 0xFFFFFFFFull) return set_error(RNG_ERANGE, "len too large for 32-bit hit counts");
  rng_tune t = {};
  if (tune) t = *tune;
  const uint32_t block = t.block ? t.block : 128;  // measured: 128 and 256 within 0.5%
  if (block % 32 != 0 || block > 256)
    return set_error(RNG_EINVAL, "tune.block %u must be a multiple of 32, <= 256", block);
  const uint32_t skip = t.skip ? t.skip : (uint32_t)SK_TABLE;
  if (skip != SK_TABLE && skip != SK_SQMUL) return set_error(RNG_EINVAL, "bad tune.skip");
  // tune.conv chooses where each RN(v*v) is formed: RNG_CONV_FP64 on the FP64
  // pipe, RNG_CONV_INT on the integer pipes (0: the default)
  const uint32_t conv = t.conv ? t.conv : kMcDefaultConv;
  if (conv != CV_INT && conv != CV_FP64) return set_error(RNG_EINVAL, "bad tune.conv");
  cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
  McParams p;
  p.ebase = host_exponent_base(start_index, 0);
  p.block0 = block0;
  p.nblocks = nblocks;
  p.len = len;
  p.hits_total = reinterpret_cast<unsigned long long*>(hits_total);
  p.hits = hits;
  p.sum = sum;
  p.sumsq = sumsq;
  p.skip = skip;
  cudaError_t e = cudaMemsetAsync(hits_total, 0, sizeof(uint64_t), cs);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(hits_total)");
  const uint64_t wpb = block / 32;
  const uint64_t grid = (nblocks + wpb - 1) / wpb;
  if (grid > 0x7fffffffull) return set_error(RNG_ERANGE, "too many blocks for one launch");
  void* args[] = {&p};
  const void* fn = mc_kernel_fn(conv == CV_FP64);
  e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(block), args, 0, cs);
  if (e != cudaSuccess) return cuda_error(e, "mc kernel launch");
  return RNG_OK;
}

}  // extern "C"
