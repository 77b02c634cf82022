// bcn_m40_api.cu -- host side of the 3^40 generator: argument checks, the
// launch shape a call resolves to, and the launch.  The kernels are in
// bcn_m40.cu.
#include "bcn_m40.cuh"
#include "bcn_math40.cuh"

namespace bcn {

// Defaults for fields left zero (measured on GB300 with the 2^28-variate
// FP64 workload).
constexpr uint32_t k40DefDepth = 31, k40DefBlock = 896, k40DefChains = 1, k40DefBuffers = 1;
// FP32 on one chain makes each run from one product; 44-deep runs stored four
// variates at a time measured 1431-1435 G variates/s against 1318 for 31-deep
// runs stored one at a time (2^28 FP32).
constexpr uint32_t k40DefDepthF32 = 44, k40DefBlockF32 = 1024;

struct Launch40 {
  int dt, layout;
  uint32_t depth, block, grid, chains, buffers;
  size_t smem_bytes;
};

static rng_status resolve40(uint64_t n, int dt, const rng_tune* tune, Launch40* out) {
  rng_tune t = {};
  if (tune) t = *tune;
  if (t.step || t.conv || t.skip || t.unit)
    return set_error(RNG_EINVAL,
                     "the 3^40 variant has one step, conversion and skip-ahead: tune.step, "
                     "conv, skip and unit must be 0");
  if (dt != DT_F64 && dt != DT_F32 && dt != DT_U64)
    return set_error(RNG_EINVAL, "dtype %d is not an rng_dtype", dt);
  Launch40 L = {};
  L.dt = dt;
  L.layout = t.layout ? (int)t.layout : RNG_LAYOUT_TILED;
  if (L.layout != RNG_LAYOUT_TILED && L.layout != RNG_LAYOUT_DIRECT)
    return set_error(RNG_EINVAL, "tune.layout %u is not a layout", t.layout);
  if (t.chains > 2) return set_error(RNG_EINVAL, "tune.chains %u must be 0, 1 or 2", t.chains);
  if (t.buffers > 2) return set_error(RNG_EINVAL, "tune.buffers %u must be 0, 1 or 2", t.buffers);
  DeviceInfo di;
  rng_status st = device_info(&di);
  if (st != RNG_OK) return st;
  if (L.layout == RNG_LAYOUT_TILED) {
    // FP32 on one chain also takes 44-deep runs (four-variate stores)
    const bool one_chain32 = dt == DT_F32 && (t.chains ? t.chains : k40DefChains) == 1;
    L.depth = t.depth ? t.depth : (one_chain32 ? k40DefDepthF32 : k40DefDepth);
    L.block = t.block ? t.block : (one_chain32 && L.depth == k40DefDepthF32 ? k40DefBlockF32
                                                                            : k40DefBlock);
    const bool four = one_chain32 && L.depth == k40DefDepthF32;
    if ((L.depth % 2 == 0 && !four) || L.depth > kMaxDepth)
      return set_error(RNG_EINVAL,
                       "tune.depth %u must be odd (FP32 on one chain: or 44) and at most %u",
                       L.depth, kMaxDepth);
    if (L.block % 32 != 0 || L.block == 0 || L.block > 1024)
      return set_error(RNG_EINVAL, "tune.block %u must be a multiple of 32, <= 1024", L.block);
    L.chains = t.chains ? t.chains : k40DefChains;
    if (L.depth < 3) L.chains = 1;
    L.buffers = t.buffers ? t.buffers : k40DefBuffers;
    const size_t warp_bytes = (size_t)L.buffers * 32 * L.depth * dtype_size(dt);
    L.smem_bytes = (size_t)(L.block / 32) * warp_bytes;
    // a chosen block that does not fit shrinks, four warps at a time while it
    // can, then by halves (whole warps throughout)
    while (!t.block && L.smem_bytes > di.smem_optin && L.block > 32) {
      L.block = L.block > 128 ? L.block - 128 : L.block / 2;
      L.smem_bytes = (size_t)(L.block / 32) * warp_bytes;
    }
    if (L.smem_bytes > di.smem_optin)
      return set_error(RNG_EINVAL, "tile buffers need %zu bytes of shared memory, %zu available",
                       L.smem_bytes, di.smem_optin);
    const void* fn = pick40(dt, L.layout, L.chains, L.depth);
    st = enable_smem(fn, di.device, L.smem_bytes);
    if (st != RNG_OK) return st;
    if (t.grid) {
      L.grid = t.grid;
    } else {
      int per_sm = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)L.block,
                                                                    L.smem_bytes);
      if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (per_sm < 1) per_sm = 1;
      const uint64_t full = (uint64_t)per_sm * (uint64_t)di.sms;
      const uint64_t tiles = n / (32ull * L.depth);
      uint64_t need = (tiles + L.block / 32 - 1) / (L.block / 32);
      if (need < 1) need = 1;
      L.grid = (uint32_t)(need < full ? need : full);
    }
  } else {
    L.chains = 1;
    L.block = t.block ? t.block : 256;
    if (L.block == 0 || L.block > 1024)
      return set_error(RNG_EINVAL, "tune.block %u must be in 1..1024", L.block);
    if (t.grid) {
      L.grid = t.grid;
    } else {
      const uint64_t threads = (n + 4095) / 4096;
      uint64_t g = (threads + L.block - 1) / L.block;
      if (g < 1) g = 1;
      if (g > (1u << 30)) g = 1u << 30;
      L.grid = (uint32_t)g;
    }
  }
  if (L.grid == 0 || L.grid > (1u << 30))
    return set_error(RNG_EINVAL, "tune.grid %u out of range", L.grid);
  *out = L;
  return RNG_OK;
}

static uint64_t jump40(uint64_t steps) {
  return host40_mont_form(host40_pow2((uint64_t)(((u128)53 * steps) % k40P)));
}

static rng_status launch40(const Launch40& L, uint64_t seed, uint64_t i0, uint64_t n, void* out,
                           cudaStream_t cs) {
  const void* fn = pick40(L.dt, L.layout, L.chains, L.depth);
  if (!fn) return set_error(RNG_EINVAL, "no kernel for this combination");
  const uint64_t ebase = host40_exponent_base(seed, i0);
  cudaError_t e;
  if (L.layout == RNG_LAYOUT_TILED) {
    // the tiled kernel's chains run backwards and hold, for variates, the
    // state one above the next element (the digit of which continues it)
    const uint64_t lead = L.dt == DT_U64 ? 0 : 1;
    const uint64_t c = L.depth, h = c / 2;
    M40Params p;
    p.out = static_cast<unsigned char*>(out);
    p.n = n;
    p.head = head_elems(out, dtype_size(L.dt), n);
    p.ntiles = n > p.head ? (n - p.head) / (32ull * c) : 0;
    p.ebase = ebase;
    // element 0 -> element c of the next run; a one-product FP32 run's state
    // (one past the run) moves 32c elements instead
    const bool digits = L.dt == DT_F32 && L.chains == 1 && digit_run40_depth(c);
    p.jump = digits ? jump40(32 * c) : jump40(33 * c + lead);
    p.jump_a = jump40(32 * c + h + 1 + lead); // element 0 -> element h+1 of the next run
    p.jump_b = jump40(33 * c - h - 1 + lead); // element h+1 -> element c of the next run
    p.depth = L.depth;
    p.nbuf = L.buffers;
    void* args[] = {&p};
    e = cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block), args, L.smem_bytes, cs);
  } else {
    unsigned char* o = static_cast<unsigned char*>(out);
    uint64_t nn = n, eb = ebase;
    void* args[] = {&o, &nn, &eb};
    e = cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block), args, 0, cs);
  }
  if (e != cudaSuccess) return cuda_error(e, "3^40 kernel launch");
  return RNG_OK;
}

}  // namespace bcn

using namespace bcn;

extern "C" {

rng_status rng40_generate_at(uint64_t start_index, uint64_t offset, uint64_t n, rng_dtype dt,
                             void* out, void* cuda_stream, const rng_tune* tune) {
  if (start_index < k40SeedMin)
    return set_error(RNG_ERANGE, "start index %llu below 3^40+100",
                     (unsigned long long)start_index);
  if (dt != RNG_F64 && dt != RNG_F32 && dt != RNG_U64)
    return set_error(RNG_EINVAL, "dtype %d is not an rng_dtype", (int)dt);
  if (n == 0) return RNG_OK;
  if (n > RNG_MAX_N)
    return set_error(RNG_ERANGE, "n = %llu exceeds RNG_MAX_N", (unsigned long long)n);
  if (out == nullptr) return set_error(RNG_EINVAL, "output pointer is NULL");
  if ((uintptr_t)out % dtype_size((int)dt) != 0)
    return set_error(RNG_EINVAL, "output pointer is not aligned to its %zu-byte elements",
                     dtype_size((int)dt));
  Launch40 L;
  rng_status st = resolve40(n, (int)dt, tune, &L);
  if (st != RNG_OK) return st;
  return launch40(L, start_index, offset, n, out, static_cast<cudaStream_t>(cuda_stream));
}

rng_status rng40_resolve_tune(uint64_t n, rng_dtype dt, const rng_tune* tune, rng_tune* out) {
  if (!out) return set_error(RNG_EINVAL, "out is NULL");
  Launch40 L;
  rng_status st = resolve40(n, (int)dt, tune, &L);
  if (st != RNG_OK) return st;
  rng_tune r = {};
  r.layout = (uint32_t)L.layout;
  r.depth = L.depth;
  r.block = L.block;
  r.grid = L.grid;
  r.chains = L.chains;
  r.buffers = L.buffers;
  *out = r;
  return RNG_OK;
}

}  // extern "C"
