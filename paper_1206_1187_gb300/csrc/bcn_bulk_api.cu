// bcn_bulk_api.cu -- host side of single-stream generation: the launch
// shape a call resolves to (tile depth, block, chains, buffers, grid) and the
// launch itself.  The kernels are in bcn_bulk.cu.
#include <algorithm>
#include <mutex>
#include <set>
#include <utility>

#include "bcn_bulk.cuh"
#include "bcn_host.h"
#include "bcn_strided.cuh"
#include "bcn_math.cuh"

namespace bcn {

// Large dynamic shared memory must be enabled once per kernel and device.
rng_status enable_smem(const void* fn, int device, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({fn, device})) return RNG_OK;
  DeviceInfo di;
  rng_status st = device_info(&di);
  if (st != RNG_OK) return st;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)di.smem_optin);
  if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
  (void)bytes;
  done.insert({fn, device});
  return RNG_OK;
}

static uint64_t tile_count(uint64_t n, uint64_t head, uint32_t depth) {
  return n > head ? (n - head) / (32ull * depth) : 0;
}

// The launch shape for fields left zero when no tuning is installed: the
// shape the autotuner picks on GB300 for 2^28 variates of every output type
// (FP64 756, raw states 821 G/s there, against 573 and 704 with 15-deep tiles
// in 256-thread blocks).  FP32 tiles are half the bytes, so FP32 can take
// deeper tiles in the same shared memory.  With the backward FP32 step,
// 44-deep tiles stored four variates at a time measured 1.5% faster than
// 47-deep ones stored one at a time, and those 1% faster than 63-deep.
constexpr uint32_t kDefDepth = 31, kDefBlock = 896, kDefChains = 2, kDefBuffers = 1;
constexpr uint32_t kDefDepthF32 = 44, kDefBlockF32 = 1024;
// The forward FP64 step on two chains stores two variates at a time in
// 30-deep runs (2.3% faster than 31-deep one-variate runs).
constexpr uint32_t kDefDepthF64Vec = 30;
// Its 44-deep tiles fit 32 warps per SM: 1024-thread blocks (999 against 995
// G variates/s with 896).  Other FP32 launches (forward steps, one chain)
// need odd depths: 47.
constexpr uint32_t kDefDepthF32Odd = 47;
// `vec`: the launch runs a kernel that takes even depths (the backward FP32
// runs or the forward FP64 runs on two chains with the shared step).
inline uint32_t def_depth(int dt, bool vec) {
  if (dt == DT_F32) return vec ? kDefDepthF32 : kDefDepthF32Odd;
  if (dt == DT_F64 && vec) return kDefDepthF64Vec;
  return kDefDepth;
}

rng_status resolve_bulk(uint64_t n, int dt, const rng_tune* tune, BulkLaunch* out,
                        bool constant) {
  rng_tune t = {};
  if (tune) t = *tune;
  // a block the caller (or BCN_RNG_TUNE) chose, before installed defaults fill it
  const bool caller_block = t.block != 0 || (!constant && env_tune_sets_block());
  if (!constant) {  // zero fields take the installed (measured) defaults
    const rng_status env = env_tune_check();
    if (env != RNG_OK) return env;
    const rng_tune d = auto_defaults(dt);
    if (d.layout == RNG_LAYOUT_STRIDED)
      return set_error(RNG_EINVAL, "the strided layout permutes the output; only a call's own "
                                   "tuning may name it, not a default");
    const bool same_layout = t.layout != RNG_LAYOUT_STRIDED &&
                             (!t.layout || !d.layout || t.layout == d.layout);
    if (!t.step) t.step = d.step;
    if (!t.conv) t.conv = d.conv;
    if (!t.skip) t.skip = d.skip;
    if (same_layout) {
      if (!t.layout) t.layout = d.layout;
      // an even default depth (the backward FP32 runs' four-variate stores)
      // goes only to calls that run that same kernel kind
      const bool same_kind = t.step == d.step && t.conv == d.conv &&
                             (!t.chains || !d.chains || t.chains == d.chains);
      if (!t.depth && (d.depth % 2 == 1 || same_kind)) t.depth = d.depth;
      if (!t.block) t.block = d.block;
      if (!t.chains) t.chains = d.chains;
      if (!t.buffers) t.buffers = d.buffers;
    }
  }
  BulkLaunch L = {};
  L.dt = dt;
  L.layout = t.layout ? (int)t.layout : RNG_LAYOUT_TILED;
  L.step = constant ? ST_CONST : (t.step ? (int)t.step : ST_SHARED);
  L.conv = t.conv ? (int)t.conv : CV_INT;
  L.skip = t.skip ? (int)t.skip : SK_TABLE;
  if (L.layout != RNG_LAYOUT_TILED && L.layout != RNG_LAYOUT_DIRECT &&
      L.layout != RNG_LAYOUT_STRIDED)
    return set_error(RNG_EINVAL, "tune.layout %u is not a layout", t.layout);
  if (!constant && L.step != ST_BARRETT && L.step != ST_MONT && L.step != ST_SHARED &&
      L.step != ST_LECUYER && L.step != ST_BCLASSIC)
    return set_error(RNG_EINVAL, "tune.step %u is not a step variant", t.step);
  if (L.conv != CV_INT && L.conv != CV_FP64)
    return set_error(RNG_EINVAL, "tune.conv %u is not a conversion", t.conv);
  if (L.skip != SK_TABLE && L.skip != SK_SQMUL)
    return set_error(RNG_EINVAL, "tune.skip %u is not a skip-ahead method", t.skip);
  if (dt != DT_F64 && dt != DT_F32 && dt != DT_U64)
    return set_error(RNG_EINVAL, "dtype %d is not an rng_dtype", dt);
  if (constant && dt == DT_U64)
    return set_error(RNG_EINVAL, "the constant fill writes RNG_F64 or RNG_F32");
  DeviceInfo di;
  rng_status st = device_info(&di);
  if (st != RNG_OK) return st;
  if (t.chains > 2) return set_error(RNG_EINVAL, "tune.chains %u must be 0, 1 or 2", t.chains);
  if (L.layout == RNG_LAYOUT_STRIDED) {  // the paper's coalesced kernels (Sec. 2.2)
    L.depth = t.depth ? t.depth : 4096;   // W: variates per thread, the paper's choice
    L.chains = t.unit ? t.unit : 8;       // here: the generation loop's unroll factor
    if (L.chains != 1 && L.chains != 8)
      return set_error(RNG_EINVAL, "tune.unit %u: the strided layout unrolls by 1 or 8", t.unit);
    if (n % L.depth != 0)
      return set_error(RNG_EINVAL, "the strided layout needs n = %llu to be a multiple of "
                                   "tune.depth = %u variates per thread",
                       (unsigned long long)n, L.depth);
    const uint64_t threads = n / L.depth;
    L.block = t.block ? t.block : 512;  // the paper's best block on its GPU
    if (L.block == 0 || L.block > 1024)
      return set_error(RNG_EINVAL, "tune.block %u must be in 1..1024", L.block);
    const uint64_t need = (threads + L.block - 1) / L.block;
    if (t.grid && (uint64_t)t.grid < need)
      return set_error(RNG_EINVAL, "tune.grid %u leaves threads of the strided layout out",
                       t.grid);
    if (need > 0x7fffffffull) return set_error(RNG_ERANGE, "too many threads for one launch");
    L.grid = t.grid ? t.grid : (uint32_t)need;
    L.buffers = 0;
    L.smem_bytes = 0;
    if (!pick_strided(dt, L.step, L.conv, L.chains))
      return set_error(RNG_EINVAL, "no kernel for this combination");
    *out = L;
    return RNG_OK;
  }
  L.chains = 1;
  // FP32 with the shared step and the integer conversion in the tiled layout
  // takes one chain by default, whose runs come from one product each, unless
  // the call names a depth those runs do not take
  const bool f32_one_product = dt == DT_F32 && L.step == ST_SHARED && L.conv == CV_INT &&
                               L.layout == RNG_LAYOUT_TILED &&
                               (!t.depth || digit_run_depth(t.depth));
  const uint32_t want_chains = t.chains ? t.chains : f32_one_product ? 1u : kDefChains;
  if (L.layout == RNG_LAYOUT_TILED && (L.step == ST_SHARED || L.step == ST_BARRETT) &&
      want_chains == 2 && (t.depth ? t.depth : def_depth(dt, false)) >= 3)
    L.chains = 2;
  // FP32 with the shared step on two chains runs the backward step (depths
  // odd or 4 mod 8), FP64 the forward step on scaled chains (odd or 2 mod 4)
  const bool two_shared = L.step == ST_SHARED && L.conv == CV_INT && L.chains == 2;
  const bool back32 = dt == DT_F32 && two_shared, scaled64 = dt == DT_F64 && two_shared;
  // FP32 with the shared step on one chain makes each run from one product
  // in runs of the depths digit_run_depth names
  const bool digits32 = dt == DT_F32 && L.step == ST_SHARED && L.conv == CV_INT &&
                        L.chains == 1 && L.layout == RNG_LAYOUT_TILED;
  const uint32_t depth0 = L.layout == RNG_LAYOUT_TILED
                              ? (t.depth ? t.depth : def_depth(dt, back32 || scaled64 || digits32))
                              : 0;
  const void* fn = pick_kernel(L.layout, dt, L.step, L.conv, (int)L.chains, depth0);
  if (!fn) return set_error(RNG_EINVAL, "no kernel for this combination");
  if (L.layout == RNG_LAYOUT_TILED) {
    L.depth = t.depth ? t.depth : def_depth(dt, back32 || scaled64 || digits32);
    L.block = t.block ? t.block : (back32 || digits32 ? kDefBlockF32 : kDefBlock);
    // odd depths keep the one-variate shared-memory stores bank-conflict free;
    // the backward FP32 runs also take depths of 4 mod 8 (four-variate
    // stores), the forward FP64 runs on two chains 2 mod 4 (two-variate)
    const bool even_ok = (back32 && vec4_depth(L.depth)) || (scaled64 && vec2_depth(L.depth)) ||
                         (digits32 && digit_run_depth(L.depth));
    if ((L.depth % 2 == 0 && !even_ok) || L.depth > kMaxDepth)
      return set_error(RNG_EINVAL,
                       "tune.depth %u must be odd (on two chains with the shared step also "
                       "4 mod 8 for FP32, 2 mod 4 for FP64) and at most %u",
                       L.depth, kMaxDepth);
    if (L.block % 32 != 0 || L.block == 0 || L.block > 1024)
      return set_error(RNG_EINVAL, "tune.block %u must be a multiple of 32, <= 1024",
                       L.block);
    if (t.buffers > 2) return set_error(RNG_EINVAL, "tune.buffers %u must be 0, 1 or 2", t.buffers);
    L.buffers = t.buffers ? t.buffers : kDefBuffers;
    const size_t warp_bytes = (size_t)L.buffers * 32 * L.depth * dtype_size(dt);
    L.smem_bytes = (size_t)(L.block / 32) * warp_bytes;
    // a chosen block that does not fit shrinks, four warps at a time while it
    // can (whole warps for each of the SM's four schedulers), then by halves
    while (!t.block && L.smem_bytes > di.smem_optin && L.block > 32) {
      L.block = L.block > 128 ? L.block - 128 : L.block / 2;
      L.smem_bytes = (size_t)(L.block / 32) * warp_bytes;
    }
    if (L.smem_bytes > di.smem_optin)
      return set_error(RNG_EINVAL, "tile buffers need %zu bytes of shared memory, %zu available",
                       L.smem_bytes, di.smem_optin);
    // A call with too few tiles to give every SM a full block takes blocks
    // just large enough to spread its tiles over all SMs (whole groups of four
    // warps from four warps up), unless the caller chose the block or the
    // grid: 10^6 FP64 variates ran 14.8 us in 896-thread blocks on 36 SMs and
    // 9.2 us in 256-thread blocks on 126.
    if (!caller_block && !t.grid) {
      const uint64_t per_sm = (tile_count(n, 0, L.depth) + di.sms - 1) / di.sms;
      uint64_t b = std::max<uint64_t>(per_sm, 1) * 32;
      if (b >= 128) b = (b + 127) / 128 * 128;
      if (b < L.block) {
        L.block = (uint32_t)b;
        L.smem_bytes = (size_t)(L.block / 32) * warp_bytes;
      }
    }
    if (t.grid) {
      L.grid = t.grid;
    } else {
      st = enable_smem(fn, di.device, L.smem_bytes);
      if (st != RNG_OK) return st;
      int per_sm = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)L.block,
                                                                    L.smem_bytes);
      if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (per_sm < 1) per_sm = 1;
      uint64_t full = (uint64_t)per_sm * (uint64_t)di.sms;
      // no more warps than tiles (at least one block for the edges)
      uint64_t tiles = tile_count(n, 0, L.depth);
      uint64_t need = (tiles + L.block / 32 - 1) / (L.block / 32);
      if (need < 1) need = 1;
      L.grid = (uint32_t)(need < full ? need : full);
    }
  } else {
    L.depth = 0;
    L.block = t.block ? t.block : 256;
    if (L.block == 0 || L.block > 1024)
      return set_error(RNG_EINVAL, "tune.block %u must be in 1..1024", L.block);
    if (t.grid) {
      L.grid = t.grid;
    } else {
      // the paper's best split: about 4096 variates per thread (Sec. 2.2)
      uint64_t threads = (n + 4095) / 4096;
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

rng_status launch_bulk(const BulkLaunch& L, uint64_t seed, uint64_t i0, uint64_t n,
                       void* out, uint64_t const_bits, cudaStream_t cs) {
  const uint64_t ebase = (L.step == ST_CONST) ? 0 : host_exponent_base(seed, i0);
  cudaError_t e;
  if (L.layout == RNG_LAYOUT_STRIDED) {
    const void* sf = pick_strided(L.dt, L.step, L.conv, L.chains);
    if (!sf || n % L.depth != 0) return set_error(RNG_EINVAL, "strided launch does not fit n");
    StridedParams p;
    p.out = static_cast<unsigned char*>(out);
    p.nthreads = n / L.depth;
    p.per = L.depth;
    p.ebase = ebase;
    p.cbits = const_bits;
    p.skip = (uint32_t)L.skip;
    void* args[] = {&p};
    e = cudaLaunchKernel(sf, dim3(L.grid), dim3(L.block), args, 0, cs);
    if (e != cudaSuccess) return cuda_error(e, "strided kernel launch");
    return RNG_OK;
  }
  const void* fn = pick_kernel(L.layout, L.dt, L.step, L.conv, (int)L.chains, L.depth);
  if (!fn) return set_error(RNG_EINVAL, "no kernel for this combination");
  if (L.layout == RNG_LAYOUT_TILED) {
    DeviceInfo di;
    rng_status st = device_info(&di);
    if (st != RNG_OK) return st;
    st = enable_smem(fn, di.device, L.smem_bytes);
    if (st != RNG_OK) return st;
    TiledParams p;
    p.out = static_cast<unsigned char*>(out);
    p.n = n;
    p.head = head_elems(out, dtype_size(L.dt), n);
    p.ntiles = tile_count(n, p.head, L.depth);
    p.ebase = ebase;
    // a forward chain moves c steps through its run, the backward Montgomery
    // chain c steps back, the one-product FP32 run's state not at all
    const bool digits = L.dt == DT_F32 && L.step == ST_SHARED && L.conv == CV_INT &&
                        L.chains == 1 && digit_run_depth(L.depth);
    const uint64_t stride = (L.step == ST_MONT) ? 33ull : digits ? 32ull : 31ull;
    p.jump = host_pow2((53ull * stride * L.depth) % kP);
    p.jump_q = host_mulmod_quotient(p.jump);
    // FP32 with the shared step on two chains runs the backward step
    const bool back = L.dt == DT_F32 && L.step == ST_SHARED && L.conv == CV_INT && L.chains == 2;
    p.jump_a = host_pow2((53ull * chain_jump_a(back, L.depth)) % kP);
    p.jump_aq = host_mulmod_quotient(p.jump_a);
    p.jump_b = host_pow2((53ull * chain_jump_b(back, L.depth)) % kP);
    p.jump_bq = host_mulmod_quotient(p.jump_b);
    p.cbits = const_bits;
    p.depth = L.depth;
    p.skip = (uint32_t)L.skip;
    p.nbuf = L.buffers;
    void* args[] = {&p};
    e = cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block), args, L.smem_bytes, cs);
  } else {
    DirectParams p;
    p.out = static_cast<unsigned char*>(out);
    p.n = n;
    p.ebase = ebase;
    p.cbits = const_bits;
    p.skip = (uint32_t)L.skip;
    void* args[] = {&p};
    e = cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block), args, 0, cs);
  }
  if (e != cudaSuccess) return cuda_error(e, "bulk kernel launch");
  return RNG_OK;
}

}  // namespace bcn
