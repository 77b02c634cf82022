// bcn_bulk.cu -- bulk generation kernels for one stream (sm_103a).
//
// TILED layout (the fast path).  Output elements [head, head + ntiles*32*c)
// are cut into tiles of 32*c elements (c = depth, odd).  Each warp owns a
// contiguous range of tiles; in a tile, lane l owns elements [l*c, (l+1)*c)
// and produces them with c consecutive steps of Eq. 3 from one state, so the
// per-variate work is one reduction and one conversion.  Lanes write their
// runs to a per-warp shared-memory tile (odd c makes the 8-byte and 4-byte
// stores bank-conflict free), and one lane hands the whole tile to the bulk
// async-copy engine (cp.async.bulk shared::cta -> global), so global memory
// sees one contiguous, 16-byte aligned write per tile with no per-thread
// store instructions.  A warp keeps one or two tile buffers: with two, the
// copy of one tile overlaps the generation of the next; with one (the
// measured choice at depth 31), the warp waits for its last copy to finish
// reading before refilling, and twice as many warps fit per SM to cover the
// wait.  Moving from a tile to the warp's next tile is one modular product by
// a precomputed power of 2^53.
//
// DIRECT layout (the paper's per-thread split, Sec. 1): thread t of T owns
// [t*n/T, (t+1)*n/T) and stores each variate itself.  It serves odd thread
// counts (down to one thread) and is the uncoalesced baseline.
//
// The head (elements before the first 16-byte boundary) and the tail (fewer
// than one tile) are produced by the last warp of the grid with direct
// stores.  Every element's value depends only on its index, so the result is
// identical for every layout, depth, block and grid.
#include <mutex>
#include <set>
#include <utility>

#include "bcn_gen.cuh"

namespace bcn {

struct TiledParams {
  unsigned char* out;  // element 0 of the call
  uint64_t n;          // elements in the call
  uint64_t head;       // elements before the first 16-byte boundary
  uint64_t ntiles;     // full tiles of 32*depth elements after the head
  uint64_t ebase;      // (seed - 3^33 + 53*i0) mod P
  uint64_t jump;       // 2^(53*31*depth) (Barrett) / 2^(53*33*depth) (Montgomery)
  uint64_t jump_q;     // floor(jump * 2^64 / m), for the precomputed-quotient product
  uint64_t jump_a;     // two chains: 2^(53*(32c-h-1)) and 2^(53*(31c+h+1)), h = depth/2
  uint64_t jump_aq;
  uint64_t jump_b;
  uint64_t jump_bq;
  uint64_t cbits;      // ST_CONST: the word written
  uint32_t depth;
  uint32_t skip;
  uint32_t nbuf;       // tile buffers per warp (1 or 2)
};

struct DirectParams {
  unsigned char* out;
  uint64_t n;
  uint64_t ebase;
  uint64_t cbits;
  uint32_t skip;
};

template <int DT, int STEP, int CONV, int ILP, int CDEPTH = 0>
__global__ void __launch_bounds__(1024) tiled_kernel(const TiledParams p) {
  typedef typename Word<DT>::type W;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t wpb = blockDim.x >> 5;
  const uint64_t gw = (uint64_t)blockIdx.x * wpb + warp;
  const uint64_t nw = (uint64_t)gridDim.x * wpb;
  const uint32_t c = CDEPTH > 0 ? (uint32_t)CDEPTH : p.depth;
  const uint32_t tile_elems = 32u * c;
  W* const buf0 = reinterpret_cast<W*>(smem + (size_t)warp * p.nbuf * tile_elems * sizeof(W));
  W* const out = reinterpret_cast<W*>(p.out);

  const uint64_t t0 = gw * p.ntiles / nw;
  const uint64_t t1 = (gw + 1) * p.ntiles / nw;
  if (t0 < t1) {
    // this lane's first element in the warp's first tile
    const uint64_t first = p.head + t0 * tile_elems + (uint64_t)lane * c;
    uint32_t issued = 0;
    if constexpr (ILP == 2) {
      Gen<DT, STEP, CONV> a = lane_chain<DT, STEP, CONV>(p.ebase, first, c, p.skip);
      Gen<DT, STEP, CONV> b = lane_chain<DT, STEP, CONV>(p.ebase, first + c / 2 + 1, c, p.skip);
      warp_tiles2<DT, STEP, CONV, CDEPTH>(out, p.head + t0 * tile_elems, t1 - t0, c, p.jump_a,
                                          p.jump_aq, p.jump_b, p.jump_bq, a, b, buf0, issued,
                                          lane, p.nbuf);
    } else {
      Gen<DT, STEP, CONV> g = lane_chain<DT, STEP, CONV>(p.ebase, first, c, p.skip);
      warp_tiles<DT, STEP, CONV, CDEPTH>(out, p.head + t0 * tile_elems, t1 - t0, c, p.jump,
                                         p.jump_q, g, buf0, issued, lane, p.cbits, p.nbuf);
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }

  if (gw == nw - 1) {  // head and tail, split contiguously over the lanes
    const uint64_t tail0 = p.head + p.ntiles * tile_elems;
    const uint64_t tl = p.n - tail0;
    run_direct<DT, STEP, CONV>(out, p.ebase, p.skip, lane * p.head / 32,
                               (lane + 1) * p.head / 32, p.cbits);
    run_direct<DT, STEP, CONV>(out, p.ebase, p.skip, tail0 + lane * tl / 32,
                               tail0 + (lane + 1) * tl / 32, p.cbits);
  }
}

template <int DT, int STEP, int CONV>
__global__ void __launch_bounds__(1024) direct_kernel(const DirectParams p) {
  typedef typename Word<DT>::type W;
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t a = (uint64_t)((u128)p.n * t / T);
  const uint64_t b = (uint64_t)((u128)p.n * (t + 1) / T);
  run_direct<DT, STEP, CONV>(reinterpret_cast<W*>(p.out), p.ebase, p.skip, a, b, p.cbits);
}

// ------------------------------------------------------------ dispatch
template <int DT, int ST, int CV>
static const void* pick_ilp(int layout, int ilp, uint32_t depth) {
  if (layout != RNG_LAYOUT_TILED) return (const void*)direct_kernel<DT, ST, CV>;
  // the production path gets tile depths fixed at compile time (full unroll)
  if constexpr (ST == ST_SHARED && CV == CV_INT && DT != DT_U64) {
    if (ilp == 2) {
      if (depth == 9) return (const void*)tiled_kernel<DT, ST, CV, 2, 9>;
      if (depth == 15) return (const void*)tiled_kernel<DT, ST, CV, 2, 15>;
      if (depth == 31) return (const void*)tiled_kernel<DT, ST, CV, 2, 31>;
    }
  }
  if constexpr (ST == ST_BARRETT || ST == ST_SHARED)
    if (ilp == 2) return (const void*)tiled_kernel<DT, ST, CV, 2>;
  if constexpr (ST == ST_SHARED && CV == CV_INT && DT != DT_U64) {
    if (depth == 9) return (const void*)tiled_kernel<DT, ST, CV, 1, 9>;
    if (depth == 15) return (const void*)tiled_kernel<DT, ST, CV, 1, 15>;
    if (depth == 31) return (const void*)tiled_kernel<DT, ST, CV, 1, 31>;
  }
  return (const void*)tiled_kernel<DT, ST, CV, 1>;
}

template <int DT, int ST>
static const void* pick_cv(int layout, int cv, int ilp, uint32_t depth) {
  return cv == CV_FP64 ? pick_ilp<DT, ST, CV_FP64>(layout, ilp, depth)
                       : pick_ilp<DT, ST, CV_INT>(layout, ilp, depth);
}

template <int DT>
static const void* pick_st(int layout, int st, int cv, int ilp, uint32_t depth) {
  if (DT == DT_U64) cv = CV_INT;  // no conversion for raw states
  switch (st) {
    case ST_BARRETT: return pick_cv<DT, ST_BARRETT>(layout, cv, ilp, depth);
    case ST_MONT: return pick_cv<DT, ST_MONT>(layout, cv, 1, depth);
    case ST_SHARED: return pick_cv<DT, ST_SHARED>(layout, cv, ilp, depth);
    case ST_LECUYER: return pick_cv<DT, ST_LECUYER>(layout, cv, 1, depth);
    case ST_BCLASSIC: return pick_cv<DT, ST_BCLASSIC>(layout, cv, 1, depth);
    default: return nullptr;
  }
}

static const void* pick_kernel(int layout, int dt, int st, int cv, int ilp, uint32_t depth) {
  if (st == ST_CONST) {
    if (dt == DT_F64) return layout == RNG_LAYOUT_TILED
                                 ? (const void*)tiled_kernel<DT_F64, ST_CONST, CV_INT, 1>
                                 : (const void*)direct_kernel<DT_F64, ST_CONST, CV_INT>;
    if (dt == DT_F32) return layout == RNG_LAYOUT_TILED
                                 ? (const void*)tiled_kernel<DT_F32, ST_CONST, CV_INT, 1>
                                 : (const void*)direct_kernel<DT_F32, ST_CONST, CV_INT>;
    return nullptr;
  }
  switch (dt) {
    case DT_F64: return pick_st<DT_F64>(layout, st, cv, ilp, depth);
    case DT_F32: return pick_st<DT_F32>(layout, st, cv, ilp, depth);
    case DT_U64: return pick_st<DT_U64>(layout, st, cv, ilp, depth);
    default: return nullptr;
  }
}

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
// (FP64 752, FP32 719, raw states 820 G/s there, against 573, 628 and 704
// with 15-deep tiles in 256-thread blocks).
constexpr uint32_t kDefDepth = 31, kDefBlock = 896, kDefChains = 2, kDefBuffers = 1;

rng_status resolve_bulk(uint64_t n, int dt, const rng_tune* tune, BulkLaunch* out,
                        bool constant) {
  rng_tune t = {};
  if (tune) t = *tune;
  if (!constant) {  // zero fields take the installed (measured) defaults
    const rng_tune d = auto_defaults(dt);
    const bool same_layout = !t.layout || !d.layout || t.layout == d.layout;
    if (!t.step) t.step = d.step;
    if (!t.conv) t.conv = d.conv;
    if (!t.skip) t.skip = d.skip;
    if (same_layout) {
      if (!t.layout) t.layout = d.layout;
      if (!t.depth) t.depth = d.depth;
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
  if (L.layout != RNG_LAYOUT_TILED && L.layout != RNG_LAYOUT_DIRECT)
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
  L.chains = 1;
  const uint32_t want_chains = t.chains ? t.chains : kDefChains;
  if (L.layout == RNG_LAYOUT_TILED && (L.step == ST_SHARED || L.step == ST_BARRETT) &&
      want_chains == 2 && (t.depth ? t.depth : kDefDepth) >= 3)
    L.chains = 2;
  const uint32_t depth0 = L.layout == RNG_LAYOUT_TILED ? (t.depth ? t.depth : kDefDepth) : 0;
  const void* fn = pick_kernel(L.layout, dt, L.step, L.conv, (int)L.chains, depth0);
  if (!fn) return set_error(RNG_EINVAL, "no kernel for this combination");
  if (L.layout == RNG_LAYOUT_TILED) {
    L.depth = t.depth ? t.depth : kDefDepth;
    L.block = t.block ? t.block : kDefBlock;
    if (L.depth % 2 == 0 || L.depth > kMaxDepth)
      return set_error(RNG_EINVAL, "tune.depth %u must be odd and at most %u", L.depth,
                       kMaxDepth);
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
  const void* fn = pick_kernel(L.layout, L.dt, L.step, L.conv, (int)L.chains, L.depth);
  if (!fn) return set_error(RNG_EINVAL, "no kernel for this combination");
  const uint64_t ebase = (L.step == ST_CONST) ? 0 : host_exponent_base(seed, i0);
  cudaError_t e;
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
    const uint64_t stride = (L.step == ST_MONT) ? 33ull : 31ull;
    p.jump = host_pow2((53ull * stride * L.depth) % kP);
    p.jump_q = host_mulmod_quotient(p.jump);
    const uint64_t h = L.depth / 2;
    p.jump_a = host_pow2((53ull * (32ull * L.depth - h - 1)) % kP);
    p.jump_aq = host_mulmod_quotient(p.jump_a);
    p.jump_b = host_pow2((53ull * (31ull * L.depth + h + 1)) % kP);
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
