// bcn_bulk.cu -- bulk generation kernels for one stream (sm_103a).
//
// TILED layout (the fast path).  Output elements [head, head + ntiles*32*c)
// are cut into tiles of 32*c elements (c = depth: odd, or 4 mod 8 for the
// backward FP32 runs, which store four variates at a time, or 2 mod 4 for the
// forward FP64 runs on two chains, which store two).  Each warp owns a
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
// than one tile) are produced with direct stores by the grid's last warps.
// Every element's value depends only on its index, so the result is
// identical for every layout, depth, block and grid.
#include "bcn_bulk.cuh"
#include "bcn_digits.cuh"
#include "bcn_gen.cuh"

namespace bcn {

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
      Gen<DT, STEP, CONV> a{0}, b{0};
      lane_chains2<DT, STEP, CONV>(p.ebase, first, c, p.skip, a, b);
      warp_tiles2<DT, STEP, CONV, CDEPTH>(out, p.head + t0 * tile_elems, t1 - t0, c, p.jump_a,
                                          p.jump_aq, p.jump_b, p.jump_bq, a, b, buf0, issued,
                                          lane, p.nbuf);
    } else if constexpr (kDigitsF32<DT, STEP, CONV, CDEPTH>) {
      // each FP32 run from one product, starting from the state one past it
      warp_tiles_digits<CDEPTH>(out, p.head + t0 * tile_elems, t1 - t0, p.jump, p.jump_q,
                                state_of(p.ebase, first + c, p.skip), buf0, issued, lane,
                                p.nbuf);
    } else {
      Gen<DT, STEP, CONV> g = lane_chain<DT, STEP, CONV>(p.ebase, first, c, p.skip);
      warp_tiles<DT, STEP, CONV, CDEPTH>(out, p.head + t0 * tile_elems, t1 - t0, c, p.jump,
                                         p.jump_q, g, buf0, issued, lane, p.cbits, p.nbuf);
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }

  // The tail (less than one tile) is spread over the grid's last warps, at
  // most four elements per lane, so that no warp's exact single-chain steps
  // outlast the tiles (a 640-element tail on one warp added about a microsecond
  // to a 10^6-variate call); the head (under 16 bytes) goes to the last warp.
  const uint64_t tail0 = p.head + p.ntiles * tile_elems;
  const uint64_t tl = p.n - tail0;
  const uint64_t wt = min(nw, (tl + 127) / 128);
  if (gw + wt >= nw) {
    const uint64_t k = gw - (nw - wt);
    const uint64_t lo = tail0 + k * tl / wt, len = tail0 + (k + 1) * tl / wt - lo;
    run_direct<DT, STEP, CONV>(out, p.ebase, p.skip, lo + lane * len / 32,
                               lo + (lane + 1) * len / 32, p.cbits);
  }
  if (gw == nw - 1)
    run_direct<DT, STEP, CONV>(out, p.ebase, p.skip, lane * p.head / 32,
                               (lane + 1) * p.head / 32, p.cbits);
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
      if constexpr (DT == DT_F64) {  // two variates per shared-memory store
        if (depth == 30) return (const void*)tiled_kernel<DT, ST, CV, 2, 30>;
      }
      if constexpr (DT == DT_F32) {  // FP32 tiles are half the bytes: deeper ones fit
        if (depth == 44) return (const void*)tiled_kernel<DT, ST, CV, 2, 44>;
        if (depth == 47) return (const void*)tiled_kernel<DT, ST, CV, 2, 47>;
        if (depth == 63) return (const void*)tiled_kernel<DT, ST, CV, 2, 63>;
      }
    }
  }
  if constexpr (ST == ST_BARRETT || ST == ST_SHARED)
    if (ilp == 2) return (const void*)tiled_kernel<DT, ST, CV, 2>;
  if constexpr (ST == ST_SHARED && CV == CV_INT && DT != DT_U64) {
    if constexpr (DT == DT_F32) {  // each run from one product (digit_run_f32)
      if (depth == 44) return (const void*)tiled_kernel<DT, ST, CV, 1, 44>;
    }
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

const void* pick_kernel(int layout, int dt, int st, int cv, int ilp, uint32_t depth) {
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

}  // namespace bcn
