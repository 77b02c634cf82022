// bcn_batch.cu -- many streams of uneven length in one persistent launch: the
// kernel (the plans, the allocation-free call and the launches are in
// bcn_batch_api.cu).
//
// A batch plan holds one descriptor per stream (exponent base, length, output
// pointer, element type), longest stream first, and cuts every stream into
// work units of unit_tiles tiles (32*depth elements each); the last unit of a
// stream may be short.  One persistent grid, sized to fill the GPU, pulls
// unit numbers from a device counter; a warp maps its unit to a stream by binary search over the
// prefix of unit counts, jumps every lane to its run (Eq. 2), and produces the
// unit's full tiles through the same shared-memory + bulk-copy path as the
// single-stream kernel, its short remainder with plain stores.  Unit 0 of a
// stream also writes the stream's head (elements before its first 16-byte
// boundary).  The counter is cleared by a memset node before each launch, so a
// plan can be replayed as a two-node CUDA graph.
//
// This follows the paper's parallel split (Sec. 1): every unit is a block of
// a stream reached by skip-ahead, so no result depends on which warp runs it.
#include "bcn_batch.cuh"
#include "bcn_digits.cuh"
#include "bcn_gen.cuh"

namespace bcn {

// The unit's elements [s0, s1) of stream d: full tiles by bulk copy, the
// remainder by plain stores; unit 0 also writes the head [0, head).
template <int DT, int STEP, int CONV, int ILP, int CDEPTH>
__device__ __forceinline__ void batch_unit(const BatchDesc& d, uint64_t k, const BatchParams& p,
                                           unsigned char* buf0_bytes, uint32_t& issued,
                                           uint32_t lane) {
  typedef typename Word<DT>::type W;
  W* const out = reinterpret_cast<W*>(d.out);
  const uint32_t c = CDEPTH > 0 ? (uint32_t)CDEPTH : p.depth[DT];
  const uint64_t tile_elems = 32ull * c;
  const uint64_t unit_elems = tile_elems * p.unit_tiles;
  const uint64_t s0 = d.head + k * unit_elems;
  const uint64_t s1 = min(s0 + unit_elems, d.n);
  if (k == 0)
    run_direct<DT, STEP, CONV>(out, d.ebase, p.skip, lane * d.head / 32,
                               (lane + 1) * d.head / 32, 0);
  if (s0 >= s1) return;
  const uint64_t ntiles = (s1 - s0) / tile_elems;
  if (ntiles > 0) {
    const uint64_t first = s0 + (uint64_t)lane * c;
    if constexpr (ILP == 2 && kDigitsF32<DT, STEP, CONV, CDEPTH>) {
      // each FP32 run from one product, from the state one past it
      warp_tiles_digits<CDEPTH>(out, s0, ntiles, p.ja[DT], p.jaq[DT],
                                state_of(d.ebase, first + c, p.skip),
                                reinterpret_cast<W*>(buf0_bytes), issued, lane, p.nbuf);
    } else if constexpr (ILP == 2) {
      Gen<DT, STEP, CONV> a{0}, b{0};
      lane_chains2<DT, STEP, CONV>(d.ebase, first, c, p.skip, a, b);
      warp_tiles2<DT, STEP, CONV, CDEPTH>(out, s0, ntiles, c, p.ja[DT], p.jaq[DT], p.jb[DT],
                                          p.jbq[DT], a, b, reinterpret_cast<W*>(buf0_bytes),
                                          issued, lane, p.nbuf);
    } else {
      Gen<DT, STEP, CONV> g = lane_chain<DT, STEP, CONV>(d.ebase, first, c, p.skip);
      warp_tiles<DT, STEP, CONV, CDEPTH>(out, s0, ntiles, c, p.jump, p.jump_q, g,
                                         reinterpret_cast<W*>(buf0_bytes), issued, lane, 0,
                                         p.nbuf);
    }
  }
  const uint64_t r0 = s0 + ntiles * tile_elems, rl = s1 - r0;
  run_direct<DT, STEP, CONV>(out, d.ebase, p.skip, r0 + lane * rl / 32, r0 + (lane + 1) * rl / 32,
                             0);
}

// C64, C32: compile-time tile depths of the FP64 and FP32 streams (0: the
// run-time depths); raw states always take their run-time depth.
template <int STEP, int CONV, int ILP, int C64, int C32>
__global__ void __launch_bounds__(1024) batch_kernel(const BatchParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5;
  // p.nbuf tile buffers per warp, each sized for the largest type's tile
  unsigned char* const buf0 = smem + (size_t)warp * p.nbuf * p.warp_bytes;
  uint32_t issued = 0;
  for (;;) {
    unsigned long long u = 0;
    if (lane == 0) u = atomicAdd(p.counter, 1ull);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= p.total_units) break;
    // stream s: prefix[s] <= u < prefix[s+1]
    uint32_t lo = 0, hi = p.nstreams;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(&p.prefix[mid]) <= u) lo = mid;
      else hi = mid;
    }
    const BatchDesc d = p.desc[lo];
    const uint64_t k = u - d.unit0;
    if (d.dt == DT_F64) batch_unit<DT_F64, STEP, CONV, ILP, C64>(d, k, p, buf0, issued, lane);
    else if (d.dt == DT_F32) batch_unit<DT_F32, STEP, CONV, ILP, C32>(d, k, p, buf0, issued, lane);
    else batch_unit<DT_U64, STEP, CONV, ILP, 0>(d, k, p, buf0, issued, lane);
  }
  if (lane == 0) bulk_wait_all();
  __syncwarp();
}

static const void* pick_batch(int st, int cv, int ilp, const uint32_t d[3]) {
  const bool same = d[DT_F64] == d[DT_F32] && d[DT_F64] == d[DT_U64];
  if (st == ST_SHARED && cv == CV_INT) {  // the production path: fixed depths
    if (ilp == 2) {
      if (batch_f32_digits(st, cv, ilp, d))
        return (const void*)batch_kernel<ST_SHARED, CV_INT, 2, kBatchDepthF64, kBatchDepthF32>;
      if (same && d[0] == 15) return (const void*)batch_kernel<ST_SHARED, CV_INT, 2, 15, 15>;
      if (same && d[0] == 31) return (const void*)batch_kernel<ST_SHARED, CV_INT, 2, 31, 31>;
      return (const void*)batch_kernel<ST_SHARED, CV_INT, 2, 0, 0>;
    }
    if (same && d[0] == 15) return (const void*)batch_kernel<ST_SHARED, CV_INT, 1, 15, 15>;
    if (same && d[0] == 31) return (const void*)batch_kernel<ST_SHARED, CV_INT, 1, 31, 31>;
    return (const void*)batch_kernel<ST_SHARED, CV_INT, 1, 0, 0>;
  }
  switch (st) {
    case ST_SHARED: return (const void*)batch_kernel<ST_SHARED, CV_FP64, 1, 0, 0>;
    case ST_BARRETT:
      if (ilp == 2) return cv == CV_FP64 ? (const void*)batch_kernel<ST_BARRETT, CV_FP64, 2, 0, 0>
                                         : (const void*)batch_kernel<ST_BARRETT, CV_INT, 2, 0, 0>;
      return cv == CV_FP64 ? (const void*)batch_kernel<ST_BARRETT, CV_FP64, 1, 0, 0>
                           : (const void*)batch_kernel<ST_BARRETT, CV_INT, 1, 0, 0>;
    case ST_MONT: return cv == CV_FP64 ? (const void*)batch_kernel<ST_MONT, CV_FP64, 1, 0, 0>
                                       : (const void*)batch_kernel<ST_MONT, CV_INT, 1, 0, 0>;
    default: return nullptr;
  }
}

const void* batch_kernel_fn(int step, int conv, int chains, const uint32_t d[3]) {
  return pick_batch(step, conv, chains, d);
}

}  // namespace bcn
