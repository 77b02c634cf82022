// bcn_strided.cu -- the paper's coalesced kernels (Sec. 2.2).
//
// The paper makes its global writes coalesced by spacing each thread's
// outputs `step` apart, step being the number of threads: thread t of T
// produces the consecutive variates t*W .. t*W+W-1 of the call (its block of
// the sequence, reached by skip-ahead, Sec. 1) and writes variate t*W+j to
// position j*T+t, so the T threads' j-th outputs fill T consecutive
// positions.  The array then holds a permutation of the sequence.  Its
// "Unrolled" kernels unroll the generation loop by eight (Sec. 2.2's
// partial-unrolling listing).  These kernels reproduce that protocol on this
// GPU; the library's own in-order path is the tiled layout.
#include "bcn_gen.cuh"
#include "bcn_strided.cuh"

namespace bcn {

template <int DT, int STEP, int CONV, int UNROLL>
__global__ void __launch_bounds__(1024) strided_kernel(const StridedParams p) {
  typedef typename Word<DT>::type W;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.nthreads) return;
  W* const out = reinterpret_cast<W*>(p.out);
  const uint64_t T = p.nthreads, per = p.per;
  if constexpr (STEP == ST_CONST) {
#pragma unroll UNROLL
    for (uint64_t j = 0; j < per; ++j) out[j * T + t] = (W)p.cbits;
  } else if constexpr (STEP != ST_MONT) {
    Gen<DT, STEP, CONV> g{state_of(p.ebase, t * per, p.skip)};
#pragma unroll UNROLL
    for (uint64_t j = 0; j < per; ++j) out[j * T + t] = g.next();
  } else {  // the Montgomery step runs backwards from the block's last variate
    Gen<DT, STEP, CONV> g{state_of(p.ebase, t * per + per - 1, p.skip)};
#pragma unroll UNROLL
    for (uint64_t j = per; j-- > 0;) out[j * T + t] = g.next();
  }
}

template <int DT, int ST, int CV>
static const void* pick_unroll(uint32_t unroll) {
  return unroll == 1 ? (const void*)strided_kernel<DT, ST, CV, 1>
                     : (const void*)strided_kernel<DT, ST, CV, 8>;
}

template <int DT, int ST>
static const void* pick_cv(int cv, uint32_t unroll) {
  if (DT == DT_U64 || cv != CV_FP64) return pick_unroll<DT, ST, CV_INT>(unroll);
  return pick_unroll<DT, ST, CV_FP64>(unroll);
}

template <int DT>
static const void* pick_st(int st, int cv, uint32_t unroll) {
  switch (st) {
    case ST_BARRETT: return pick_cv<DT, ST_BARRETT>(cv, unroll);
    case ST_MONT: return pick_cv<DT, ST_MONT>(cv, unroll);
    case ST_SHARED: return pick_cv<DT, ST_SHARED>(cv, unroll);
    case ST_LECUYER: return pick_cv<DT, ST_LECUYER>(cv, unroll);
    case ST_BCLASSIC: return pick_cv<DT, ST_BCLASSIC>(cv, unroll);
    default: return nullptr;
  }
}

const void* pick_strided(int dt, int st, int cv, uint32_t unroll) {
  if (st == ST_CONST) {
    if (dt == DT_F64) return pick_unroll<DT_F64, ST_CONST, CV_INT>(unroll);
    if (dt == DT_F32) return pick_unroll<DT_F32, ST_CONST, CV_INT>(unroll);
    return nullptr;
  }
  switch (dt) {
    case DT_F64: return pick_st<DT_F64>(st, cv, unroll);
    case DT_F32: return pick_st<DT_F32>(st, cv, unroll);
    case DT_U64: return pick_st<DT_U64>(st, cv, unroll);
    default: return nullptr;
  }
}

}  // namespace bcn
