// bcn_m40.cu -- bulk generation for the larger-modulus variant (modulus 3^40,
// Sec. 1; arithmetic in bcn_math40.cuh) on sm_103a.
//
// Layout and data movement are those of the 3^33 tiled kernel: the output
// is cut into tiles of 32*c elements (c odd), each warp owns a contiguous
// range of tiles, lane l of a tile produces its elements [l*c, (l+1)*c) into
// the warp's shared-memory tile buffer, and one lane hands the tile to the
// bulk async-copy engine.  Head (before the first 16-byte boundary) and tail
// (less than a tile) are stored directly by the grid's last warp.
//
// Per variate: one quotient floor(2^53 z / 3^40) (three 64-bit partial
// products), one remainder (one product), and a shift-and-or that joins two
// consecutive quotients into the truncated FP64 variate.  A chain therefore
// runs one quotient ahead of the variate it emits: it holds the state after
// the next variate's state and that variate's quotient.
#include "bcn_gen.cuh"
#include "bcn_m40.cuh"
#include "bcn_math40.cuh"

namespace bcn {

// One chain.  Variates (F64/F32): z is the state after the next variate's
// state, q the next variate's quotient.  States (U64): z is the next state.
template <int DT>
struct Chain40 {
  uint64_t z, q;
  // Begin at the variate whose state is s.
  __device__ __forceinline__ void start(uint64_t s) {
    if constexpr (DT == DT_U64) {
      z = s;
    } else {
      q = quot40(s);
      z = rem40(s, q);
    }
  }
  // A variate by the fast quotient and conversion (F64/F32 only).  qmin
  // tracks the smallest high word of the quotients used as a variate's
  // leading window (0 means a variate below 2^-21); fmax the largest high
  // word of the estimates' fractions (>= 0xFFFFFFFC means undecided).
  __device__ __forceinline__ typename Word<DT>::type next_fast(uint32_t& qmin, uint32_t& fmax) {
    uint32_t fhi;
    const uint64_t q1 = quot40_fast(z, fhi);
    fmax = max(fmax, fhi);
    const uint64_t bits = bits40_fast(q, q1);
    z = rem40(z, q1);
    q = q1;
    qmin = min(qmin, (uint32_t)(q1 >> 32));
    if constexpr (DT == DT_F64) return bits;
    else return f32_bits_from_f64_bits(bits);
  }
  __device__ __forceinline__ typename Word<DT>::type next() {
    if constexpr (DT == DT_U64) {
      const uint64_t w = z;
      z = rem40(z, quot40(z));
      return w;
    } else {
      const uint64_t q1 = quot40(z);
      const uint64_t bits = q != 0 ? bits40(q, q1) : bits40_small(z, q1);
      z = rem40(z, q1);
      q = q1;
      if constexpr (DT == DT_F64) return bits;
      else return f32_bits_from_f64_bits(bits);
    }
  }
};

// Steps between what a chain holds after emitting the variate before index
// i and the state of variate i: one for variates (the look-ahead), none for
// states.
template <int DT>
constexpr uint64_t kAhead40 = DT == DT_U64 ? 0 : 1;

__device__ __forceinline__ uint64_t state_of40(uint64_t ebase, uint64_t idx) {
  return seed_state40(exponent_add40(ebase, idx + 1));
}

template <int DT>
__device__ void run_direct40(typename Word<DT>::type* __restrict__ out, uint64_t ebase,
                             uint64_t a, uint64_t b) {
  if (a >= b) return;
  Chain40<DT> g;
  g.start(state_of40(ebase, a));
  for (uint64_t i = a; i < b; ++i) out[i] = g.next();
}

template <int DT, int ILP, int CDEPTH>
__global__ void __launch_bounds__(1024) tiled40_kernel(const M40Params p) {
  typedef typename Word<DT>::type W;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t wpb = blockDim.x >> 5;
  const uint64_t gw = (uint64_t)blockIdx.x * wpb + warp;
  const uint64_t nw = (uint64_t)gridDim.x * wpb;
  const uint32_t c = CDEPTH > 0 ? (uint32_t)CDEPTH : p.depth;
  const uint32_t tile_elems = 32u * c;
  const uint32_t tile_bytes = tile_elems * (uint32_t)sizeof(W);
  W* const buf0 = reinterpret_cast<W*>(smem + (size_t)warp * p.nbuf * tile_elems * sizeof(W));
  W* const out = reinterpret_cast<W*>(p.out);

  const uint64_t t0 = gw * p.ntiles / nw;
  const uint64_t t1 = (gw + 1) * p.ntiles / nw;
  if (t0 < t1) {
    const uint64_t first = p.head + t0 * tile_elems + (uint64_t)lane * c;
    const uint32_t h = c >> 1;
    Chain40<DT> a, b;
    a.start(state_of40(p.ebase, first));
    if constexpr (ILP == 2) b.start(state_of40(p.ebase, first + h + 1));
    uint32_t issued = 0;
    for (uint64_t t = t0; t < t1; ++t) {
      W* const buf = buf0 + (issued % p.nbuf) * tile_elems;
      wait_buffer_free(issued, p.nbuf, lane);
      W* const mine = buf + lane * c;
      if constexpr (DT == DT_U64) {
        if constexpr (ILP == 2) {
#pragma unroll
          for (uint32_t i = 0; i < (CDEPTH > 0 ? (uint32_t)CDEPTH / 2 : h); ++i) {
            mine[i] = a.next();
            mine[h + 1 + i] = b.next();
          }
          mine[h] = a.next();
        } else {
#pragma unroll
          for (uint32_t i = 0; i < (CDEPTH > 0 ? (uint32_t)CDEPTH : c); ++i) mine[i] = a.next();
        }
      } else {
        // fast path for the whole run; a lane whose run met an undecided
        // quotient or a variate below 2^-21 redoes it exactly
        const Chain40<DT> a0 = a, b0 = b;
        uint32_t qmin = (uint32_t)(a.q >> 32), fmax = 0;
        if constexpr (ILP == 2) {
          qmin = min(qmin, (uint32_t)(b.q >> 32));
#pragma unroll
          for (uint32_t i = 0; i < (CDEPTH > 0 ? (uint32_t)CDEPTH / 2 : h); ++i) {
            mine[i] = a.next_fast(qmin, fmax);
            mine[h + 1 + i] = b.next_fast(qmin, fmax);
          }
          mine[h] = a.next_fast(qmin, fmax);
        } else {
#pragma unroll
          for (uint32_t i = 0; i < (CDEPTH > 0 ? (uint32_t)CDEPTH : c); ++i)
            mine[i] = a.next_fast(qmin, fmax);
        }
        const bool rare = qmin == 0 || fmax >= 0xFFFFFFFCu;
        if (__any_sync(0xffffffffu, rare)) {
          if (rare) {
            a = a0;
            b = b0;
            if constexpr (ILP == 2) {
              for (uint32_t i = 0; i < h; ++i) {
                mine[i] = a.next();
                mine[h + 1 + i] = b.next();
              }
              mine[h] = a.next();
            } else {
              for (uint32_t i = 0; i < c; ++i) mine[i] = a.next();
            }
          }
          __syncwarp();
        }
      }
      fence_proxy_async_shared();
      __syncwarp();
      if (lane == 0) {
        bulk_store(out + p.head + t * tile_elems, buf, tile_bytes);
        bulk_commit();
      }
      ++issued;
      if (t + 1 < t1) {
        if constexpr (ILP == 2) {
          a.start(mont40(a.z, p.jump_a));
          b.start(mont40(b.z, p.jump_b));
        } else {
          a.start(mont40(a.z, p.jump));
        }
      }
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }

  if (gw == nw - 1) {  // head and tail, split contiguously over the lanes
    const uint64_t tail0 = p.head + p.ntiles * tile_elems;
    const uint64_t tl = p.n - tail0;
    run_direct40<DT>(out, p.ebase, lane * p.head / 32, (lane + 1) * p.head / 32);
    run_direct40<DT>(out, p.ebase, tail0 + lane * tl / 32, tail0 + (lane + 1) * tl / 32);
  }
}

template <int DT>
__global__ void __launch_bounds__(1024) direct40_kernel(unsigned char* out, uint64_t n,
                                                        uint64_t ebase) {
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t a = (uint64_t)((u128)n * t / T);
  const uint64_t b = (uint64_t)((u128)n * (t + 1) / T);
  run_direct40<DT>(reinterpret_cast<typename Word<DT>::type*>(out), ebase, a, b);
}

template <int DT>
static const void* pick40_dt(int layout, uint32_t chains, uint32_t depth) {
  if (layout == RNG_LAYOUT_DIRECT) return (const void*)direct40_kernel<DT>;
  if (chains == 2) {
    if (depth == 15) return (const void*)tiled40_kernel<DT, 2, 15>;
    if (depth == 31) return (const void*)tiled40_kernel<DT, 2, 31>;
    return (const void*)tiled40_kernel<DT, 2, 0>;
  }
  if (depth == 15) return (const void*)tiled40_kernel<DT, 1, 15>;
  if (depth == 31) return (const void*)tiled40_kernel<DT, 1, 31>;
  return (const void*)tiled40_kernel<DT, 1, 0>;
}

const void* pick40(int dt, int layout, uint32_t chains, uint32_t depth) {
  switch (dt) {
    case DT_F64: return pick40_dt<DT_F64>(layout, chains, depth);
    case DT_F32: return pick40_dt<DT_F32>(layout, chains, depth);
    case DT_U64: return pick40_dt<DT_U64>(layout, chains, depth);
    default: return nullptr;
  }
}

}  // namespace bcn
