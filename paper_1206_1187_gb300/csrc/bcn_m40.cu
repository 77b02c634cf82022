// bcn_m40.cu -- bulk generation for the larger-modulus variant (modulus 3^40,
// Sec. 1; arithmetic in bcn_math40.cuh) on sm_103a.
//
// Layout and data movement are those of the 3^33 tiled kernel: the output
// is cut into tiles of 32*c elements (c odd, or 44 for FP32 runs made from
// one product), each warp owns a contiguous
// range of tiles, lane l of a tile produces its elements [l*c, (l+1)*c) into
// the warp's shared-memory tile buffer, and one lane hands the tile to the
// bulk async-copy engine.  Head (before the first 16-byte boundary) and tail
// (less than a tile) are stored directly by the grid's last warp.
//
// Per variate: one step of Eq. 3 run backwards (back40), which gives the
// previous state together with its exact quotient digit floor(2^53 z / 3^40),
// and a shift-and-or that joins two consecutive digits into the truncated
// FP64 variate.  Lanes walk their runs from the end down, so a chain holds,
// besides its state, the digit of the state above the variate it emits next.
// The head and tail, and runs holding a variate below 2^-21, are made forward
// with the exact quotient.
#include "bcn_digits.cuh"
#include "bcn_gen.cuh"
#include "bcn_m40.cuh"
#include "bcn_math40.cuh"

namespace bcn {

// One forward chain with the exact quotient (head, tail and the rare runs).
// Variates (F64/F32): z is the state after the next variate's state, q the
// next variate's quotient.  States (U64): z is the next state.
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

// One chain run backwards (back40): z is one step past the next state to
// emit, q (variates only) the quotient digit of z.  A step back gives the
// previous state and its digit, which leads the variate emitted; z's own
// digit continues it.  Every digit is exact, so only variates below 2^-21
// (leading digit's high word zero) leave the fast conversion.
template <int DT>
struct Back40 {
  uint64_t z, q;
  // Begin with the state s one past (variates: two past) the first element
  // emitted; for variates one step back gives the digit of the state above.
  __device__ __forceinline__ void start(uint64_t s) {
    z = s;
    if constexpr (DT != DT_U64) z = back40(z, q);
  }
  __device__ __forceinline__ typename Word<DT>::type next(uint32_t& qmin) {
    uint64_t u;
    const uint64_t zp = back40(z, u);
    z = zp;
    if constexpr (DT == DT_U64) {
      return zp;
    } else {
      const uint64_t bits = bits40_fast(u, q);
      qmin = min(qmin, (uint32_t)(u >> 32));
      q = u;
      if constexpr (DT == DT_F64) return bits;
      else return f32_bits_from_f64_bits(bits);
    }
  }
};

__device__ __forceinline__ uint64_t state_of40(uint64_t ebase, uint64_t idx) {
  return seed_state40(exponent_add40(ebase, idx + 1));
}

// ------------------------------------------- FP32 runs from one product
// The identity behind the 3^33 kernel's one-product runs holds for 3^40 as
// well (back40's step is the same reduction): the digits q of the C states
// before z are the 53-bit fields of z N mod 2^(53C), N = -3^-40 mod 2^(53C),
// field i being the digit of element C - 1 - i, and the bits below a field
// are the next element's digit, i.e. the continuation of the expansion.
// The FP32 variate truncates z/3^40 to 24 significant bits, so it is read
// from a field with no rounding question at all: Q's leading 24 bits, which
// lie inside the field whenever Q >= 2^23 (a run with a smaller digit,
// probability about 2^-30 per variate, is redone by its lane with the exact
// forward chain).  Runs of 44 (4 mod 8, the FP32 default) store four
// variates per 16-byte shared-memory store, odd runs one at a time.
static_assert((make_neg_minv_words<2, k40M>().w[0] |
               ((uint64_t)make_neg_minv_words<2, k40M>().w[1] << 32)) == k40NegMinv,
              "-3^-40 mod 2^64");

// Word I of z N for a full 64-bit state z = (z1:z0).  V = (v1:v0), the part
// of the lower words' sum above word I - 1, stays below 2^34 (v1 <= 3);
// x = V + z1 N_(I-1) can pass 2^64, so it takes a third word (x2 <= 1), and
// x + z0 N_I gives word I and the next V.  Four 32-bit multiply-adds and two
// adds per word.
template <int W, int I>
__device__ __forceinline__ void run40_product_word(uint32_t z0, uint32_t z1, uint32_t& r,
                                                   uint32_t& v0, uint32_t& v1) {
  constexpr uint32_t nI = RunMinv<W, k40M>::t.w[I];
  if constexpr (I == 0) {
    r = z0 * nI;
    v0 = __umulhi(z0, nI);
    v1 = 0;
  } else if constexpr (I == W - 1) {  // the top word: no carry out
    constexpr uint32_t nP = RunMinv<W, k40M>::t.w[I - 1];
    asm("{\n\t"
        ".reg .u32 x0;\n\t"
        "mad.lo.u32 x0, %3, %5, %1;\n\t"
        "mad.lo.u32 %0, %2, %4, x0;\n\t"
        "}"
        : "=r"(r)
        : "r"(v0), "r"(z0), "r"(z1), "n"(nI), "n"(nP));
  } else {
    constexpr uint32_t nP = RunMinv<W, k40M>::t.w[I - 1];
    // r is early-clobber: it must not share a register with z0
    asm("{\n\t"
        ".reg .u32 x0, x1, x2;\n\t"
        "mad.lo.cc.u32 x0, %4, %6, %1;\n\t"   // x = V + z1 N_(I-1), three words
        "madc.hi.cc.u32 x1, %4, %6, %2;\n\t"
        "addc.u32 x2, 0, 0;\n\t"
        "mad.lo.cc.u32 %0, %3, %5, x0;\n\t"   // x + z0 N_I: word I ...
        "madc.hi.cc.u32 %1, %3, %5, x1;\n\t"  // ... and the next V
        "addc.u32 %2, x2, 0;\n\t"
        "}"
        : "=&r"(r), "+r"(v0), "+r"(v1)
        : "r"(z0), "r"(z1), "n"(nI), "n"(nP));
  }
}

// FP32 bits of the truncated variate from X = (u1:u0), the field's digit Q
// times 2^11 followed by the next digit's top 11 bits: with c the leading
// zeros of u1 (Q >= 2^23: c <= 29), Q's leading 24 bits W = (X << c) >> 40
// and the exponent 126 - c, i.e. W + (125 - c) 2^23.
__device__ __forceinline__ uint32_t f32_from_digit_words40(uint32_t u1, uint32_t u0) {
  uint32_t b;
  asm("{\n\t"
      ".reg .u32 c, mant, e;\n\t"
      "bfind.shiftamt.u32 c, %1;\n\t"
      "shf.l.clamp.b32 mant, %2, %1, c;\n\t"
      "shr.b32 mant, mant, 8;\n\t"
      "mad.lo.u32 e, c, 0xFF800000, 0x3E800000;\n\t"
      "add.u32 %0, mant, e;\n\t"
      "}"
      : "=r"(b)
      : "r"(u1), "r"(u0));
  return b;
}

template <int C>
struct DigitRun40 : DigitGeometry<C> {
  // 2^(-53C) mod 3^40 in Montgomery form: one past the run -> element 0
  static constexpr uint64_t back =
      host40_mont_form(host40_pow2((k40P - (53ull * C) % k40P) % k40P));
};

template <int C, int I>
__device__ __forceinline__ void digit_run40_word(uint32_t z0, uint32_t z1,
                                                 uint32_t (&r)[DigitRun40<C>::W], uint32_t& v0,
                                                 uint32_t& v1, uint32_t (&d)[4], uint32_t* mine,
                                                 uint32_t& qmin) {
  run40_product_word<DigitRun40<C>::W, I>(z0, z1, r[I], v0, v1);
  constexpr int i = DigitRun40<C>::digit_of_word(I);
  if constexpr (i >= 0) {
    const uint32_t u1 = run_bits32<53 * i + 21>(r);
    const uint32_t u0 = run_bits32<53 * i - 11>(r);  // field 0: zeros below, unread
    qmin = min(qmin, u1);
    if constexpr (vec4_depth(C)) {  // four variates per 16-byte store
      d[i % 4] = f32_from_digit_words40(u1, u0);
      if constexpr (i % 4 == 3)
        *reinterpret_cast<uint4*>(mine + C - 4 * (i / 4 + 1)) = make_uint4(d[3], d[2], d[1], d[0]);
    } else {
      mine[C - 1 - i] = f32_from_digit_words40(u1, u0);
    }
  }
}

template <int C, int... I>
__device__ __forceinline__ void digit_run40_words(std::integer_sequence<int, I...>, uint64_t z,
                                                  uint32_t* mine, uint32_t& qmin) {
  const uint32_t z0 = (uint32_t)z, z1 = (uint32_t)(z >> 32);
  uint32_t r[DigitRun40<C>::W];
  uint32_t v0 = 0, v1 = 0, d[4];
  (digit_run40_word<C, I>(z0, z1, r, v0, v1, d, mine, qmin), ...);
}

// One lane's FP32 run of C elements from z, the state one past it.  A run
// with a digit below 2^23 (its u1 below 4) is redone by its lane, forward
// from element 0's state.
template <int C>
__device__ __forceinline__ void digit_run40_f32(uint32_t* mine, uint64_t z) {
  uint32_t qmin = 0xffffffffu;
  digit_run40_words<C>(std::make_integer_sequence<int, DigitRun40<C>::W>{}, z, mine, qmin);
  const bool rare = qmin < 4u;
  if (__any_sync(0xffffffffu, rare)) {
    if (rare) {
      Chain40<DT_F32> f;
      f.start(mont40(z, DigitRun40<C>::back));
      for (uint32_t i = 0; i < (uint32_t)C; ++i) mine[i] = f.next();
    }
    __syncwarp();
  }
}

// Whether a tile loop of this kind makes its runs that way.
template <int DT, int ILP, int CDEPTH>
constexpr bool kDigits40 = DT == DT_F32 && ILP == 1 && CDEPTH > 0 && digit_run40_depth(CDEPTH);

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
  if constexpr (kDigits40<DT, ILP, CDEPTH>) {
    if (t0 < t1) {
      // each run from one product; z is the state one past this lane's run,
      // and p.jump = 2^(53*32c) moves it to the lane's run in the next tile
      uint64_t z = state_of40(p.ebase, p.head + t0 * tile_elems + (uint64_t)lane * c + c);
      uint32_t issued = 0;
      for (uint64_t t = t0; t < t1; ++t) {
        W* const buf = buf0 + tile_buffer(issued, p.nbuf) * tile_elems;
        wait_buffer_free(issued, p.nbuf, lane);
        digit_run40_f32<CDEPTH>(buf + lane * c, z);
        fence_proxy_async_shared();
        __syncwarp();
        if (lane == 0) {
          bulk_store(out + p.head + t * tile_elems, buf, tile_bytes);
          bulk_commit();
        }
        ++issued;
        if (t + 1 < t1) z = mont40(z, p.jump);
      }
      if (lane == 0) bulk_wait_all();
      __syncwarp();
    }
  } else if (t0 < t1) {
    // Backward chains: a single chain emits c-1 .. 0 of the lane's run; two
    // chains split it, b emitting c-1 .. h+1 and a h .. 0.  Afterwards chain
    // a holds element 0 (its state), chain b element h+1.
    const uint64_t first = p.head + t0 * tile_elems + (uint64_t)lane * c;
    const uint32_t h = c >> 1;
    constexpr uint64_t lead = DT == DT_U64 ? 0 : 1;  // the digit of the state above
    Back40<DT> a, b;
    if constexpr (ILP == 2) {
      a.start(state_of40(p.ebase, first + h + 1 + lead));
      b.start(state_of40(p.ebase, first + c + lead));
    } else {
      a.start(state_of40(p.ebase, first + c + lead));
    }
    uint32_t issued = 0;
    for (uint64_t t = t0; t < t1; ++t) {
      W* const buf = buf0 + tile_buffer(issued, p.nbuf) * tile_elems;
      wait_buffer_free(issued, p.nbuf, lane);
      W* const mine = buf + lane * c;
      uint32_t qmin = 0xffffffffu;
      if constexpr (ILP == 2) {
        const uint32_t last = CDEPTH > 0 ? (uint32_t)CDEPTH - 1 : c - 1;
#pragma unroll
        for (uint32_t i = 0; i < (CDEPTH > 0 ? (uint32_t)CDEPTH / 2 : h); ++i) {
          mine[last - i] = b.next(qmin);
          mine[h - i] = a.next(qmin);
        }
        mine[0] = a.next(qmin);
      } else {
#pragma unroll
        for (uint32_t i = (CDEPTH > 0 ? (uint32_t)CDEPTH : c); i-- > 0;) mine[i] = a.next(qmin);
      }
      if constexpr (DT != DT_U64) {
        // a lane whose run holds a variate below 2^-21 redoes it exactly,
        // forward from element 0
        const bool rare = qmin == 0;
        if (__any_sync(0xffffffffu, rare)) {
          if (rare) {
            Chain40<DT> f;
            f.start(a.z);
            for (uint32_t i = 0; i < c; ++i) mine[i] = f.next();
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
  if constexpr (DT == DT_F32) {  // four-variate stores
    if (depth == 44) return (const void*)tiled40_kernel<DT, 1, 44>;
  }
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
