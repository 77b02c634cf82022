// bcn_mc.cu -- a Monte-Carlo consumer fused with generation (no variates are
// stored).  The paper notes that variates are often used by a simulation on
// the GPU rather than written out (Sec. 2.2); this kernel is that use, with
// the sequence split into blocks as in the paper's parallel split (Sec. 1).
//
// Block b covers variates [b*len, (b+1)*len) of the sequence seeded with a.
// Its variates are taken in pairs (x, y) = (v_2j, v_2j+1); the block reports
//   hits  = #{pairs with RN(RN(x*x) + RN(y*y)) <= 1}   (quarter-circle test),
//   sum   = RN(exact sum of v),   sumsq = RN(exact sum of RN(v*v)),
// with RN round-to-nearest-even.  Everything is decided in integers:
//   * every variate is a multiple of 2^-105 below 1, so v*2^105 is an integer
//     below 2^105 and a lane's sum fits 128 bits;
//   * every RN(v*v) is a multiple of 2^-157 (the smallest variate is about
//     1.62*2^-53, so the smallest square has exponent -105), so RN(v*v)*2^157
//     is an integer below 2^157.  For every variate above about 2^-20 its low
//     64 bits are zero, so those squares are summed exactly as 128-bit
//     integers on the 2^-93 grid; the rare smaller ones (below 2^117 on the
//     2^-157 grid) go to a second 128-bit sum, and the two are joined into one
//     192-bit integer per block;
//   * RN(X + Y) <= 1 exactly when X + Y <= 1 + 2^-53 (the tie rounds to the
//     even 1.0), i.e. when the two grid integers sum to at most 2^157 + 2^104.
//     That bound is a multiple of 2^64, so the test can be made on the 2^-93
//     grid with each rare small square rounded up: X + Y <= T exactly when
//     hi(X) + ceil(Y / 2^64) <= T / 2^64 for X a multiple of 2^64.
// Integer sums do not depend on order, so the warp reduction and the final
// per-block rounding give the same bits for any launch shape.
#include "bcn_gen.cuh"
#include "bcn_mc.cuh"

namespace bcn {

// (a1:a0) += (b1:b0) with one carry chain.
__device__ __forceinline__ void add128(uint64_t& a0, uint64_t& a1, uint64_t b0, uint64_t b1) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a0), "+l"(a1) : "l"(b0), "l"(b1));
}

// x << k as (lo, hi) for x < 2^64, 0 <= k < 64 (no branch for k = 0).
__device__ __forceinline__ void shl128(uint64_t x, uint32_t k, uint64_t& lo, uint64_t& hi) {
  lo = x << k;
  hi = (x >> 1) >> (63u - k);
}

// The exact grid images of one FP64 variate v (bits of RN(z*r3i)):
//   (v0, v1)  = v * 2^105, an integer below 2^105;
//   RN(v*v) * 2^157 = M2 << k with k = 2e + sh - 1993 >= 0.  When k >= 64
//   (every variate from about 2^-20 up) its low 64 bits are zero and
//   (q0, q1) = RN(v*v) * 2^93 exactly, `fast` is set; otherwise (q0, q1) =
//   ceil(RN(v*v) * 2^93) for the hit test, and the exact value (below 2^117)
//   goes to (s0, s1).
struct Terms {
  uint64_t v0, v1, q0, q1, s0, s1;
  bool fast;
};

// The grid images of RN(v*v) = M2 * 2^(e2 - 1075), M2 with its leading one:
// on the 2^-157 grid it is M2 << k, k = e2 - 918 >= 0 (every square is at
// least 2^-105).  Shared by both forms of the square.
__device__ __forceinline__ void square_terms(uint64_t m2, uint32_t k, Terms& t) {
  t.s0 = t.s1 = 0;
  t.fast = k >= 64u;
  if (__builtin_expect(t.fast, 1)) {
    shl128(m2, k - 64u, t.q0, t.q1);
  } else {
    shl128(m2, k, t.s0, t.s1);            // exact, below 2^117
    t.q0 = t.s1 + (t.s0 != 0 ? 1ull : 0ull);  // ceiling on the 2^-93 grid
    t.q1 = 0;
  }
}

__device__ __forceinline__ Terms variate_terms(uint64_t bits) {
  Terms t;
  const uint32_t e = (uint32_t)(bits >> 52);  // biased exponent, >= 970
  const uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  shl128(mant, e - 970u, t.v0, t.v1);          // v * 2^105, shift <= 52
  // RN(mant^2) to 53 significant bits, ties to even
  const uint64_t plo = mant * mant, phi = __umul64hi(mant, mant);  // < 2^106
  const uint32_t sh = 52u + ((uint32_t)(phi >> 41) & 1u);           // 53 if bit 105 set
  uint64_t m2 = (phi << (64u - sh)) | (plo >> sh);
  const uint64_t rest = plo & ((1ull << sh) - 1ull);
  const uint64_t half = 1ull << (sh - 1u);
  m2 += (rest > half) | ((rest == half) & (m2 & 1ull));
  square_terms(m2, 2u * e + sh - 1993u, t);
  return t;
}

// The same terms with the square taken on the FP64 pipe: one round-to-nearest
// multiply is RN(v*v) by definition, and its bits give M2 and e2 directly, so
// the integer pipes only place the result on the grids.
__device__ __forceinline__ Terms variate_terms_fp64(uint64_t bits) {
  Terms t;
  const uint32_t e = (uint32_t)(bits >> 52);
  const uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  shl128(mant, e - 970u, t.v0, t.v1);
  const double v = __longlong_as_double((long long)bits);
  const uint64_t sb = (uint64_t)__double_as_longlong(__dmul_rn(v, v));
  square_terms((sb & ((1ull << 52) - 1)) | (1ull << 52), (uint32_t)(sb >> 52) - 918u, t);
  return t;
}

// The fast-grid image of RN(v*v) for a variate v >= 2^-20, as every variate
// of a kept chunk is: RN(v*v) >= 2^-40, so its image on the 2^-157 grid is
// M2 << k with k = e2 - 918 >= 65, and RN(v*v) * 2^93 = M2 << (e2 - 982)
// exactly, with no branch on the square's size.
__device__ __forceinline__ void square_fast_fp64(uint64_t bits, uint64_t& q0, uint64_t& q1) {
  const double v = __longlong_as_double((long long)bits);
  const uint64_t sb = (uint64_t)__double_as_longlong(__dmul_rn(v, v));
  const uint64_t m2 = (sb & ((1ull << 52) - 1)) | (1ull << 52);
  shl128(m2, (uint32_t)(sb >> 52) - 982u, q0, q1);
}

// hits += [ (r1:r0) <= (lim1:lim0) ]: the borrow of (r1:r0) - (lim1:lim0) - 1
// (one subtract-with-borrow chain instead of three 64-bit compares).
__device__ __forceinline__ void count_hit(uint32_t& hits, uint64_t r0, uint64_t r1,
                                          uint64_t lim0p1, uint64_t lim1) {
  asm("{\n\t"
      ".reg .u64 t0, t1;\n\t"
      ".reg .u32 b;\n\t"
      "sub.cc.u64 t0, %1, %2;\n\t"
      "subc.cc.u64 t1, %3, %4;\n\t"
      "subc.u32 b, 0, 0;\n\t"
      "sub.u32 %0, %0, b;\n\t"
      "}"
      : "+r"(hits)
      : "l"(r0), "l"(lim0p1), "l"(r1), "l"(lim1));
}

// (a1:a0) += v * 2^105 for a variate v >= 2^-21 (the branch-free path, where
// every variate of a kept chunk is at least 2^-21): its biased exponent e is
// in [1002, 1022], so v * 2^105 = mant * 2^(32 + j) with j = e - 1002 in
// [0, 20], and the image's low 32-bit word is zero.  The shift is made as
// products by 2^j on the multiply-add pipe, whose carries feed the
// accumulator directly: the integer ALU pipe, which binds this kernel, keeps
// only the exponent and the two-word split (measured: 424 -> 437 G
// variates/s with the hit test and the sums' adds below also moved there).
__device__ __forceinline__ void add_variate_fast(uint64_t& a0, uint64_t& a1, uint64_t bits) {
  const uint32_t hi = (uint32_t)(bits >> 32), lo = (uint32_t)bits;
  const uint32_t pj = 1u << ((hi >> 20) - 1002u);
  const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
  asm("{\n\t"
      ".reg .u32 A0, A1, A2, A3;\n\t"
      "mov.b64 {A0, A1}, %0;\n\t"
      "mov.b64 {A2, A3}, %1;\n\t"
      "mad.lo.cc.u32 A1, %2, %4, A1;\n\t"   // + lo * 2^j, word 1
      "madc.hi.cc.u32 A2, %2, %4, A2;\n\t"  // + its high word, word 2
      "madc.hi.u32 A3, %3, %4, A3;\n\t"     // + high word of mh * 2^j, word 3
      "mad.lo.cc.u32 A2, %3, %4, A2;\n\t"   // + low word of mh * 2^j, word 2
      "addc.u32 A3, A3, 0;\n\t"
      "mov.b64 %0, {A0, A1};\n\t"
      "mov.b64 %1, {A2, A3};\n\t"
      "}"
      : "+l"(a0), "+l"(a1)
      : "r"(lo), "r"(mh), "r"(pj));
}

// (a1:a0) += (b1:b0) as multiply-adds by 1 with carries (the multiply-add
// pipe, not the integer ALU pipe).
__device__ __forceinline__ void add128_fma(uint64_t& a0, uint64_t& a1, uint64_t b0, uint64_t b1) {
  asm("{\n\t"
      ".reg .u32 A0, A1, A2, A3, B0, B1, B2, B3;\n\t"
      "mov.b64 {A0, A1}, %0;\n\t"
      "mov.b64 {A2, A3}, %1;\n\t"
      "mov.b64 {B0, B1}, %2;\n\t"
      "mov.b64 {B2, B3}, %3;\n\t"
      "mad.lo.cc.u32 A0, B0, 1, A0;\n\t"
      "madc.lo.cc.u32 A1, B1, 1, A1;\n\t"
      "madc.lo.cc.u32 A2, B2, 1, A2;\n\t"
      "madc.lo.u32 A3, B3, 1, A3;\n\t"
      "mov.b64 %0, {A0, A1};\n\t"
      "mov.b64 %1, {A2, A3};\n\t"
      "}"
      : "+l"(a0), "+l"(a1)
      : "l"(b0), "l"(b1));
}

// misses += [ (r1:r0) > lim ]: the carry out of (r1:r0) + ~lim, summed by
// multiply-adds with carries.
__device__ __forceinline__ void count_miss_fma(uint32_t& miss, uint64_t r0, uint64_t r1,
                                               uint64_t nlim0, uint64_t nlim1) {
  asm("{\n\t"
      ".reg .u32 R0, R1, R2, R3, C0, C1, C2, C3, t;\n\t"
      "mov.b64 {R0, R1}, %1;\n\t"
      "mov.b64 {R2, R3}, %2;\n\t"
      "mov.b64 {C0, C1}, %3;\n\t"
      "mov.b64 {C2, C3}, %4;\n\t"
      "mad.lo.cc.u32 t, R0, 1, C0;\n\t"
      "madc.lo.cc.u32 t, R1, 1, C1;\n\t"
      "madc.lo.cc.u32 t, R2, 1, C2;\n\t"
      "madc.lo.cc.u32 t, R3, 1, C3;\n\t"
      "madc.lo.u32 %0, 0, 0, %0;\n\t"
      "}"
      : "+r"(miss)
      : "l"(r0), "l"(r1), "l"(nlim0), "l"(nlim1));
}

// Round (w2:w1:w0) * 2^-scale to the nearest double, ties to even.
__device__ double round_words(uint64_t w0, uint64_t w1, uint64_t w2, int scale) {
  int top;
  if (w2) top = 128 + 63 - __clzll((long long)w2);
  else if (w1) top = 64 + 63 - __clzll((long long)w1);
  else if (w0) top = 63 - __clzll((long long)w0);
  else return 0.0;
  auto bit_range = [&](int lo) -> uint64_t {  // 64 bits starting at bit lo (lo >= 0)
    const uint64_t ws[3] = {w0, w1, w2};
    const int q = lo >> 6, r = lo & 63;
    uint64_t a = q < 3 ? ws[q] : 0, b = q + 1 < 3 ? ws[q + 1] : 0;
    return r ? ((a >> r) | (b << (64 - r))) : a;
  };
  if (top <= 52) return ldexp((double)w0, -scale);  // exact
  const int low = top - 52;                          // lowest kept bit
  uint64_t mant = bit_range(low) & ((1ull << 53) - 1);
  const uint64_t guard = (bit_range(low - 1) & 1ull);
  bool sticky = false;
  for (int k = 0; k < low - 1 && !sticky; k += 64) {
    uint64_t chunk = bit_range(k);
    const int nb = low - 1 - k;  // bits of this chunk below the guard bit
    if (nb < 64) chunk &= (1ull << nb) - 1ull;
    sticky = chunk != 0;
  }
  if (guard && (sticky || (mant & 1ull))) mant += 1;
  return ldexp((double)mant, low - scale);
}

// FP64SQ: each RN(v*v) by one multiply on the FP64 pipe, else formed on the
// integer pipes; the hit test and the sums stay integer either way (taking
// the test's add on the FP64 pipe as well measured slower: that pipe is the
// scarcer one).  The two forms give identical bits.
template <bool FP64SQ>
__global__ void __launch_bounds__(256) mc_kernel(const McParams p) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t wpb = blockDim.x >> 5;
  const uint64_t b = (uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
  if (b >= p.nblocks) return;
  const uint64_t pairs = p.len / 2;
  const uint64_t j0 = lane * pairs / 32, j1 = (lane + 1) * pairs / 32;
  const uint64_t first = (p.block0 + b) * p.len + 2 * j0;
  uint32_t hits = 0;        // hits of the exactly made pairs
  uint32_t miss = 0, kept = 0;  // misses among the pairs of kept chunks, and those pairs
  uint64_t a0 = 0, a1 = 0;  // sum of v * 2^105
  uint64_t h0 = 0, h1 = 0;  // sum of the fast RN(v*v) * 2^93
  uint64_t l0 = 0, l1 = 0;  // sum of the other RN(v*v) * 2^157 (rare)
  // hit iff RN(x^2) + RN(y^2) <= 1 + 2^-53, i.e. on the 2^-93 grid
  // (exact high parts, ceilings of the rare small squares) <= 2^93 + 2^40
  const uint64_t lim0 = 1ull << 40, lim1 = 1ull << 29;
  if (j0 < j1) {
    uint64_t z = seed_state(exponent_add(p.ebase, first + 1), p.skip);
    // One pair of variates into the accumulators; `exact` selects the
    // conversion with its own rare-case branch, else the branch-free one
    // that only lowers qmin when it cannot be trusted.
    auto pair = [&](bool exact, uint32_t& qmin) {
      const uint64_t bx = exact ? shared_step_f64(z) : shared_step_f64_ptx(z, qmin);
      const uint64_t by = exact ? shared_step_f64(z) : shared_step_f64_ptx(z, qmin);
      if constexpr (FP64SQ) {
        if (!exact) {  // a kept chunk: both squares on the fast grid, no branch
          uint64_t xq0, xq1, yq0, yq1;
          square_fast_fp64(bx, xq0, xq1);
          square_fast_fp64(by, yq0, yq1);
          add_variate_fast(a0, a1, bx);
          add_variate_fast(a0, a1, by);
          add128_fma(xq0, xq1, yq0, yq1);
          count_miss_fma(miss, xq0, xq1, ~lim0, ~lim1);
          add128_fma(h0, h1, xq0, xq1);
          return;
        }
      }
      const Terms x = FP64SQ ? variate_terms_fp64(bx) : variate_terms(bx);
      const Terms y = FP64SQ ? variate_terms_fp64(by) : variate_terms(by);
      if (exact) {
        add128(a0, a1, x.v0, x.v1);
        add128(a0, a1, y.v0, y.v1);
      } else {  // every variate of a kept chunk is at least 2^-21
        add_variate_fast(a0, a1, bx);
        add_variate_fast(a0, a1, by);
      }
      uint64_t r0 = x.q0, r1 = x.q1;
      add128(r0, r1, y.q0, y.q1);
      count_hit(hits, r0, r1, lim0 + 1, lim1);
      if (__builtin_expect(x.fast & y.fast, 1)) {
        add128(h0, h1, r0, r1);
      } else {
        if (x.fast) add128(h0, h1, x.q0, x.q1);
        if (y.fast) add128(h0, h1, y.q0, y.q1);
        add128(l0, l1, x.s0, x.s1);
        add128(l0, l1, y.s0, y.s1);
      }
    };
    // Chunks of kChunk pairs with the branch-free conversion; a lane whose
    // chunk met a variate below 2^-20 (a quotient window below 2^33, about
    // one chunk in 2^13) restores the chunk's starting point and redoes it
    // exactly.  Every variate of a kept chunk is then at least 2^-20, so its
    // square lies on the fast grid and its image has a zero low word.
    constexpr uint32_t kChunk = 64;
    uint64_t j = j0;
    for (; j + kChunk <= j1; j += kChunk) {
      const uint64_t zs = z, sa0 = a0, sa1 = a1, sh0 = h0, sh1 = h1, sl0 = l0, sl1 = l1;
      const uint32_t shits = hits, smiss = miss;
      uint32_t qmin = 0xffffffffu;
#pragma unroll 4
      for (uint32_t k = 0; k < kChunk; ++k) pair(false, qmin);
      if (__builtin_expect(qmin < 2, 0)) {
        z = zs; a0 = sa0; a1 = sa1; h0 = sh0; h1 = sh1; l0 = sl0; l1 = sl1; hits = shits;
        miss = smiss;
        uint32_t unused = 0;
        for (uint32_t k = 0; k < kChunk; ++k) pair(true, unused);
      } else {
        kept += kChunk;
      }
    }
    for (uint32_t unused = 0; j < j1; ++j) pair(true, unused);
    if constexpr (FP64SQ) hits += kept - miss;  // the kept chunks counted their misses
  }
  // exact warp reduction (integer addition is order-free)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    hits += __shfl_xor_sync(0xffffffffu, hits, off);
    uint64_t o0 = __shfl_xor_sync(0xffffffffu, a0, off);
    uint64_t o1 = __shfl_xor_sync(0xffffffffu, a1, off);
    add128(a0, a1, o0, o1);
    o0 = __shfl_xor_sync(0xffffffffu, h0, off);
    o1 = __shfl_xor_sync(0xffffffffu, h1, off);
    add128(h0, h1, o0, o1);
    o0 = __shfl_xor_sync(0xffffffffu, l0, off);
    o1 = __shfl_xor_sync(0xffffffffu, l1, off);
    add128(l0, l1, o0, o1);
  }
  // sum of squares on the 2^-157 grid: (h << 64) + l
  uint64_t w0 = l0, w1 = l1, w2 = 0;
  add128(w1, w2, h0, h1);
  if (lane == 0) {
    p.sum[b] = round_words(a0, a1, 0, 105);
    p.sumsq[b] = round_words(w0, w1, w2, 157);
    if (p.hits) p.hits[b] = hits;
    atomicAdd(p.hits_total, (unsigned long long)hits);
    if (p.totals) {  // exact totals over the call: every 32-bit piece into its own word
      const uint64_t words[kMcSumWords + kMcSqWords] = {a0, a0 >> 32, a1, a1 >> 32,
                                                          w0, w0 >> 32, w1, w1 >> 32,
                                                          w2, w2 >> 32};
#pragma unroll
      for (uint32_t k = 0; k < kMcSumWords + kMcSqWords; ++k)
        atomicAdd(&p.totals[k], (unsigned long long)(words[k] & 0xFFFFFFFFull));
    }
  }
}

const void* mc_kernel_fn(bool fp64_squares) {
  return fp64_squares ? (const void*)mc_kernel<true> : (const void*)mc_kernel<false>;
}

}  // namespace bcn
