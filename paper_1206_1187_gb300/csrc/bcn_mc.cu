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
//     below 2^105 and a block's sum (len <= 2^33) fits 138 bits, kept in
//     three 64-bit words;
//   * every RN(v*v) is a multiple of 2^-157 (the smallest variate is about
//     1.62*2^-53, so the smallest square has exponent -105), so RN(v*v)*2^157
//     is an integer below 2^157.  For every variate above about 2^-20 its low
//     64 bits are zero, so those squares are summed exactly as 128-bit
//     integers on the 2^-93 grid; the rare smaller ones (below 2^117 on the
//     2^-157 grid) go to a second 128-bit sum, and the two are joined into one
//     192-bit integer per block.  Chunks whose variates are all at least
//     2^-16 (nearly all) take their squares on the coarser 2^-84 grid, where
//     every such square is an integer below 2^84, and fold them in;
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

// (a2:a1:a0) += (b1:b0) with one carry chain.
__device__ __forceinline__ void add192(uint64_t& a0, uint64_t& a1, uint64_t& a2, uint64_t b0,
                                       uint64_t b1) {
  asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, 0;"
      : "+l"(a0), "+l"(a1), "+l"(a2)
      : "l"(b0), "l"(b1));
}

// ---- the kept-chunk path: every variate of a kept chunk is at least 2^-16 ----
//
// A variate v >= 2^-16 has biased exponent e in [1007, 1022], so
//   v * 2^105 = (mh 2^32 + lo) * pj * 2^32,  pj = 2^(e - 1002) in [2^5, 2^20],
// with mh the top 21 bits of its significand (leading one included) and lo
// the low 32.  Its square RN(v*v) >= 2^-32 has biased exponent e2 in
// [991, 1022], so on the 2^-84 grid
//   RN(v*v) * 2^84 = (mh2 2^32 + ml2) * pk,  pk = 2^(e2 - 991) in [1, 2^31].
// Both powers of two come from one funnel rotate of a constant by the
// exponent (the rotate takes the amount mod 32): e - 1002 = (e + 22) mod 32
// and e2 - 991 = (e2 + 1) mod 32 on those ranges.  The shifts are then
// products on the multiply-add pipe, which also sums them: per chunk of 64
// pairs, lo*pj and mh*pj go to 64-bit partial sums (below 2^59 and 2^48),
// and each pair's exact x'+y' (below 2^85, three words) to three more.
// The integer ALU pipe keeps only the field extractions.
__device__ __forceinline__ void variate_parts(uint64_t bits, uint32_t& lo, uint32_t& mh,
                                              uint32_t& pj) {
  const uint32_t hi = (uint32_t)(bits >> 32);
  lo = (uint32_t)bits;
  mh = (hi & 0xFFFFFu) | 0x100000u;
  pj = __funnelshift_l(1u << 22, 1u << 22, hi >> 20);  // 2^(e - 1002)
}

__device__ __forceinline__ void square_parts(uint64_t sb, uint32_t& ml, uint32_t& mh,
                                             uint32_t& pk) {
  const uint32_t hi = (uint32_t)(sb >> 32);
  ml = (uint32_t)sb;
  mh = (hi & 0xFFFFFu) | 0x100000u;
  pk = __funnelshift_l(2u, 2u, hi >> 20);  // 2^(e2 - 991)
}

// The bits of RN(v*v) for a variate v >= 2^-16 (no subnormal, no overflow):
// one round-to-nearest multiply on the FP64 pipe, or the same rounding of
// mant^2 made on the integer pipes (ties to even; a carry into bit 53 moves
// the exponent up through the addition).
template <bool FP64SQ>
__device__ __forceinline__ uint64_t square_bits(uint64_t bits) {
  if constexpr (FP64SQ) {
    const double v = __longlong_as_double((long long)bits);
    return (uint64_t)__double_as_longlong(__dmul_rn(v, v));
  } else {
    const uint32_t e = (uint32_t)(bits >> 52);
    const uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const uint64_t plo = mant * mant, phi = __umul64hi(mant, mant);
    const uint32_t sh = 52u + ((uint32_t)(phi >> 41) & 1u);
    uint64_t m2 = (phi << (64u - sh)) | (plo >> sh);
    const uint64_t rest = plo & ((1ull << sh) - 1ull);
    const uint64_t half = 1ull << (sh - 1u);
    m2 += (rest > half) | ((rest == half) & (m2 & 1ull));
    return ((uint64_t)(2u * e + sh - 1076u) << 52) + m2;
  }
}

// (s2:s1:s0) = x' + y' for the 2^-84-grid images of two squares: the two
// low-part products fit one 64-bit sum (each below 2^63), the two high-part
// products another (below 2^53), and the result is their sum with the
// second shifted by 32.
__device__ __forceinline__ void pair_square_sum(uint32_t mlx, uint32_t mhx, uint32_t pkx,
                                                uint32_t mly, uint32_t mhy, uint32_t pky,
                                                uint32_t& s0, uint32_t& s1, uint32_t& s2) {
  asm("{\n\t"
      ".reg .u64 TL, TH;\n\t"
      ".reg .u32 l1, h0, h1;\n\t"
      "mul.wide.u32 TL, %3, %5;\n\t"
      "mad.wide.u32 TL, %6, %8, TL;\n\t"
      "mul.wide.u32 TH, %4, %5;\n\t"
      "mad.wide.u32 TH, %7, %8, TH;\n\t"
      "mov.b64 {%0, l1}, TL;\n\t"
      "mov.b64 {h0, h1}, TH;\n\t"
      "add.cc.u32 %1, l1, h0;\n\t"
      "addc.u32 %2, h1, 0;\n\t"
      "}"
      : "=&r"(s0), "=&r"(s1), "=&r"(s2)
      : "r"(mlx), "r"(mhx), "r"(pkx), "r"(mly), "r"(mhy), "r"(pky));
}

// misses += [S > 2^84 + 2^31] for S = (s2:s1:s0): the carry out of S plus
// the 96-bit complement of that bound, taken as multiply-adds by 1.  A pair
// is a hit iff RN(x^2) + RN(y^2) <= 1 + 2^-53 (the tie rounds to the even
// 1.0), which on the 2^-84 grid is S <= 2^84 + 2^31.
__device__ __forceinline__ void count_miss3(uint32_t& miss, uint32_t s0, uint32_t s1,
                                            uint32_t s2) {
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "mad.lo.cc.u32 t, %1, 1, 0x7FFFFFFF;\n\t"
      "madc.lo.cc.u32 t, %2, 1, 0xFFFFFFFF;\n\t"
      "madc.lo.cc.u32 t, %3, 1, 0xFFEFFFFF;\n\t"
      "madc.lo.u32 %0, 0, 0, %0;\n\t"
      "}"
      : "+r"(miss)
      : "r"(s0), "r"(s1), "r"(s2));
}

// q += s as one 64-bit multiply-add (the multiply-add pipe, not the ALU).
__device__ __forceinline__ void acc_wide(uint64_t& q, uint32_t s) {
  asm("mad.wide.u32 %0, %1, 1, %0;" : "+l"(q) : "r"(s));
}

// Lane jumps of the warp's shared redo: lane l starts 2 l pairs (4 l steps)
// after the first state of the run being redone, at z 2^(53 * 4 l) mod m (Eq. 3
// applied 4 l times), with the precomputed quotient of each multiplier.
struct RedoJump {
  uint64_t j[32], q[32];
};
constexpr RedoJump make_redo_jump() {
  RedoJump t{};
  for (uint64_t l = 0; l < 32; ++l) {
    t.j[l] = host_pow2((53ull * 4ull * l) % kP);
    t.q[l] = host_mulmod_quotient(t.j[l]);
  }
  return t;
}
static __device__ const RedoJump kRedoJump = make_redo_jump();
static_assert(make_redo_jump().j[0] == 1 && make_redo_jump().j[1] == host_pow2(212),
              "redo jumps");

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
// integer pipes; the hit test and the sums stay integer either way.  The two
// forms give identical bits.  At most 64 registers (the launch bound), which
// measured faster than the 68 the compiler takes unbounded: more warps hide
// the step's latency while the three pipes stay near 70% busy.
template <bool FP64SQ>
__global__ void __launch_bounds__(256, 4) mc_kernel(const McParams p) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t wpb = blockDim.x >> 5;
  const uint64_t b = (uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
  if (b >= p.nblocks) return;
  const uint64_t pairs = p.len / 2;
  const uint64_t j0 = lane * pairs / 32, j1 = (lane + 1) * pairs / 32;
  const uint64_t first = (p.block0 + b) * p.len + 2 * j0;
  uint32_t hits = 0;            // hits of the exactly made pairs
  uint32_t miss = 0, kept = 0;  // misses among the pairs of kept chunks, and those pairs
  uint64_t a0 = 0, a1 = 0, a2 = 0;  // sum of v * 2^105 (below 2^138: len <= 2^33)
  uint64_t h0 = 0, h1 = 0;          // sum of the fast RN(v*v) * 2^93
  uint64_t l0 = 0, l1 = 0;          // sum of the other RN(v*v) * 2^157 (rare)
  // exact path: hit iff RN(x^2) + RN(y^2) <= 1 + 2^-53, i.e. on the 2^-93
  // grid (exact high parts, ceilings of the rare small squares) <= 2^93 + 2^40
  const uint64_t lim0 = 1ull << 40, lim1 = 1ull << 29;
  {  // every lane of the warp runs this block (the chunk loop votes), also one
     // with no pairs (j0 = j1, a block shorter than 64 variates)
    // the kept chunks step a chain scaled by 2^10 (see shared_step_f64_ptx),
    // the exact pairs the plain state
    uint64_t z = seed_state(exponent_add(p.ebase, first + 1), p.skip);
    uint64_t Z = z << kZShift;
    // One pair with the exact conversion and the general grids.
    auto exact_pair = [&]() {
      const uint64_t bx = shared_step_f64(z);
      const uint64_t by = shared_step_f64(z);
      const Terms x = FP64SQ ? variate_terms_fp64(bx) : variate_terms(bx);
      const Terms y = FP64SQ ? variate_terms_fp64(by) : variate_terms(by);
      add192(a0, a1, a2, x.v0, x.v1);
      add192(a0, a1, a2, y.v0, y.v1);
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
    // Chunks of kChunk pairs with the branch-free conversion and per-chunk
    // partial sums.  A kept chunk folds its partials into the block's sums:
    // v-sum += P1 2^32 + P2 2^64, and on the 2^-93 grid the squares'
    // h += (Q0 + Q1 2^32 + Q2 2^64) 2^9.  A chunk that met a variate below
    // 2^-16 (a quotient window below 2^37, qmin < 32: about one chunk in 2^9)
    // drops its partials and misses (its state advance is exact either way),
    // and the whole warp redoes it exactly: lane l takes pairs 2l and 2l + 1
    // of the chunk from one jump of the chunk's first state, adding them to
    // its own sums (the warp's totals are the same whoever adds them).  One
    // lane alone redoing 64 pairs left the other 31 idle: 473 against 523 G
    // variates/s.  The chunk loop runs the chunks every lane has, so that the
    // vote sees the whole warp; the lanes' pair counts differ by at most one.
    constexpr uint32_t kChunk = 64;
    static_assert(kChunk == 2 * 32, "the redo gives each lane two pairs");
    const uint32_t nch = __reduce_min_sync(0xffffffffu, (uint32_t)((j1 - j0) / kChunk));
    for (uint32_t ch = 0; ch < nch; ++ch) {
      const uint64_t zs = Z;
      const uint32_t smiss = miss;
      uint64_t P1 = 0, P2 = 0, Q0 = 0, Q1 = 0;
      uint32_t Q2 = 0, qmin = 0xffffffffu;
#pragma unroll 4
      for (uint32_t k = 0; k < kChunk; ++k) {
        const uint64_t bx = shared_step_f64_ptx(Z, qmin);
        const uint64_t by = shared_step_f64_ptx(Z, qmin);
        uint32_t xl, xm, xp, yl, ym, yp;
        variate_parts(bx, xl, xm, xp);
        variate_parts(by, yl, ym, yp);
        P1 += (uint64_t)xl * xp;
        P2 += (uint64_t)xm * xp;
        P1 += (uint64_t)yl * yp;
        P2 += (uint64_t)ym * yp;
        uint32_t sxl, sxm, sxp, syl, sym, syp;
        square_parts(square_bits<FP64SQ>(bx), sxl, sxm, sxp);
        square_parts(square_bits<FP64SQ>(by), syl, sym, syp);
        uint32_t s0, s1, s2;
        pair_square_sum(sxl, sxm, sxp, syl, sym, syp, s0, s1, s2);
        count_miss3(miss, s0, s1, s2);
        acc_wide(Q0, s0);
        acc_wide(Q1, s1);
        Q2 += s2;
      }
      const bool redo_mine = qmin < 32;
      if (__builtin_expect(redo_mine, 0)) {
        miss = smiss;
      } else {
        kept += kChunk;
        add192(a0, a1, a2, P1 << 32, P1 >> 32);
        add128(a1, a2, P2, 0);
        add128(h0, h1, Q0 << 9, 0);
        add128(h0, h1, Q1 << 41, Q1 >> 23);
        h1 += (uint64_t)Q2 << 9;
      }
      uint32_t redo = __ballot_sync(0xffffffffu, redo_mine);
      while (__builtin_expect(redo != 0, 0)) {
        const int L = __ffs(redo) - 1;
        redo &= redo - 1;
        const uint64_t zr = __shfl_sync(0xffffffffu, zs, L) >> kZShift;
        z = mulmod_pre(zr, kRedoJump.j[lane], kRedoJump.q[lane]);
        exact_pair();
        exact_pair();
      }
    }
    z = Z >> kZShift;
    for (uint64_t j = j0 + (uint64_t)kChunk * nch; j < j1; ++j) exact_pair();
    hits += kept - miss;  // the kept chunks counted their misses
  }
  // exact warp reduction (integer addition is order-free)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    hits += __shfl_xor_sync(0xffffffffu, hits, off);
    uint64_t o0 = __shfl_xor_sync(0xffffffffu, a0, off);
    uint64_t o1 = __shfl_xor_sync(0xffffffffu, a1, off);
    const uint64_t o2 = __shfl_xor_sync(0xffffffffu, a2, off);
    add192(a0, a1, a2, o0, o1);
    a2 += o2;
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
    p.sum[b] = round_words(a0, a1, a2, 105);
    p.sumsq[b] = round_words(w0, w1, w2, 157);
    if (p.hits) p.hits[b] = hits;
    atomicAdd(p.hits_total, (unsigned long long)hits);
    if (p.totals) {  // exact totals over the call: every 32-bit piece into its own word
      const uint64_t words[kMcSumWords + kMcSqWords] = {a0, a0 >> 32, a1, a1 >> 32, a2,
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
