// bcn_digits_math.cuh -- a run of variates' digits from one product (sm_103a):
// the arithmetic shared by the library's FP32 kernels and the device-side
// header (bcn_device.cuh).
//
// Run backwards, Eq. 3 is a Montgomery-style reduction with R = 2^53 whose
// quotient is the exact digit of the state it steps to: for
// z_k = 2^53 z_(k-1) mod m,
//   Q_k = floor(2^53 z_(k-1) / m) = -z_k m^-1 mod 2^53,
//   z_(k-1) = (z_k + Q_k m) / 2^53.
// The second line gives -z_k / m = Q_k + 2^53 (-z_(k-1) / m) in the 2-adic
// integers, so Q_k, Q_(k-1), ..., Q_(k-j+1) are the base-2^53 digits of
// -z_k/m and all j of them come from one product by a constant:
//   z_k N mod 2^(53 j),  N = -m^-1 mod 2^(53 j),
// whose 53-bit field i (from the bottom) is Q_(k-i), the truncated variate
// of the state i + 1 steps before z_k.  No state in between is formed: a run
// of C variates costs about 6.6 32-bit multiply-adds per variate against the
// eleven of a backward step, and each digit becomes a float as the backward
// step's digit does.
#pragma once
#include <cstdint>
#include <utility>

#include "bcn_math.cuh"

namespace bcn {

// -M^-1 mod 2^(32 W) for an odd modulus M < 2^64 as W 32-bit words, lowest
// first, solved word by word: A = (M * (words so far) + 1) / 2^(32 w), and
// the next word n makes A + M n divisible by 2^32 (n = -A M^-1 mod 2^32).
template <int W>
struct NegMinvWords {
  uint32_t w[W];
};
template <int W, uint64_t M>
constexpr NegMinvWords<W> make_neg_minv_words() {
  NegMinvWords<W> t{};
  const uint32_t inv = (uint32_t)inv_mod_2_64(M);  // M^-1 mod 2^32
  u128 A = 1;
  for (int i = 0; i < W; ++i) {
    const uint32_t n = 0u - (uint32_t)A * inv;
    A += (u128)M * n;  // low word now zero; A < 2^97
    t.w[i] = n;
    A >>= 32;
  }
  return t;
}
static_assert((make_neg_minv_words<2, kM>().w[0] |
               ((uint64_t)(make_neg_minv_words<2, kM>().w[1] & 0x1FFFFFu) << 32)) == kNegMinv53,
              "the low 53 bits of -m^-1 mod 2^64");

template <int W, uint64_t M = kM>
struct RunMinv {
  static constexpr NegMinvWords<W> t = make_neg_minv_words<W, M>();
};

// Where a run's C digits sit in its product: W words, and the digit whose
// top bit lies in word I (-1 if none; at most one, as 53 > 32).
template <int C>
struct DigitGeometry {
  static constexpr int W = (53 * C + 31) / 32;
  __host__ __device__ static constexpr int digit_of_word(int I) {
    const int num = 32 * I + 31 - 52;
    const int i = num < 0 ? 0 : num / 53;
    return i < C && (53 * i + 52) / 32 == I ? i : -1;
  }
};

#ifdef __CUDACC__
// Word I of z N (z = (z1:z0) on 32-bit words, z1 < 2^21), built from the
// bottom: it collects lo(z0 N_I), hi(z0 N_(I-1)), lo(z1 N_(I-1)),
// hi(z1 N_(I-2)) and the carry.  With V = (v1:v0) the part of the lower
// words' sum above word I - 1 (below 2^33), x = V + z1 N_(I-1) stays below
// 2^54 and x + z0 N_I below 2^65: word I is its low word and the next V its
// upper 33 bits.  Four 32-bit multiply-adds and one add per word.
template <int W, int I>
__device__ __forceinline__ void run_product_word(uint32_t z0, uint32_t z1, uint32_t& r,
                                                 uint32_t& v0, uint32_t& v1) {
  constexpr uint32_t nI = RunMinv<W>::t.w[I];
  if constexpr (I == 0) {
    r = z0 * nI;
    v0 = __umulhi(z0, nI);
    v1 = 0;
  } else if constexpr (I == W - 1) {  // the top word: no carry out
    constexpr uint32_t nP = RunMinv<W>::t.w[I - 1];
    asm("{\n\t"
        ".reg .u32 x0;\n\t"
        "mad.lo.u32 x0, %3, %5, %1;\n\t"
        "mad.lo.u32 %0, %2, %4, x0;\n\t"
        "}"
        : "=r"(r)
        : "r"(v0), "r"(z0), "r"(z1), "n"(nI), "n"(nP));
  } else {
    constexpr uint32_t nP = RunMinv<W>::t.w[I - 1];
    // r is early-clobber: it must not share a register with z0
    asm("{\n\t"
        ".reg .u32 x0, x1;\n\t"
        "mad.lo.cc.u32 x0, %4, %6, %1;\n\t"   // x = V + z1 N_(I-1)
        "madc.hi.u32 x1, %4, %6, %2;\n\t"
        "mad.lo.cc.u32 %0, %3, %5, x0;\n\t"   // x + z0 N_I: word I ...
        "madc.hi.cc.u32 %1, %3, %5, x1;\n\t"  // ... and the next V
        "addc.u32 %2, 0, 0;\n\t"
        "}"
        : "=&r"(r), "+r"(v0), "+r"(v1)
        : "r"(z0), "r"(z1), "n"(nI), "n"(nP));
  }
}

// Bits [POS, POS + 32) of the product's words r (POS >= -31; bits below 0
// read as zeros).
template <int POS, int W>
__device__ __forceinline__ uint32_t run_bits32(const uint32_t (&r)[W]) {
  if constexpr (POS < 0) {
    return r[0] << (-POS);
  } else if constexpr (POS % 32 == 0) {
    return r[POS / 32];
  } else {
    static_assert(POS / 32 + 1 < W, "bits inside the product");
    return __funnelshift_r(r[POS / 32], r[POS / 32 + 1], POS % 32);
  }
}

// The FP32 bits of a digit Q held as X = Q 2^11 = (u1:u0), and the running
// flag minimum, formed as back_step_f32_ptx forms them (the float is Q's
// leading 24 bits with exponent 126 - c, c = leading zeros of u1; a zero
// flag marks a digit that may need the exact path).  Bits 0 .. 10 of u0 may
// hold the next digit's top bits instead of zeros: neither the float (read
// from bit 40 - c >= 21 of X whenever the flag is not raised) nor the flag
// (u0 | 0xFFF) reads them.
__device__ __forceinline__ uint32_t f32_from_digit_words(uint32_t u1, uint32_t u0,
                                                         uint32_t& qmin) {
  uint32_t b, qo;
  asm("{\n\t"
      ".reg .u32 c, mant, e, nv;\n\t"
      "bfind.shiftamt.u32 c, %2;\n\t"
      "shf.l.clamp.b32 mant, %3, %2, c;\n\t"
      "shr.b32 mant, mant, 8;\n\t"
      "mad.lo.u32 e, c, 0xFF800000, 0x3E800000;\n\t"
      "or.b32 nv, %3, 0xFFF;\n\t"
      "not.b32 nv, nv;\n\t"
      "shl.b32 nv, nv, c;\n\t"
      "add.u32 %0, mant, e;\n\t"
      "min.u32 %1, %4, nv;\n\t"
      "}"
      : "=&r"(b), "=&r"(qo)
      : "r"(u1), "r"(u0), "r"(qmin));
  qmin = qo;
  return b;
}
#endif  // __CUDACC__

}  // namespace bcn
