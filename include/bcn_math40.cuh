// bcn_math40.cuh -- arithmetic of the larger-modulus variant of the
// alpha_{2,3} generator: Eq. 2 and Eq. 3 with the modulus 3^40 instead of
// 3^33.  Sec. 1 notes that a modulus as large as 3^40 lengthens the period
// (2*3^39, about 8.1e18) and needs 128-bit integer arithmetic: a state is a
// full 64-bit word (3^40 > 2^63) and the step's product 2^53 z has 117 bits.
//
//   seed a in [3^40+100, 2^64-1];  z_0 = 2^(a-3^40) * floor(3^40/2) mod 3^40;
//   z_k = 2^53 z_(k-1) mod 3^40;  variate = z_k / 3^40 rounded toward zero.
//
// The variate is truncated, not rounded to nearest: its 53 significant
// digits are then binary digits of alpha_{2,3}, and it stays below 1 (rounded
// to nearest, the top states round to 1.0 because 3^40 > 2^54).
//
// Quotient digits.  With q_k = floor(2^53 z_k / 3^40), Eq. 3 is
// z_(k+1) = 2^53 z_k - q_k 3^40, and z_(k+1)/3^40 is the fractional part of
// 2^53 z_k / 3^40.  So z_k / 3^40 = 0.q_k q_(k+1) q_(k+2) ... in base 2^53:
// the quotients are the successive 53-bit windows of the variate's binary
// expansion.  The generator computes one quotient per step (it needs it for
// the remainder anyway) and forms a variate from two consecutive quotients.
#pragma once
#include <cstdint>

#include "bcn_math.cuh"

namespace bcn {

constexpr uint64_t k40M = 12157665459056928801ULL;  // 3^40
constexpr uint64_t k40H = k40M / 2;                 // floor(3^40/2)   (Eq. 2)
constexpr uint64_t k40P = 2ULL * (k40M / 3);        // 2*3^39, the period
constexpr uint64_t k40SeedMin = k40M + 100;
static_assert(pow3(40) == k40M, "m = 3^40");
static_assert(k40M > (1ULL << 63), "a state fills a 64-bit word");

// R = floor(2^181 / 3^40), 118 bits, as (k40Rhi, k40Rlo).  For every state z,
// floor(z R / 2^128) = floor(2^53 z / 3^40) exactly: z R / 2^128 falls short
// of 2^53 z / 3^40 by less than z / 2^128 < 2^-64, while the fractional part
// of 2^53 z / 3^40 is (2^53 z mod 3^40) / 3^40 >= 1/3^40 > 2^-64 (the
// remainder is never 0, as z is prime to 3).
constexpr uint64_t k40Rhi = (uint64_t)(((u128)1 << 117) / k40M);
constexpr uint64_t k40Rlo =
    (uint64_t)(((((u128)1 << 117) - (u128)k40Rhi * k40M) << 64) / k40M);
static_assert(k40Rhi == 0x308daaa1c6f6a0ULL && k40Rlo == 0xc7be877cc9c0fcdeULL,
              "floor(2^181 / 3^40)");

// -m^-1 mod 2^64 for Montgomery products with R = 2^64.
constexpr uint64_t k40NegMinv = 0 - inv_mod_2_64(k40M);
static_assert(k40M * k40NegMinv + 1 == 0, "m * (-m^-1) = -1 mod 2^64");

// ------------------------------------------------------- host-side helpers
constexpr uint64_t host40_mulmod(uint64_t a, uint64_t b) {
  return (uint64_t)(((u128)a * b) % k40M);
}
constexpr uint64_t host40_pow2(uint64_t e) {
  uint64_t r = 1, g = 2;
  while (e) {
    if (e & 1) r = host40_mulmod(r, g);
    g = host40_mulmod(g, g);
    e >>= 1;
  }
  return r;
}
static_assert(host40_pow2(k40P) == 1 && host40_pow2(k40P / 2) == k40M - 1, "period");
// c * 2^64 mod m: the Montgomery form of a constant multiplier c.
constexpr uint64_t host40_mont_form(uint64_t c) {
  return (uint64_t)(((u128)c << 64) % k40M);
}
// (a - 3^40 + 53*i0) mod P: exponent of the state before variate i0.
inline uint64_t host40_exponent_base(uint64_t seed, uint64_t i0) {
  return (uint64_t)(((u128)(seed - k40M) + (u128)53 * (i0 % k40P)) % k40P);
}

// Fixed-base exponent table for e < P < 2^63, one row per byte of e.  Row 0
// holds floor(3^40/2) * 2^d mod m in plain form; rows 1..7 hold
// 2^(d * 256^k) in Montgomery form, so that a Montgomery product of a plain
// value by a row entry is a plain modular product.
constexpr int k40TabRows = 8;
struct PowTable40 {
  uint64_t t[k40TabRows][256];
};
constexpr PowTable40 make_pow_table40() {
  PowTable40 T{};
  uint64_t g = 2;  // 2^(256^k)
  for (int k = 0; k < k40TabRows; ++k) {
    uint64_t v = (k == 0) ? k40H : 1;
    for (int d = 0; d < 256; ++d) {
      T.t[k][d] = (k == 0) ? v : host40_mont_form(v);
      v = host40_mulmod(v, g);
    }
    for (int s = 0; s < 8; ++s) g = host40_mulmod(g, g);
  }
  return T;
}
static_assert(make_pow_table40().t[0][3] == host40_mulmod(8, k40H), "row 0");
static_assert(make_pow_table40().t[2][1] == host40_mont_form(host40_pow2(65536)), "row 2");

#ifdef __CUDACC__
static __device__ const PowTable40 k40PowTable = make_pow_table40();

// q = floor(2^53 z / 3^40) for a state z (see k40Rhi): the high word of the
// 182-bit product z*R, from z*Rhi (128 bits) plus the carry that the high
// word of z*Rlo brings into it (the low word of z*Rlo cannot change it).
__device__ __forceinline__ uint64_t quot40(uint64_t z) {
  const uint64_t alo = z * k40Rhi;
  const uint64_t ahi = umulhi(z, k40Rhi);
  const uint64_t bhi = umulhi(z, k40Rlo);
  return ahi + (alo + bhi < alo ? 1 : 0);
}

// The variate bits of bits40 when q0 >= 2^32 (a variate of at least 2^-21;
// the caller routes smaller ones to the exact path): q0's leading one is in
// its high word, and the digits taken from q1 come from q1's high word only.
// On 32-bit words: the mantissa's high word is q0 funnel-shifted left by t,
// its low word q0's low word funnel-shifted over q1's high word (placed at
// the top of a word), and (1032 - c) << 20, c = t + 11 the leading zeros of
// q0's high word, puts the exponent on the high word (the mantissa's leading
// one then lifts it by one).
__device__ __forceinline__ uint64_t bits40_fast(uint64_t q0, uint64_t q1) {
  const uint32_t q0l = (uint32_t)q0, q0h = (uint32_t)(q0 >> 32), q1h = (uint32_t)(q1 >> 32);
  uint32_t hi, lo;
  asm("{\n\t"
      ".reg .u32 c, t, x, mh, ew;\n\t"
      "clz.b32 c, %3;\n\t"
      "sub.u32 t, c, 11;\n\t"                 // 0..20
      "shf.l.clamp.b32 mh, %2, %3, t;\n\t"
      "shl.b32 x, %4, 11;\n\t"
      "shf.l.clamp.b32 %1, x, %2, t;\n\t"
      "shl.b32 ew, c, 20;\n\t"
      "sub.u32 ew, 0x40800000, ew;\n\t"       // (1032 - c) << 20
      "add.u32 %0, mh, ew;\n\t"
      "}"
      : "=r"(hi), "=r"(lo)
      : "r"(q0l), "r"(q0h), "r"(q1h));
  return ((uint64_t)hi << 32) | lo;
}
static_assert((1032u << 20) == 0x40800000u, "exponent constant of bits40_fast");

// Eq. 3 with the quotient q of z: 2^53 z - q 3^40, which lies in [1, 3^40),
// so arithmetic modulo 2^64 gives it exactly.
__device__ __forceinline__ uint64_t rem40(uint64_t z, uint64_t q) {
  return (z << 53) - q * k40M;
}

// Montgomery product a*b*2^-64 mod m for a, b < m.  The sum t + u*m is a
// multiple of 2^64 below m^2 + 2^64 m, so its high word lies below 2m < 2^65:
// the carry out of the 64-bit addition is tracked, then m is taken out once.
__device__ __forceinline__ uint64_t mont40(uint64_t a, uint64_t b) {
  const uint64_t tlo = a * b;
  const uint64_t thi = umulhi(a, b);
  const uint64_t u = tlo * k40NegMinv;
  const uint64_t uhi = umulhi(u, k40M);
  // t + u*m = (thi + uhi + [tlo != 0]) * 2^64: the low words cancel, with a
  // carry exactly when tlo is nonzero.
  const uint64_t s1 = thi + uhi;
  const bool c1 = s1 < thi;
  const uint64_t s = s1 + (tlo != 0 ? 1 : 0);
  const bool c2 = s < s1;
  return (c1 || c2 || s >= k40M) ? s - k40M : s;
}

// (e0 + 53*x) mod P for e0 < P and 53*x < P.
__device__ __forceinline__ uint64_t exponent_add40(uint64_t e0, uint64_t x) {
  const uint64_t e = e0 + 53ull * x;
  return e >= k40P ? e - k40P : e;
}

// Eq. 2 (modulus 3^40): floor(3^40/2) * 2^e mod 3^40 from the table.
__device__ __forceinline__ uint64_t seed_state40(uint64_t e) {
  uint64_t z = __ldg(&k40PowTable.t[0][e & 255]);
#pragma unroll
  for (int k = 1; k < k40TabRows; ++k)
    z = mont40(z, __ldg(&k40PowTable.t[k][(e >> (8 * k)) & 255]));
  return z;
}

// FP64 bits of 0.q0 q1 ... (base 2^53) rounded toward zero, for q0 != 0:
// the 53 digits from q0's leading one, continued into q1.  q0 has t leading
// zeros in its 53-bit window, so the variate lies in [2^-(t+1), 2^-t).
__device__ __forceinline__ uint64_t bits40(uint64_t q0, uint64_t q1) {
  const uint32_t t = (uint32_t)__clzll((long long)q0) - 11u;
  const uint64_t mant = (q0 << t) | (q1 >> (53u - t));  // in [2^52, 2^53)
  return ((uint64_t)(1021u - t) << 52) + mant;          // the leading one lifts the exponent
}

// Eq. 3 run backwards (Montgomery-style, R = 2^53) with its exact quotient.
// For consecutive states z_(k-1), z_k = 2^53 z_(k-1) - Q 3^40 with
// Q = floor(2^53 z_(k-1) / 3^40) < 2^53:
//   Q = (z_k * m') mod 2^53                      (m' = -3^-40 mod 2^53),
//   z_(k-1) = (z_k + Q 3^40) / 2^53              (an exact division).
// So one step back yields the previous state and the quotient digit that
// the forward step would have had to estimate: no undecided band.  S = z_k +
// Q 3^40 < 2^117 is summed on 32-bit limbs.  Its low 53 bits are zero, so
// limb 0 is zero and carries 1 into limb 1 exactly when the low word of z_k
// is non-zero (the low word of Q 3^40 then being its complement), and the
// product's own low word is never formed.
constexpr uint64_t k40Mp = (0 - inv_mod_2_64(k40M)) & kMask53;  // -3^-40 mod 2^53
static_assert(((k40M * k40Mp + 1) & kMask53) == 0, "3^40 * m' = -1 mod 2^53");
__device__ __forceinline__ uint64_t back40(uint64_t z, uint64_t& q) {
  constexpr uint32_t mp0 = (uint32_t)k40Mp, mp1 = (uint32_t)(k40Mp >> 32);
  constexpr uint32_t m0 = (uint32_t)k40M, m1 = (uint32_t)(k40M >> 32);
  uint32_t r0, r1, u0, u1;
  // outputs are written last: no output register may share an input's
  asm("{\n\t"
      ".reg .u32 a0, a1, q0, q1, th, h0, x, l1, l2, l3;\n\t"
      ".reg .u64 t;\n\t"
      "mov.u32 a0, %4;\n\t"
      "mov.u32 a1, %5;\n\t"
      "mul.wide.u32 t, a0, %6;\n\t"            // Q = z m' mod 2^53
      "mov.b64 {q0, th}, t;\n\t"
      "mad.lo.u32 th, a0, %7, th;\n\t"
      "mad.lo.u32 th, a1, %6, th;\n\t"
      "and.b32 q1, th, 0x1FFFFF;\n\t"
      "mul.hi.u32 h0, q0, %8;\n\t"             // S = z + Q m from limb 1 up
      "add.cc.u32 x, a0, 0xFFFFFFFF;\n\t"      // carry = (low word of z != 0)
      "addc.cc.u32 l1, h0, a1;\n\t"
      "addc.u32 l2, 0, 0;\n\t"
      "mad.lo.cc.u32 l1, q0, %9, l1;\n\t"
      "madc.hi.cc.u32 l2, q0, %9, l2;\n\t"
      "addc.u32 l3, 0, 0;\n\t"
      "mad.lo.cc.u32 l1, q1, %8, l1;\n\t"
      "madc.hi.cc.u32 l2, q1, %8, l2;\n\t"
      "addc.u32 l3, l3, 0;\n\t"
      "mad.lo.cc.u32 l2, q1, %9, l2;\n\t"
      "madc.hi.u32 l3, q1, %9, l3;\n\t"
      "shf.r.clamp.b32 %0, l1, l2, 21;\n\t"    // z_(k-1) = S >> 53
      "shf.r.clamp.b32 %1, l2, l3, 21;\n\t"
      "mov.u32 %2, q0;\n\t"
      "mov.u32 %3, q1;\n\t"
      "}"
      : "=r"(r0), "=r"(r1), "=r"(u0), "=r"(u1)
      : "r"((uint32_t)z), "r"((uint32_t)(z >> 32)), "n"(mp0), "n"(mp1), "n"(m0), "n"(m1));
  q = ((uint64_t)u1 << 32) | u0;
  return ((uint64_t)r1 << 32) | r0;
}

// A variate below 2^-53 (q0 == 0, about once in 2^53 variates): its leading
// one is in the next window (the variate is at least 3^-40 > 2^-64), so the
// digits come from q1 and q2, 53 places further down.  z1 is the state whose
// quotient is q1.
static __device__ __noinline__ uint64_t bits40_small(uint64_t z1, uint64_t q1) {
  const uint64_t q2 = quot40(rem40(z1, q1));
  const uint32_t t = (uint32_t)__clzll((long long)q1) - 11u;
  const uint64_t mant = (q1 << t) | (q2 >> (53u - t));
  return ((uint64_t)(1021u - 53u - t) << 52) + mant;
}
#endif  // __CUDACC__

}  // namespace bcn
