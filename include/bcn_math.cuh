// bcn_math.cuh -- constants and modular arithmetic of the alpha_{2,3} generator
// for sm_103a.  Everything here is integer arithmetic on 64-bit words; the
// only floating-point value is r3i, used by the FP64-pipe conversion variant.
//
// The generator (Beliakov et al., Algorithm BB with Eq. 2 and Eq. 3):
//   seed a in [3^33+100, 2^53];  z_0 = 2^(a-3^33) * floor(3^33/2) mod 3^33;
//   z_k = 2^53 z_(k-1) mod 3^33;  variate = z_k * 3^-33.
// Variate i (0-based) of a stream therefore has the state
//   z = 2^e * floor(3^33/2) mod 3^33,  e = (a - 3^33 + 53*(i+1)) mod P,
// with P = 2*3^32 the period (Sec. 1).  Output is "step, then emit".
#pragma once
#include <cstdint>

namespace bcn {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------- constants
constexpr uint64_t kM = 5559060566555523ULL;       // 3^33 (Eq. 3 modulus)
constexpr uint64_t kH = kM / 2;                    // floor(3^33/2)   (Eq. 2)
constexpr uint64_t kP = 2ULL * (kM / 3);           // 2*3^32, period  (Sec. 1)
constexpr uint64_t kTwo53 = 1ULL << 53;
constexpr uint64_t kMask53 = kTwo53 - 1;
constexpr uint64_t kSeedMin = kM + 100;            // Algorithm BB, step 1
constexpr uint64_t kSeedMax = kTwo53;              // Algorithm BB, step 1

constexpr uint64_t pow3(int k) { return k == 0 ? 1 : 3 * pow3(k - 1); }
static_assert(pow3(33) == kM, "m = 3^33");

// Barrett's mu = floor(2^(2k)/m) with k = 53 (Sec. 2.1, Barrett and
// Modified Barrett); Fig. 4 prints it as 0x33D9481681D79D.
constexpr uint64_t kMu = (uint64_t)(((u128)1 << 106) / kM);
static_assert(kMu == 0x33D9481681D79DULL, "mu as printed in Fig. 4");

// r3i = RN(1/3^33) (Fig. 4).  Its significand as an integer: r3i = kMr*2^-105.
// kMu + 1 = 2*kMr, so the Barrett product z*mu also yields the exact product
// z*r3i*2^106 = z*mu + z that the integer conversion rounds.
constexpr uint64_t kMr = 0x19ECA40B40EBCFULL;
constexpr double kR3i = 0x1.9eca40b40ebcfp-53;
static_assert(kMu + 1 == 2 * kMr, "mu + 1 = 2 * significand(r3i)");
static_assert(kR3i == 1.0 / 5559060566555523.0, "r3i as printed in Fig. 4");
static_assert(kR3i == (double)kMr * 0x1p-105, "r3i = kMr * 2^-105");

// K = mu + 1 = 2*kMr: z*K = z*r3i*2^106 exactly, and floor(z*K / 2^53) is a
// Barrett quotient estimate for 2^53 z / m (see shared_step_f64).
constexpr uint64_t kK = kMu + 1;
constexpr uint32_t kK0 = (uint32_t)kK, kK1 = (uint32_t)(kK >> 32);
constexpr uint32_t kM0 = (uint32_t)kM, kM1 = (uint32_t)(kM >> 32);

// -m^-1 mod 2^53 for the Montgomery-style reduction with R = 2^53.
constexpr uint64_t inv_mod_2_64(uint64_t x) {  // Newton: y <- y(2 - xy)
  uint64_t y = x;  // correct to 3 bits for odd x
  for (int i = 0; i < 6; ++i) y *= 2 - x * y;
  return y;
}
constexpr uint64_t kNegMinv53 = (0 - inv_mod_2_64(kM)) & kMask53;
static_assert(((kM * kNegMinv53 + 1) & kMask53) == 0, "m * (-m^-1) = -1 mod 2^53");

// ------------------------------------------------------- host-side helpers
constexpr uint64_t host_mulmod(uint64_t a, uint64_t b) {
  return (uint64_t)(((u128)a * b) % kM);
}
constexpr uint64_t host_pow2(uint64_t e) {  // 2^e mod m, square-and-multiply
  uint64_t r = 1, g = 2;
  while (e) {
    if (e & 1) r = host_mulmod(r, g);
    g = host_mulmod(g, g);
    e >>= 1;
  }
  return r;
}
static_assert(host_pow2(kP) == 1 && host_pow2(kP / 2) == kM - 1, "period");
// floor(j * 2^64 / m): the precomputed quotient of a fixed multiplier j < m.
constexpr uint64_t host_mulmod_quotient(uint64_t j) {
  return (uint64_t)(((u128)j << 64) / kM);
}

// Fixed-base exponent table: 2^e mod m for e < P < 2^56 is the product of
// one entry per byte of e.  Row 0 also carries the floor(3^33/2) factor of
// Eq. 2, so  z = T[0][e_0] * T[1][e_1] * ... * T[6][e_6]  mod m.
// This is square-and-multiply with the squarings of the fixed base 2 done
// once, at compile time.
constexpr int kTabRows = 7;
struct PowTable {
  uint64_t t[kTabRows][256];
};
constexpr PowTable make_pow_table() {
  PowTable T{};
  uint64_t g = 2;  // 2^(256^k)
  for (int k = 0; k < kTabRows; ++k) {
    T.t[k][0] = (k == 0) ? kH : 1;
    for (int d = 1; d < 256; ++d) T.t[k][d] = host_mulmod(T.t[k][d - 1], g);
    for (int s = 0; s < 8; ++s) g = host_mulmod(g, g);
  }
  return T;
}
static_assert(make_pow_table().t[1][1] == host_pow2(256), "table row 1");
static_assert(make_pow_table().t[0][5] == host_mulmod(32, kH), "table row 0");

// Exponent of the state that precedes variate `index` of a stream whose
// first call starts at absolute count i0:  (a - 3^33 + 53*i0) mod P.
inline uint64_t host_exponent_base(uint64_t seed, uint64_t i0) {
  return (uint64_t)(((u128)(seed - kM) + (u128)53 * (i0 % kP)) % kP);
}

#ifdef __CUDACC__
// --------------------------------------------------------- device helpers
// One copy per translation unit, constant-initialised when the module loads.
static __device__ const PowTable kPowTable = make_pow_table();

__device__ __forceinline__ uint64_t umulhi(uint64_t a, uint64_t b) {
  return __umul64hi(a, b);
}

// x*y mod m for x, y < m (Barrett, Sec. 2.1.2, with k = 53: q1 = t >> 52,
// q3 = (q1*mu) >> 54 lies in [Q-2, Q], so t - q3*m < 3m < 2^55 fits a word).
__device__ __forceinline__ uint64_t mulmod(uint64_t x, uint64_t y) {
  uint64_t lo = x * y, hi = umulhi(x, y);
  uint64_t q1 = (hi << 12) | (lo >> 52);
  uint64_t q3 = (umulhi(q1, kMu) << 10) | ((q1 * kMu) >> 54);
  uint64_t r = lo - q3 * kM;
  r = (r >= kM) ? r - kM : r;
  r = (r >= kM) ? r - kM : r;
  return r;
}

// z*j mod m for a fixed multiplier j with its precomputed quotient
// jq = floor(j * 2^64 / m): q = floor(z*jq / 2^64) is floor(z*j/m) or one
// less, so z*j - q*m lies in [0, 2m) and one subtraction finishes (the
// precomputed-quotient modular product known from Shoup's NTL).
__device__ __forceinline__ uint64_t mulmod_pre(uint64_t z, uint64_t j, uint64_t jq) {
  const uint64_t q = umulhi(z, jq);
  const uint64_t r = z * j - q * kM;
  return (r >= kM) ? r - kM : r;
}

// (e0 + 53*x) mod P for e0 < P, any 64-bit x.
__device__ __forceinline__ uint64_t exponent_add(uint64_t e0, uint64_t x) {
  uint64_t e = e0 + 53ULL * (x % kP);  // < 2^59
  return e % kP;
}

// 2^e * floor(3^33/2) mod m (Eq. 2) from the fixed-base table: 6 products.
__device__ __forceinline__ uint64_t seed_state_table(uint64_t e) {
  uint64_t z = __ldg(&kPowTable.t[0][e & 255]);
#pragma unroll
  for (int k = 1; k < kTabRows; ++k)
    z = mulmod(z, __ldg(&kPowTable.t[k][(e >> (8 * k)) & 255]));
  return z;
}

// The same value by plain right-to-left square-and-multiply (about 52
// squarings and 26 products); kept as a selectable variant.
__device__ __forceinline__ uint64_t seed_state_sqmul(uint64_t e) {
  uint64_t r = kH, g = 2;
  while (e) {
    if (e & 1) r = mulmod(r, g);
    g = mulmod(g, g);
    e >>= 1;
  }
  return r;
}

// ---------------------------------------------------------------- steps
// Modified Barrett (Sec. 2.1.3): q3 = floor(mu*z / 2^53) lies in {Q-1, Q}
// for Q = floor(2^53 z / m); r = 2^53 - (q3*m mod 2^53); if r >= m, r -= m.
// For m = 3^33 the 53-bit wrap of x - q3*m cannot happen: q3 = Q-1 needs
// frac(2^53 z/m) < z*(2^106/m - mu)/2^53 < m/2^53 ~ 0.6172, while a wrap
// needs frac(2^53 z/m) >= 2^53/m - 1 ~ 0.6203.  The step consumes the
// product z*mu, which the caller forms once and shares with the conversion.
__device__ __forceinline__ uint64_t barrett_from_product(uint64_t phi, uint64_t plo) {
  uint64_t q3 = (phi << 11) | (plo >> 53);
  uint64_t r = kTwo53 - ((q3 * kM) & kMask53);
  return (r >= kM) ? r - kM : r;
}

// Montgomery-style inverse step with R = 2^53: 2^-53 z mod m, i.e. Eq. 3
// run backwards.  u = -z/m mod 2^53 makes z + u*m divisible by 2^53, and
// (z + u*m)/2^53 = floor(u*m/2^53) + 1 lies in [1, m-1] for 0 < z < m, so
// no final subtraction is needed.
__device__ __forceinline__ uint64_t montgomery_back(uint64_t z) {
  uint64_t u = (z * kNegMinv53) & kMask53;
  uint64_t hi = umulhi(u, kM), lo = u * kM;
  return ((hi << 11) | (lo >> 53)) + 1;
}

// L'Ecuyer's decomposition (Sec. 2.1.1) with a = 2^25: m = a*q + r, r < a,
// a^2 < m, so a*s mod m = a*(s mod q) - floor(s/q)*r, corrected by one "+ m".
// For s < 4m the intermediate stays in (-m, m) because floor(s/q)*r <
// 4*a*r <= 2^52 < m.  The step of Eq. 3 is two applications: 2^25 * (4z) and
// then 2^25 * (2 * that).  The quotient floor(s/q) is an exact integer
// division by the constant q.
constexpr uint64_t kLq = kM >> 25, kLr = kM & ((1ull << 25) - 1);
static_assert(kLr < (1ull << 25) && (1ull << 50) < kM, "L'Ecuyer needs a^2 < m");
__device__ __forceinline__ uint64_t lecuyer_mul25(uint64_t s) {
  const uint64_t t = s / kLq;
  const int64_t v = (int64_t)((s - t * kLq) << 25) - (int64_t)(t * kLr);
  return v < 0 ? (uint64_t)(v + (int64_t)kM) : (uint64_t)v;
}
__device__ __forceinline__ uint64_t lecuyer_step(uint64_t z) {
  return lecuyer_mul25(lecuyer_mul25(z << 2) << 1);
}

// Barrett's algorithm (Sec. 2.1.2) with k = 53 applied to x = 2^53 z:
// q1 = x >> 52 = 2z, q3 = (mu * q1) >> 54 in [Q-2, Q], r = (x - q3*m) mod 2^54
// (x mod 2^54 is (z & 1) << 53), then at most two subtractions of m.
__device__ __forceinline__ uint64_t barrett_classic_step(uint64_t z) {
  const uint64_t q1 = z << 1;
  const uint64_t q3 = (umulhi(q1, kMu) << 10) | ((q1 * kMu) >> 54);
  const uint64_t mask54 = (1ull << 54) - 1;
  uint64_t r = (((z & 1ull) << 53) - ((q3 * kM) & mask54)) & mask54;
  r = (r >= kM) ? r - kM : r;
  r = (r >= kM) ? r - kM : r;
  return r;
}

// ---------------------------------------------------------- conversions
// FP64 bits of RN(z * r3i) by integer arithmetic only.  p = z*mu + z =
// z*r3i*2^106 exactly (< 2^106); the variate is p*2^-106 rounded to 53
// significant bits, ties to even.  q = p >> 53 is in [1, 2^53); lz leading
// zeros of q below bit 52 give the binary exponent -1-lz.
__device__ __forceinline__ uint64_t f64_bits_from_p(uint64_t phi, uint64_t plo) {
  uint64_t q = (phi << 11) | (plo >> 53);
  uint64_t low = plo & kMask53;
  int lz = __clzll((long long)q) - 11;                // 0 .. 52
  uint64_t mant = (q << lz) | (low >> (53 - lz));      // 53 significant bits
  uint64_t rest = low << (11 + lz);                    // dropped bits, top-aligned
  const uint64_t half = 1ULL << 63;
  uint64_t up = (rest > half) | ((rest == half) & (mant & 1));
  return ((uint64_t)(1021 - lz) << 52) + mant + up;   // carry may bump exponent
}

// p = z*(mu+1) as a 128-bit (hi, lo) pair, from the Barrett product z*mu.
__device__ __forceinline__ void p_from_barrett_product(uint64_t z, uint64_t phi,
                                                       uint64_t plo, uint64_t& qhi,
                                                       uint64_t& qlo) {
  qlo = plo + z;
  qhi = phi + (qlo < z ? 1ULL : 0ULL);
}

// ------------------------------------------------- shared-quotient step
// One Barrett-style step of Eq. 3 and the FP64 variate of the current state
// from a single 106-bit product p = z*K (K = mu + 1 = 2*significand(r3i)):
//
//  * Reduction.  q = floor(p / 2^53) = floor(z*(mu+1)/2^53) lies in {Q, Q+1}
//    for Q = floor(2^53 z / m): z*(mu+1)/2^53 exceeds 2^53 z/m (mu+1 > 2^106/m)
//    by less than z/2^53 < 1.  So r = 2^53 z - q*m lies in (-m, m), is exact in
//    64-bit two's complement, and one conditional "+ m" finishes the step --
//    Barrett's quotient estimate (Sec. 2.1.2) with the output scale as the
//    precomputed reciprocal.
//  * Conversion.  The variate RN(z*r3i) = RN(p * 2^-106).  With lz the number
//    of leading zeros of q below bit 52, the significand is p >> (53-lz) and
//    the first dropped bit (the guard bit) decides the rounding: p = 2*z*M_r
//    with M_r odd, so an exact tie would need v2(z) >= bitlen(z) - 2, i.e.
//    z = 2^k or 3*2^k, and none of those is a tie.  Round-to-nearest-even is
//    therefore "add the guard bit": bits = (G + (E << 53) + 1) >> 1 with
//    G = p >> (52-lz) (significand and guard) and E = 1021 - lz, where a
//    rounding carry moves into the exponent field by itself.
//  The fast path needs the top word of q to be non-zero (variate >= 2^-21);
//  the rest (probability about 2^-21) takes the general conversion.
// Everything is 32-bit words: 4 wide multiply-adds form p, 3 multiplies give
// q*m mod 2^64, funnel shifts do the normalisation.
__device__ __forceinline__ uint64_t shared_step_f64(uint64_t& z) {
  const uint32_t z0 = (uint32_t)z, z1 = (uint32_t)(z >> 32);
  const uint64_t t0 = (uint64_t)z0 * kK0;
  uint64_t t1 = (uint64_t)z0 * kK1 + (t0 >> 32);
  t1 = (uint64_t)z1 * kK0 + t1;
  const uint64_t t2 = (uint64_t)z1 * kK1 + (t1 >> 32);
  const uint32_t w1 = (uint32_t)t1, w2 = (uint32_t)t2, w3 = (uint32_t)(t2 >> 32);
  const uint32_t q0 = __funnelshift_r(w1, w2, 21);
  const uint32_t q1 = __funnelshift_r(w2, w3, 21);
  // next state: 2^53 z - q*m, then + m if negative
  const uint64_t qm = (uint64_t)q0 * kM0;
  const uint32_t qm_hi = (uint32_t)(qm >> 32) + q0 * kM1 + q1 * kM0;
  uint64_t r = ((uint64_t)(z0 << 21) << 32) - (((uint64_t)qm_hi << 32) | (uint32_t)qm);
  if ((int64_t)r < 0) r += kM;
  // conversion of the current state
  uint64_t bits;
  if (__builtin_expect(q1 != 0, 1)) {
    const uint32_t c = __clz((int)q1);        // 11 .. 31, lz = c - 11
    const uint32_t s = c - 10;                // lz + 1
    const uint32_t lh = w1 << 11;             // low bits of p below q, top-aligned
    const uint32_t g_hi = __funnelshift_l(q0, q1, s);
    const uint32_t g_lo = __funnelshift_l(lh, q0, s);
    const uint64_t x = (((uint64_t)g_hi << 32) | g_lo) + (((uint64_t)(1032 - c) << 53) | 1ULL);
    bits = x >> 1;
  } else {
    bits = f64_bits_from_p(t2, (t1 << 32) | (uint32_t)t0);
  }
  z = r;
  return bits;
}

// shared_step_f64 without its rare branch: the fast-path conversion is always
// taken, and `rare` is raised when its precondition (top word of q non-zero,
// variate >= 2^-21) fails, in which case the returned bits are meaningless
// and the caller recomputes them with shared_step_f64.  The state advance is
// exact either way.
__device__ __forceinline__ uint64_t shared_step_f64_fast(uint64_t& z, bool& rare) {
  const uint32_t z0 = (uint32_t)z, z1 = (uint32_t)(z >> 32);
  const uint64_t t0 = (uint64_t)z0 * kK0;
  uint64_t t1 = (uint64_t)z0 * kK1 + (t0 >> 32);
  t1 = (uint64_t)z1 * kK0 + t1;
  const uint64_t t2 = (uint64_t)z1 * kK1 + (t1 >> 32);
  const uint32_t w1 = (uint32_t)t1, w2 = (uint32_t)t2, w3 = (uint32_t)(t2 >> 32);
  const uint32_t q0 = __funnelshift_r(w1, w2, 21);
  const uint32_t q1 = __funnelshift_r(w2, w3, 21);
  const uint64_t qm = (uint64_t)q0 * kM0;
  const uint32_t qm_hi = (uint32_t)(qm >> 32) + q0 * kM1 + q1 * kM0;
  uint64_t r = ((uint64_t)(z0 << 21) << 32) - (((uint64_t)qm_hi << 32) | (uint32_t)qm);
  if ((int64_t)r < 0) r += kM;
  rare |= (q1 == 0);
  const uint32_t c = __clz((int)q1);
  const uint32_t s = c - 10;
  const uint32_t lh = w1 << 11;
  const uint32_t g_hi = __funnelshift_l(q0, q1, s);
  const uint32_t g_lo = __funnelshift_l(lh, q0, s);
  const uint64_t x = (((uint64_t)g_hi << 32) | g_lo) + (((uint64_t)(1032 - c) << 53) | 1ULL);
  z = r;
  return x >> 1;
}

// The same step written as inline PTX on 32-bit words for a chain that holds
// Z = z 2^10 instead of z.  With Kb = 2K (below 2^55), Z*Kb = p 2^11, so the
// quotient window q = floor(p / 2^53) is the high word of Z*Kb and the 32
// bits of p just below it are that product's word 1: no funnel shifts.  The
// next state comes out scaled as well: 2^53 z - q m times 2^10 is
// (z mod 2) 2^63 - q (m 2^10) mod 2^64 (z mod 2 is bit 10 of Z, so its term
// is Z's low word shifted left by 21), and since |2^53 z - q m| < m the
// scaled remainder is below 2^62.4 in magnitude: its sign bit says whether
// m 2^10 is to be added.  The rounding is the unscaled step's: one carry
// chain plus a funnel shift.  Every operation maps to one instruction, and
// the tiled FP64 kernel takes 3 fewer per variate than with the chain on z
// (measured 787 against 730 G variates/s at 2^28 in a test kernel).  `qmin`
// is a running minimum of q's top word: it is 0 exactly when some step of the
// run left the fast path (variate below 2^-21), and the caller then redoes
// the run.
constexpr uint32_t kZShift = 10;                 // Z = z << kZShift
constexpr uint64_t kKb = kK << 1;                // 2K < 2^55
constexpr uint64_t kMs = kM << kZShift;          // m 2^10 < 2^63
constexpr uint32_t kKb0 = (uint32_t)kKb, kKb1 = (uint32_t)(kKb >> 32);
constexpr uint32_t kMs0 = (uint32_t)kMs, kMs1 = (uint32_t)(kMs >> 32);
static_assert((kK >> 54) == 0 && (kMs >> 62) == 1, "scaled step constants");
__device__ __forceinline__ uint64_t shared_step_f64_ptx(uint64_t& Z, uint32_t& qmin) {
  const uint32_t z0 = (uint32_t)Z, z1 = (uint32_t)(Z >> 32);
  uint32_t r0, r1, b0, b1, qm_out;
  // outputs are early-clobber: none shares a register with an input
  asm("{\n\t"
      ".reg .u32 h0, w1, x, y, q0, q1, ml, mh, zh, c, s, gh, gl, ew, x0, x1;\n\t"
      ".reg .u64 qm;\n\t"
      ".reg .pred neg;\n\t"
      "mul.hi.u32 h0, %5, %7;\n\t"          // Z*Kb on 32-bit carry chains:
      "mad.lo.cc.u32 w1, %5, %8, h0;\n\t"   // word 1 (the bits of p below q)
      "madc.hi.u32 x, %5, %8, 0;\n\t"
      "mad.lo.cc.u32 w1, %6, %7, w1;\n\t"
      "madc.hi.cc.u32 x, %6, %7, x;\n\t"
      "addc.u32 y, 0, 0;\n\t"
      "mad.lo.cc.u32 q0, %6, %8, x;\n\t"    // words 2, 3: q
      "madc.hi.u32 q1, %6, %8, y;\n\t"
      "mul.wide.u32 qm, q0, %9;\n\t"        // q (m 2^10) mod 2^64
      "mov.b64 {ml, mh}, qm;\n\t"
      "mad.lo.u32 mh, q0, %10, mh;\n\t"
      "mad.lo.u32 mh, q1, %9, mh;\n\t"
      "shl.b32 zh, %5, 21;\n\t"             // (z mod 2) 2^31
      "sub.cc.u32 %0, 0, ml;\n\t"
      "subc.u32 %1, zh, mh;\n\t"
      "setp.lt.s32 neg, %1, 0;\n\t"
      "@neg add.cc.u32 %0, %0, %9;\n\t"
      "@neg addc.u32 %1, %1, %10;\n\t"
      "min.u32 %4, %11, q1;\n\t"
      "clz.b32 c, q1;\n\t"
      "sub.u32 s, c, 10;\n\t"
      "shf.l.clamp.b32 gh, q0, q1, s;\n\t"
      "shf.l.clamp.b32 gl, w1, q0, s;\n\t"
      "mad.lo.u32 ew, c, 0xFFE00000, 0x81000000;\n\t"
      "add.cc.u32 x0, gl, 1;\n\t"
      "addc.u32 x1, gh, ew;\n\t"
      "shf.r.clamp.b32 %2, x0, x1, 1;\n\t"
      "shr.b32 %3, x1, 1;\n\t"
      "}"
      : "=&r"(r0), "=&r"(r1), "=&r"(b0), "=&r"(b1), "=&r"(qm_out)
      : "r"(z0), "r"(z1), "n"(kKb0), "n"(kKb1), "n"(kMs0), "n"(kMs1), "r"(qmin));
  Z = ((uint64_t)r1 << 32) | r0;
  qmin = qm_out;
  return ((uint64_t)b1 << 32) | b0;
}
static_assert((1032u << 21) == 0x81000000u, "exponent constant of the PTX step");

// The state advance of shared_step_f64_ptx alone, on a scaled chain.
__device__ __forceinline__ uint64_t shared_advance_scaled(uint64_t Z) {
  const uint64_t q = (uint64_t)(((u128)Z * kKb) >> 64);
  uint64_t r = ((uint64_t)((uint32_t)Z << 21) << 32) - q * kMs;
  if ((int64_t)r < 0) r += kMs;
  return r;
}


// ------------------------------------ backward step with its exact quotient
// Eq. 3 run backwards by a Montgomery-style reduction with R = 2^53 gives the
// exact quotient digit of the state it steps to at no extra cost.  For
// consecutive states z_(k-1) and z_k = 2^53 z_(k-1) mod m, let
// Q = floor(2^53 z_(k-1) / m) < 2^53.  Then z_k + Q m = 2^53 z_(k-1), so
//   Q = -z_k m^-1 mod 2^53 = (z_k * m') mod 2^53        (m' = -m^-1 mod 2^53),
//   z_(k-1) = (z_k + Q m) / 2^53 = floor(Q m / 2^53) + 1    (0 < z_k < 2^53).
// The chain holds y = z - 1, so that z_k m' = y m' + m' is one multiply-add and
// y_(k-1) = floor(Q m / 2^53) needs no final add.
//
// Q is the variate z_(k-1)/m truncated to 53 fraction bits, and the FP32
// variate (RN(z*r3i) toward zero) is the float made of Q's leading 24
// significant bits, W, unless the bits of Q below W are all ones or all ones
// but the last.  Proof: r3i = M_r 2^-105 exceeds 1/m by less than 2^-106, so
// z*r3i lies in (Q 2^-53, (Q + 1.62) 2^-53).  If the bits below W are at most
// all ones minus 2, the next float B above W is at least (Q + 3) 2^-53, and
// RN to 53 bits (whose ulp below 1 is at most 2^-53) cannot reach B from below
// B - 1.38 * 2^-53; nor can it go below Q 2^-53, a double.  So every value it
// can take truncates to W.
//
// The step is computed on X = Q 2^11, which is what a multiplier of
// m' 2^11 mod 2^64 gives directly: X = (y + 1)(m' 2^11) mod 2^64 (a 64-bit
// product needs no mask), and y_(k-1) = floor(Q m / 2^53) = floor(X m / 2^64)
// is the high word of X m with no final shift.  X = (u1:u0) on 32-bit words,
// Q's leading one at bit 63 - c with c = leading zeros of u1.  The high word
// of (u1:u0) << c, shifted right by 8, is W with its leading one at bit 23,
// and the float's bits are W + (125 - c) 2^23 (biased exponent 126 - c, the
// leading one adding its 1).  The flag is v = ~(u0 | 0xFFF) << c, zero when
// Q's bits 1 .. 20 - c are all ones: a superset of the cases above, since
// Q's bits below W are bits 0 .. 28 - c (it also flags a one-in-2^(20-c)
// share of the other steps, about one step in 2^16 overall).  Q below 2^33
// (variate below 2^-20) gives c >= 20 and v = 0, and u1 = 0 makes
// bfind.shiftamt return 2^32 - 1 and v = 0 as well.  `qmin` keeps the
// running minimum of v: it is 0 when some step of the run needs the exact
// path, and the caller redoes the run.  The product X m is formed with
// 32-bit carry chains (measured fewer instructions than 64-bit multiply-adds
// with zero-extended addends), and the whole step takes 24.1 instructions per
// variate in the tiled kernel against 28.2 for the same step on Q itself.
constexpr uint64_t kMp = kNegMinv53;  // m' = -m^-1 mod 2^53
static_assert((kMp >> 53) == 0, "m' < 2^53");
static_assert((kM >> 32) < (1u << 21), "m < 2^53");
constexpr uint64_t kMpX = kMp << 11;  // m' 2^11 mod 2^64
constexpr uint32_t kMpX0 = (uint32_t)kMpX, kMpX1 = (uint32_t)(kMpX >> 32);
__device__ __forceinline__ uint32_t back_step_f32_ptx(uint64_t& y, uint32_t& qmin) {
  const uint32_t y0 = (uint32_t)y, y1 = (uint32_t)(y >> 32);
  uint32_t r0, r1, b, qo;
  // outputs are early-clobber: none shares a register with an input
  asm("{\n\t"
      ".reg .u32 u0, u1, th, h0, w1, x, w, c, mant, e, nv;\n\t"
      ".reg .u64 t;\n\t"
      "mad.wide.u32 t, %4, %6, %8;\n\t"         // X = (y + 1) m' 2^11 mod 2^64
      "mov.b64 {u0, th}, t;\n\t"
      "mad.lo.u32 th, %4, %7, th;\n\t"
      "mad.lo.u32 u1, %5, %6, th;\n\t"
      "mul.hi.u32 h0, u0, %9;\n\t"              // high word of X m:
      "mad.lo.cc.u32 w1, u0, %10, h0;\n\t"      // y_(k-1) = floor(X m / 2^64)
      "madc.hi.u32 x, u0, %10, 0;\n\t"
      "mad.lo.cc.u32 w1, u1, %9, w1;\n\t"
      "madc.hi.cc.u32 x, u1, %9, x;\n\t"
      "addc.u32 w, 0, 0;\n\t"
      "mad.lo.cc.u32 %0, u1, %10, x;\n\t"
      "madc.hi.u32 %1, u1, %10, w;\n\t"
      "bfind.shiftamt.u32 c, u1;\n\t"           // leading zeros of u1; 2^32-1 if u1 = 0
      "shf.l.clamp.b32 mant, u0, u1, c;\n\t"
      "shr.b32 mant, mant, 8;\n\t"              // W, leading one at bit 23
      "mad.lo.u32 e, c, 0xFF800000, 0x3E800000;\n\t"  // (125 - c) << 23
      "or.b32 nv, u0, 0xFFF;\n\t"
      "not.b32 nv, nv;\n\t"
      "shl.b32 nv, nv, c;\n\t"                  // 0: the exact path is needed
      "add.u32 %2, mant, e;\n\t"
      "min.u32 %3, %11, nv;\n\t"
      "}"
      : "=&r"(r0), "=&r"(r1), "=&r"(b), "=&r"(qo)
      : "r"(y0), "r"(y1), "n"(kMpX0), "n"(kMpX1), "l"(kMpX), "n"(kM0), "n"(kM1), "r"(qmin));
  y = ((uint64_t)r1 << 32) | r0;
  qmin = qo;
  return b;
}
static_assert((125u << 23) == 0x3E800000u && (0u - (1u << 23)) == 0xFF800000u,
              "exponent field of the backward FP32 step");

// The state advance of shared_step_f64 alone (raw-state output).
__device__ __forceinline__ uint64_t shared_advance(uint64_t z) {
  const uint32_t z0 = (uint32_t)z, z1 = (uint32_t)(z >> 32);
  const uint64_t t0 = (uint64_t)z0 * kK0;
  uint64_t t1 = (uint64_t)z0 * kK1 + (t0 >> 32);
  t1 = (uint64_t)z1 * kK0 + t1;
  const uint64_t t2 = (uint64_t)z1 * kK1 + (t1 >> 32);
  const uint32_t q0 = __funnelshift_r((uint32_t)t1, (uint32_t)t2, 21);
  const uint32_t q1 = __funnelshift_r((uint32_t)t2, (uint32_t)(t2 >> 32), 21);
  const uint64_t qm = (uint64_t)q0 * kM0;
  const uint32_t qm_hi = (uint32_t)(qm >> 32) + q0 * kM1 + q1 * kM0;
  uint64_t r = ((uint64_t)(z0 << 21) << 32) - (((uint64_t)qm_hi << 32) | (uint32_t)qm);
  if ((int64_t)r < 0) r += kM;
  return r;
}

// FP64-pipe conversion from a scaled chain value Z = z 2^10: exact
// int->double (Z has 53 significant bits), then one RN multiply by r3i 2^-10
// (no FMA): Z (r3i 2^-10) = z r3i, so the rounding is RN(z r3i) itself.  Both
// operations run on the FP64 pipe and none on the integer pipes, which is what
// a kernel bound by its integer work wants from it.
constexpr double kR3iScaled = kR3i * 0x1p-10;
__device__ __forceinline__ uint64_t f64_bits_fp64_scaled(uint64_t Z) {
  double v = __dmul_rn(__ull2double_rn(Z), kR3iScaled);
  return (uint64_t)__double_as_longlong(v);
}

// The same value from one fused multiply-add, for conversions made entirely
// on the FP64 pipe (where that pipe binds).  D = 2^52 + (z mod 2^52) is an
// exact double built from z's words (high word 0x43300000 | (z1 & 0xFFFFF)):
// it equals 2^52 + z below 2^52 and z itself from 2^52 up.  With off =
// -2^52*r3i in the first case (exact: r3i scaled by a power of two) and 0 in
// the second, D*r3i + off = z*r3i exactly, and the FMA rounds that once:
// RN(z * r3i), with half the FP64-pipe work of the form above.
constexpr double kR3iTimes2p52 = kR3i * 4503599627370496.0;  // 2^52 * r3i
__device__ __forceinline__ uint64_t f64_bits_fp64_fma(uint64_t z) {
  const uint32_t z1 = (uint32_t)(z >> 32);
  const double d = __hiloint2double((int)(0x43300000u | (z1 & 0xFFFFFu)), (int)(uint32_t)z);
  const double off = z1 >= 0x100000u ? 0.0 : -kR3iTimes2p52;
  return (uint64_t)__double_as_longlong(__fma_rn(d, kR3i, off));
}

// FP32 variate: the FP64 variate truncated toward zero.  Every variate is
// at least 2^-53, a normal float, so this is a shift and a re-bias of the
// exponent (1023 - 127 = 896).
__device__ __forceinline__ uint32_t f32_bits_from_f64_bits(uint64_t b) {
  return (uint32_t)((b >> 29) - (896ULL << 23));
}
#endif  // __CUDACC__

}  // namespace bcn
