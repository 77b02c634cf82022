/*
 * bcn_oracle.c -- CPU oracle for the Bailey-Borwein alpha_{2,3} generator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline / reference legs may load it.  It
 * shares no code, header, table or constant generator with the CUDA library
 * under paper_1206_1187_gb300/csrc, and it never includes anything from there.
 *
 * What it follows (Beliakov et al., "Parallel random variates generator for
 * GPUs based on normal numbers"):
 *   - Algorithm BB, step 1: the seed is a start index a in [3^33+100, 2^53].
 *   - Eq. 2: z_0 = 2^(a - 3^33) * floor(3^33 / 2)  mod 3^33.
 *   - Eq. 3: z_k = 2^53 * z_(k-1)  mod 3^33, and the variate is z_k * 3^-33.
 *   - Sec. 1 (parallel split): the block of the sequence that starts at
 *     variate j is generated from the seed index a + 53*j, since each step of
 *     Eq. 3 advances the binary expansion of alpha_{2,3} by 53 digits.
 *   - Fig. 4 prints the reciprocal used for the output multiply:
 *     r3i = 1.0/5559060566555523.0.
 *
 * Arithmetic: every modular product is formed exactly in unsigned __int128
 * and reduced with the % operator -- the definition, not a fast reduction.
 * Exponents are 128-bit so that no reduction by the period is assumed.
 *
 * Readings of points the paper leaves open (each is a convention the GPU side
 * must match, and is checked by the tests against the mathematics):
 *   - The first variate of a block is z_1 (step, then emit), as in every code
 *     fragment of Sec. 2, so variate i of a stream with seed a is
 *     z = 2^(a - 3^33 + 53*(i+1)) * floor(3^33/2) mod 3^33.
 *   - The FP64 variate is one round-to-nearest multiply (double)z * r3i, with
 *     no fused multiply-add (this file is compiled with -ffp-contract=off).
 *   - The FP32 variate is the FP64 variate rounded toward zero to float, which
 *     keeps every FP32 variate inside the open interval (0,1).
 *   - The Monte-Carlo consumer pairs variates (2j, 2j+1) of a block; a pair
 *     hits when x*x + y*y <= 1.0 evaluated in FP64 with each operation rounded
 *     to nearest (no FMA).  Per-block sum and sum of squares are the exactly
 *     rounded (round-to-nearest-even) values of the exact sums of v and of
 *     RN(v*v), so they do not depend on summation order.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORACLE_M 5559060566555523ULL   /* 3^33, the modulus of Eq. 3        */
#define ORACLE_H 2779530283277761ULL   /* floor(3^33 / 2), the factor of Eq. 2 */
#define ORACLE_SEED_MIN (ORACLE_M + 100ULL)        /* Algorithm BB, step 1 */
#define ORACLE_SEED_MAX 9007199254740992ULL        /* 2^53, Algorithm BB   */

static const double ORACLE_R3I = 1.0 / 5559060566555523.0; /* Fig. 4 */

/* x*y mod 3^33 for x, y < 2^64: exact 128-bit product, then %. */
static uint64_t mulmod(uint64_t x, uint64_t y) {
  return (uint64_t)(((u128)x * (u128)y) % (u128)ORACLE_M);
}

/* 2^e mod 3^33 by right-to-left binary square-and-multiply. */
static uint64_t pow2mod(u128 e) {
  uint64_t result = 1, base = 2;
  while (e != 0) {
    if (e & 1) result = mulmod(result, base);
    base = mulmod(base, base);
    e >>= 1;
  }
  return result;
}

/* Eq. 2 for the seed index a + 53*j (the block that starts at variate j).
 * Returns 0 for a seed outside Algorithm BB's range (0 is never a state). */
uint64_t oracle_seed_state(uint64_t a, uint64_t j) {
  if (a < ORACLE_SEED_MIN || a > ORACLE_SEED_MAX) return 0;
  u128 e = (u128)(a - ORACLE_M) + (u128)53 * (u128)j;
  return mulmod(pow2mod(e), ORACLE_H);
}

/* Eq. 3 applied once: 2^53 * z mod 3^33. */
uint64_t oracle_step(uint64_t z) {
  return (uint64_t)(((u128)z << 53) % (u128)ORACLE_M);
}

/* The FP64 variate of a state: one round-to-nearest multiply by r3i. */
double oracle_to_f64(uint64_t z) {
  double zd = (double)z; /* exact: z < 2^53 */
  return zd * ORACLE_R3I;
}

/* The FP32 variate: the FP64 variate rounded toward zero. */
float oracle_to_f32(uint64_t z) {
  double v = oracle_to_f64(z);
  float f = (float)v;
  if ((double)f > v) f = nextafterf(f, 0.0f);
  return f;
}

/* States z of variates j .. j+n-1 of the stream with seed a (Eq. 2, Eq. 3). */
int oracle_states(uint64_t a, uint64_t j, uint64_t n, uint64_t *out) {
  uint64_t z = oracle_seed_state(a, j);
  if (z == 0) return -1;
  for (uint64_t k = 0; k < n; ++k) {
    z = oracle_step(z);
    out[k] = z;
  }
  return 0;
}

int oracle_f64(uint64_t a, uint64_t j, uint64_t n, double *out) {
  uint64_t z = oracle_seed_state(a, j);
  if (z == 0) return -1;
  for (uint64_t k = 0; k < n; ++k) {
    z = oracle_step(z);
    out[k] = oracle_to_f64(z);
  }
  return 0;
}

int oracle_f32(uint64_t a, uint64_t j, uint64_t n, float *out) {
  uint64_t z = oracle_seed_state(a, j);
  if (z == 0) return -1;
  for (uint64_t k = 0; k < n; ++k) {
    z = oracle_step(z);
    out[k] = oracle_to_f32(z);
  }
  return 0;
}

/* Variates at arbitrary positions, each straight from Eq. 2 (skip-ahead to
 * the position, then one step of Eq. 3).  dtype 0 = f64, 1 = f32, 2 = state. */
int oracle_at(uint64_t a, const uint64_t *idx, uint64_t n, int dtype, void *out) {
  for (uint64_t k = 0; k < n; ++k) {
    uint64_t z0 = oracle_seed_state(a, idx[k]);
    if (z0 == 0) return -1;
    uint64_t z = oracle_step(z0);
    if (dtype == 0) ((double *)out)[k] = oracle_to_f64(z);
    else if (dtype == 1) ((float *)out)[k] = oracle_to_f32(z);
    else ((uint64_t *)out)[k] = z;
  }
  return 0;
}

/* ---- exact summation: a 256-bit fixed-point accumulator on the 2^-160 grid.
 * Every FP64 variate is a multiple of 2^-105 and every RN(v*v) of one is a
 * multiple of 2^-157, so both sums are exact here. */
typedef struct { uint64_t w[4]; } acc256;
#define ACC_FRAC_BITS 160

static int acc_add(acc256 *acc, double d) {
  if (d == 0.0) return 0;
  if (!(d > 0.0)) return -1;
  int e2;
  double fr = frexp(d, &e2);                   /* d = fr * 2^e2, fr in [0.5,1) */
  uint64_t mant = (uint64_t)ldexp(fr, 53);      /* exact 53-bit integer      */
  int shift = e2 - 53 + ACC_FRAC_BITS;          /* d = mant * 2^(shift-160)  */
  while (shift < 0 && (mant & 1) == 0) {        /* drop trailing zero bits   */
    mant >>= 1;
    shift += 1;
  }
  if (shift < 0 || shift > 256 - 53) return -1; /* off the grid: not expected */
  /* the addend mant << shift, written out as four 64-bit limbs */
  uint64_t add[4] = {0, 0, 0, 0};
  int limb = shift / 64, bit = shift % 64;
  add[limb] = mant << bit;
  if (bit != 0 && limb + 1 < 4) add[limb + 1] = mant >> (64 - bit);
  uint64_t carry = 0;
  for (int i = 0; i < 4; ++i) {
    u128 s = (u128)acc->w[i] + add[i] + carry;
    acc->w[i] = (uint64_t)s;
    carry = (uint64_t)(s >> 64);
  }
  return carry ? -1 : 0;
}

/* bit k of the 256-bit accumulator */
static int acc_bit(const acc256 *acc, int k) {
  return (int)((acc->w[k / 64] >> (k % 64)) & 1ULL);
}

/* The accumulated value * 2^-160 rounded to nearest, ties to even. */
static double acc_round(const acc256 *acc) {
  int top = -1;
  for (int k = 255; k >= 0; --k)
    if (acc_bit(acc, k)) { top = k; break; }
  if (top < 0) return 0.0;
  if (top <= 52) return ldexp((double)acc->w[0], -ACC_FRAC_BITS); /* exact */
  int low = top - 52;                 /* lowest bit kept in the mantissa */
  uint64_t mant = 0;
  for (int k = top; k >= low; --k) mant = (mant << 1) | (uint64_t)acc_bit(acc, k);
  int guard = acc_bit(acc, low - 1);
  int sticky = 0;
  for (int k = low - 2; k >= 0; --k)
    if (acc_bit(acc, k)) { sticky = 1; break; }
  if (guard && (sticky || (mant & 1))) mant += 1; /* may become 2^53: exact */
  return ldexp((double)mant, low - ACC_FRAC_BITS);
}

/* Monte-Carlo consumer over blocks of `len` variates (len even) of the stream
 * with seed a.  Block b covers variates [b*len, (b+1)*len). */
int oracle_mc(uint64_t a, uint64_t len, const uint64_t *blocks, uint64_t nblocks,
              uint64_t *hits, double *sum, double *sumsq) {
  if (len % 2 != 0) return -1;
  for (uint64_t t = 0; t < nblocks; ++t) {
    uint64_t b = blocks[t];
    uint64_t z = oracle_seed_state(a, b * len);
    if (z == 0) return -1;
    acc256 s1, s2;
    memset(&s1, 0, sizeof s1);
    memset(&s2, 0, sizeof s2);
    uint64_t h = 0;
    for (uint64_t k = 0; k < len; k += 2) {
      z = oracle_step(z);
      double x = oracle_to_f64(z);
      z = oracle_step(z);
      double y = oracle_to_f64(z);
      double xx = x * x;
      double yy = y * y;
      double r2 = xx + yy;
      if (r2 <= 1.0) h += 1;
      if (acc_add(&s1, x) || acc_add(&s1, y)) return -1;
      if (acc_add(&s2, xx) || acc_add(&s2, yy)) return -1;
    }
    hits[t] = h;
    sum[t] = acc_round(&s1);
    sumsq[t] = acc_round(&s2);
  }
  return 0;
}

/* Exposed for the tests that pin the exact-rounding accumulator itself:
 * round(sum of ds[0..n)) with the accumulator above. */
int oracle_exact_sum(const double *ds, uint64_t n, double *out) {
  acc256 s;
  memset(&s, 0, sizeof s);
  for (uint64_t k = 0; k < n; ++k)
    if (acc_add(&s, ds[k])) return -1;
  *out = acc_round(&s);
  return 0;
}

/* ---- multi-threaded timing mode: the index range split by skip-ahead. ---- */
typedef struct {
  uint64_t a, j, n;
  int dtype;
  void *out;
  int rc;
} oracle_job;

static void *oracle_job_run(void *arg) {
  oracle_job *jb = (oracle_job *)arg;
  if (jb->dtype == 0) jb->rc = oracle_f64(jb->a, jb->j, jb->n, (double *)jb->out);
  else if (jb->dtype == 1) jb->rc = oracle_f32(jb->a, jb->j, jb->n, (float *)jb->out);
  else jb->rc = oracle_states(jb->a, jb->j, jb->n, (uint64_t *)jb->out);
  return NULL;
}

int oracle_generate_mt(uint64_t a, uint64_t j, uint64_t n, int dtype, void *out,
                       int nthreads) {
  if (nthreads < 1) nthreads = 1;
  size_t esz = dtype == 1 ? 4 : 8;
  oracle_job *jobs = (oracle_job *)calloc((size_t)nthreads, sizeof(oracle_job));
  pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !tids) { free(jobs); free(tids); return -1; }
  int rc = 0;
  for (int t = 0; t < nthreads; ++t) {
    uint64_t lo = (uint64_t)(((u128)n * (u128)t) / (u128)nthreads);
    uint64_t hi = (uint64_t)(((u128)n * (u128)(t + 1)) / (u128)nthreads);
    jobs[t].a = a;
    jobs[t].j = j + lo;
    jobs[t].n = hi - lo;
    jobs[t].dtype = dtype;
    jobs[t].out = (char *)out + lo * esz;
    pthread_create(&tids[t], NULL, oracle_job_run, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(tids[t], NULL);
    if (jobs[t].rc) rc = jobs[t].rc;
  }
  free(jobs);
  free(tids);
  return rc;
}

/* ==================================================================
 * The larger-modulus variant.  Sec. 1 notes that a modulus as large as 3^40
 * lengthens the period, at the price of 128-bit integer arithmetic; the
 * paper gives no further detail.  Readings taken here:
 *   - Eq. 2 and Eq. 3 with 3^40 in place of 3^33:
 *       z_0 = 2^(a - 3^40) * floor(3^40 / 2)  mod 3^40,
 *       z_k = 2^53 * z_(k-1)  mod 3^40,
 *     with the same "step, then emit" order, so variate i of seed a has the
 *     state 2^(a - 3^40 + 53*(i+1)) * floor(3^40/2) mod 3^40.
 *   - Seeds a in [3^40 + 100, 2^64 - 1]: the binary digits of alpha_{2,3}
 *     at positions n in [3^40+100, 3^41-100] come from the mod-3^40 LCG, and
 *     the seed is a 64-bit integer (2^64 - 1 < 3^41 - 100).
 *   - The period is 2*3^39 (2 is a primitive root modulo every power of 3).
 *   - The FP64 variate is the exact quotient z / 3^40 rounded toward zero:
 *     its 53 significant binary digits, from the first nonzero one, are
 *     consecutive binary digits of alpha_{2,3} (Sec. 1: the variates carry
 *     53-bit segments of alpha's expansion).  States reach 2^64, so (double)z
 *     is no longer exact and the multiply-by-reciprocal form of Fig. 4 would
 *     round twice; rounding to nearest instead would return 1.0 for the
 *     states above 3^40 (1 - 2^-54) and leave the open interval (0,1) of
 *     Algorithm BB.  It is formed here by binary long division.
 *   - The FP32 variate is the FP64 variate rounded toward zero, as for 3^33
 *     (equal to z / 3^40 rounded toward zero to float).
 * ================================================================== */
#define ORACLE40_M 12157665459056928801ULL   /* 3^40 */
#define ORACLE40_H 6078832729528464400ULL    /* floor(3^40 / 2) */
#define ORACLE40_SEED_MIN (ORACLE40_M + 100ULL)

/* x*y mod 3^40 for x, y < 2^64: exact 128-bit product, then %. */
static uint64_t mulmod40(uint64_t x, uint64_t y) {
  return (uint64_t)(((u128)x * (u128)y) % (u128)ORACLE40_M);
}

static uint64_t pow2mod40(u128 e) {
  uint64_t result = 1, base = 2;
  while (e != 0) {
    if (e & 1) result = mulmod40(result, base);
    base = mulmod40(base, base);
    e >>= 1;
  }
  return result;
}

/* Eq. 2 (modulus 3^40) for the seed index a + 53*j; 0 for a seed below
 * 3^40 + 100. */
uint64_t oracle40_seed_state(uint64_t a, uint64_t j) {
  if (a < ORACLE40_SEED_MIN) return 0;
  u128 e = (u128)(a - ORACLE40_M) + (u128)53 * (u128)j;
  return mulmod40(pow2mod40(e), ORACLE40_H);
}

/* Eq. 3 (modulus 3^40) once: 2^53 z mod 3^40 (z < 2^64, so z*2^53 < 2^117). */
uint64_t oracle40_step(uint64_t z) {
  return (uint64_t)(((u128)z << 53) % (u128)ORACLE40_M);
}

/* z / 3^40 rounded toward zero, for a state z in [1, 3^40 - 1], by binary
 * long division: each step doubles the remainder and takes out 3^40 when it
 * fits, which yields the next binary digit of z / 3^40.  The 53 digits from
 * the leading one are the significand.  Returns -1.0 for a value that is not
 * a state. */
double oracle40_to_f64(uint64_t z) {
  if (z == 0 || z >= ORACLE40_M) return -1.0;
  u128 r = z;
  int k = 0, lead = 0, nbits = 0;
  uint64_t mant = 0;
  while (nbits < 53) {
    r <<= 1;
    ++k;
    int bit = r >= (u128)ORACLE40_M;
    if (bit) r -= ORACLE40_M;
    if (nbits == 0 && !bit) continue;  /* leading zero digits */
    if (nbits == 0) lead = k;          /* the leading one has value 2^-lead */
    mant = (mant << 1) | (uint64_t)bit;
    ++nbits;
  }
  /* mant's digits have values 2^-lead .. 2^-(lead+52); the rest is dropped */
  return ldexp((double)mant, -(lead + 52));
}

float oracle40_to_f32(uint64_t z) {
  double v = oracle40_to_f64(z);
  float f = (float)v;
  if ((double)f > v) f = nextafterf(f, 0.0f);
  return f;
}

/* Variates j .. j+n-1 of seed a under the 3^40 modulus, in order.
 * dtype 0 = f64, 1 = f32, 2 = state. */
int oracle40_generate(uint64_t a, uint64_t j, uint64_t n, int dtype, void *out) {
  uint64_t z = oracle40_seed_state(a, j);
  if (z == 0 || dtype < 0 || dtype > 2) return -1;
  for (uint64_t k = 0; k < n; ++k) {
    z = oracle40_step(z);
    if (dtype == 0) ((double *)out)[k] = oracle40_to_f64(z);
    else if (dtype == 1) ((float *)out)[k] = oracle40_to_f32(z);
    else ((uint64_t *)out)[k] = z;
  }
  return 0;
}

/* Variates at arbitrary positions, each straight from Eq. 2 (modulus 3^40). */
int oracle40_at(uint64_t a, const uint64_t *idx, uint64_t n, int dtype, void *out) {
  if (dtype < 0 || dtype > 2) return -1;
  for (uint64_t k = 0; k < n; ++k) {
    uint64_t z0 = oracle40_seed_state(a, idx[k]);
    if (z0 == 0) return -1;
    uint64_t z = oracle40_step(z0);
    if (dtype == 0) ((double *)out)[k] = oracle40_to_f64(z);
    else if (dtype == 1) ((float *)out)[k] = oracle40_to_f32(z);
    else ((uint64_t *)out)[k] = z;
  }
  return 0;
}
