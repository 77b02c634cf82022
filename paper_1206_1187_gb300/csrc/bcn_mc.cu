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
//     is an integer below 2^157 and a lane's sum fits 192 bits;
//   * RN(X + Y) <= 1 exactly when X + Y <= 1 + 2^-53 (the tie rounds to the
//     even 1.0), i.e. when the two grid integers sum to at most 2^157 + 2^104.
// Integer sums do not depend on order, so the warp reduction and the final
// per-block rounding give the same bits for any launch shape.
#include "bcn_gen.cuh"

namespace bcn {

struct U192 {
  uint64_t w0, w1, w2;
};

__device__ __forceinline__ void add128(uint64_t& a0, uint64_t& a1, uint64_t b0, uint64_t b1) {
  const uint64_t s0 = a0 + b0;
  a1 = a1 + b1 + (s0 < b0 ? 1ull : 0ull);
  a0 = s0;
}

__device__ __forceinline__ void add192(U192& a, const U192& b) {
  const uint64_t s0 = a.w0 + b.w0;
  const uint64_t c0 = s0 < b.w0 ? 1ull : 0ull;
  const uint64_t t1 = a.w1 + b.w1;
  const uint64_t c1a = t1 < b.w1 ? 1ull : 0ull;
  const uint64_t s1 = t1 + c0;
  const uint64_t c1b = s1 < c0 ? 1ull : 0ull;
  a.w2 = a.w2 + b.w2 + c1a + c1b;
  a.w1 = s1;
  a.w0 = s0;
}

// m << k as a 192-bit value, for m < 2^64 and 0 <= k < 128.
__device__ __forceinline__ U192 shifted192(uint64_t m, uint32_t k) {
  const uint32_t b = k & 63u;
  const uint64_t lo = m << b;
  const uint64_t hi = b ? (m >> (64u - b)) : 0ull;
  const bool w1 = k >= 64u;
  return U192{w1 ? 0ull : lo, w1 ? lo : hi, w1 ? hi : 0ull};
}

// The exact grid images of one FP64 variate (bits of RN(z*r3i)):
//   v*2^105 as (s0, s1) and RN(v*v)*2^157 as sq.
__device__ __forceinline__ void variate_terms(uint64_t bits, uint64_t& s0, uint64_t& s1, U192& sq) {
  const uint32_t e = (uint32_t)(bits >> 52);               // biased exponent, >= 970
  const uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  const uint32_t k1 = e - 970u;                             // v*2^105 = mant << k1, k1 <= 52
  s0 = mant << k1;
  s1 = k1 ? (mant >> (64u - k1)) : 0ull;
  // RN(mant^2) to 53 significant bits, ties to even
  const uint64_t plo = mant * mant, phi = __umul64hi(mant, mant);  // mant^2 < 2^106
  const uint32_t top = (uint32_t)(phi >> 41) & 1u;          // bit 105
  const uint32_t sh = 52u + top;                            // dropped bits
  // m2 = mant^2 >> sh, rest = mant^2 mod 2^sh (sh is 52 or 53)
  const uint64_t m2 = (phi << (64u - sh)) | (plo >> sh);
  const uint64_t rest = plo & ((1ull << sh) - 1ull);
  const uint64_t half = 1ull << (sh - 1u);
  const uint64_t up = (rest > half) | ((rest == half) & (m2 & 1ull));
  // RN(v^2) = (m2 + up) * 2^(2(e-1075) + sh); on the 2^-157 grid the shift is
  // 2e - 1993 + sh, which is >= 0 for every variate.
  sq = shifted192(m2 + up, 2u * e + sh - 1993u);
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

struct McParams {
  uint64_t ebase;       // (a - 3^33) mod P
  uint64_t block0;      // global number of the first block
  uint64_t nblocks;
  uint64_t len;         // variates per block (even)
  unsigned long long* hits_total;
  uint64_t* hits;       // per block, nullable
  double* sum;
  double* sumsq;
  uint32_t skip;
};

__global__ void __launch_bounds__(256) mc_kernel(const McParams p) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t wpb = blockDim.x >> 5;
  const uint64_t b = (uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
  if (b >= p.nblocks) return;
  const uint64_t pairs = p.len / 2;
  const uint64_t j0 = lane * pairs / 32, j1 = (lane + 1) * pairs / 32;
  const uint64_t first = (p.block0 + b) * p.len + 2 * j0;
  uint32_t hits = 0;
  uint64_t a0 = 0, a1 = 0;
  U192 q = {0, 0, 0};
  if (j0 < j1) {
    uint64_t z = seed_state(exponent_add(p.ebase, first + 1), p.skip);
    for (uint64_t j = j0; j < j1; ++j) {
      const uint64_t bx = shared_step_f64(z);
      const uint64_t by = shared_step_f64(z);
      uint64_t x0, x1, y0, y1;
      U192 xx, yy;
      variate_terms(bx, x0, x1, xx);
      variate_terms(by, y0, y1, yy);
      add128(a0, a1, x0, x1);
      add128(a0, a1, y0, y1);
      U192 r2 = xx;
      add192(r2, yy);
      // r2 <= 2^157 + 2^104 : word 2 holds bit 157 as bit 29, word 1 bit 104 as bit 40
      const bool inside = (r2.w2 < (1ull << 29)) ||
                          (r2.w2 == (1ull << 29) &&
                           (r2.w1 < (1ull << 40) || (r2.w1 == (1ull << 40) && r2.w0 == 0)));
      hits += inside ? 1u : 0u;
      add192(q, xx);
      add192(q, yy);
    }
  }
  // exact warp reduction (integer addition is order-free)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    hits += __shfl_xor_sync(0xffffffffu, hits, off);
    const uint64_t o0 = __shfl_xor_sync(0xffffffffu, a0, off);
    const uint64_t o1 = __shfl_xor_sync(0xffffffffu, a1, off);
    add128(a0, a1, o0, o1);
    U192 o;
    o.w0 = __shfl_xor_sync(0xffffffffu, q.w0, off);
    o.w1 = __shfl_xor_sync(0xffffffffu, q.w1, off);
    o.w2 = __shfl_xor_sync(0xffffffffu, q.w2, off);
    add192(q, o);
  }
  if (lane == 0) {
    p.sum[b] = round_words(a0, a1, 0, 105);
    p.sumsq[b] = round_words(q.w0, q.w1, q.w2, 157);
    if (p.hits) p.hits[b] = hits;
    atomicAdd(p.hits_total, (unsigned long long)hits);
  }
}

}  // namespace bcn

using namespace bcn;

extern "C" {

rng_status rng_consume_mc(uint64_t start_index, uint64_t block0, uint64_t nblocks, uint64_t len,
                          uint64_t* hits_total, uint64_t* hits, double* sum, double* sumsq,
                          void* cuda_stream, const rng_tune* tune) {
  if (start_index < kSeedMin || start_index > kSeedMax)
    return set_error(RNG_ERANGE, "start index outside [3^33+100, 2^53]");
  if (len == 0 || len % 2 != 0) return set_error(RNG_EINVAL, "len must be even and > 0");
  if (len > RNG_MAX_N) return set_error(RNG_ERANGE, "len exceeds RNG_MAX_N");
  if (nblocks == 0) return RNG_OK;
  if (!hits_total || !sum || !sumsq) return set_error(RNG_EINVAL, "hits_total, sum and sumsq are required");
  if (((uintptr_t)hits_total | (uintptr_t)sum | (uintptr_t)sumsq | (uintptr_t)hits) % 8 != 0)
    return set_error(RNG_EINVAL, "outputs must be 8-byte aligned");
  if (block0 > UINT64_MAX / len - nblocks) return set_error(RNG_ERANGE, "block range overflows");
  if (len / 2 > 0xFFFFFFFFull) return set_error(RNG_ERANGE, "len too large for 32-bit hit counts");
  rng_tune t = {};
  if (tune) t = *tune;
  const uint32_t block = t.block ? t.block : 256;
  if (block % 32 != 0 || block > 256)
    return set_error(RNG_EINVAL, "tune.block %u must be a multiple of 32, <= 256", block);
  const uint32_t skip = t.skip ? t.skip : SK_TABLE;
  if (skip != SK_TABLE && skip != SK_SQMUL) return set_error(RNG_EINVAL, "bad tune.skip");
  cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
  McParams p;
  p.ebase = host_exponent_base(start_index, 0);
  p.block0 = block0;
  p.nblocks = nblocks;
  p.len = len;
  p.hits_total = reinterpret_cast<unsigned long long*>(hits_total);
  p.hits = hits;
  p.sum = sum;
  p.sumsq = sumsq;
  p.skip = skip;
  cudaError_t e = cudaMemsetAsync(hits_total, 0, sizeof(uint64_t), cs);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(hits_total)");
  const uint64_t wpb = block / 32;
  const uint64_t grid = (nblocks + wpb - 1) / wpb;
  if (grid > 0x7fffffffull) return set_error(RNG_ERANGE, "too many blocks for one launch");
  void* args[] = {&p};
  e = cudaLaunchKernel((const void*)mc_kernel, dim3((unsigned)grid), dim3(block), args, 0, cs);
  if (e != cudaSuccess) return cuda_error(e, "mc kernel launch");
  return RNG_OK;
}

}  // extern "C"
