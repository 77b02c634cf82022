// bcn_mc_api.cu -- host side of the fused Monte-Carlo consumer: argument
// checks and the launch.  The kernel is in bcn_mc.cu.
#include <cmath>

#include "bcn_math.cuh"
#include "bcn_mc.cuh"

using namespace bcn;

extern "C" {

rng_status rng_consume_mc(uint64_t start_index, uint64_t block0, uint64_t nblocks, uint64_t len,
                          uint64_t* hits_total, uint64_t* hits, double* sum, double* sumsq,
                          void* cuda_stream, const rng_tune* tune) {
  return rng_consume_mc_totals(start_index, block0, nblocks, len, hits_total, hits, sum, sumsq,
                               nullptr, cuda_stream, tune);
}

rng_status rng_consume_mc_totals(uint64_t start_index, uint64_t block0, uint64_t nblocks,
                                 uint64_t len, uint64_t* hits_total, uint64_t* hits, double* sum,
                                 double* sumsq, uint64_t* totals, void* cuda_stream,
                                 const rng_tune* tune) {
  if (start_index < kSeedMin || start_index > kSeedMax)
    return set_error(RNG_ERANGE, "start index outside [3^33+100, 2^53]");
  if (len == 0 || len % 2 != 0) return set_error(RNG_EINVAL, "len must be even and > 0");
  if (len > RNG_MAX_N) return set_error(RNG_ERANGE, "len exceeds RNG_MAX_N");
  if (nblocks == 0) return RNG_OK;
  if (!hits_total || !sum || !sumsq) return set_error(RNG_EINVAL, "hits_total, sum and sumsq are required");
  if (((uintptr_t)hits_total | (uintptr_t)sum | (uintptr_t)sumsq | (uintptr_t)hits |
       (uintptr_t)totals) % 8 != 0)
    return set_error(RNG_EINVAL, "outputs must be 8-byte aligned");
  if (nblocks > (1ull << 32) && totals)
    return set_error(RNG_ERANGE, "exact totals hold at most 2^32 blocks");
  if (nblocks > UINT64_MAX / len || block0 > UINT64_MAX / len - nblocks)
    return set_error(RNG_ERANGE, "block range overflows");
  if (len / 2 > 0xFFFFFFFFull) return set_error(RNG_ERANGE, "len too large for 32-bit hit counts");
  rng_tune t = {};
  if (tune) t = *tune;
  const uint32_t block = t.block ? t.block : 128;  // measured: 128 and 256 within 0.5%
  if (block % 32 != 0 || block > 256)
    return set_error(RNG_EINVAL, "tune.block %u must be a multiple of 32, <= 256", block);
  const uint32_t skip = t.skip ? t.skip : (uint32_t)SK_TABLE;
  if (skip != SK_TABLE && skip != SK_SQMUL) return set_error(RNG_EINVAL, "bad tune.skip");
  // tune.conv chooses where each RN(v*v) is formed: RNG_CONV_FP64 on the FP64
  // pipe, RNG_CONV_INT on the integer pipes (0: the default)
  const uint32_t conv = t.conv ? t.conv : kMcDefaultConv;
  if (conv != CV_INT && conv != CV_FP64) return set_error(RNG_EINVAL, "bad tune.conv");
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
  p.totals = reinterpret_cast<unsigned long long*>(totals);
  p.skip = skip;
  cudaError_t e = cudaMemsetAsync(hits_total, 0, sizeof(uint64_t), cs);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(hits_total)");
  if (totals) {
    e = cudaMemsetAsync(totals, 0, sizeof(uint64_t) * RNG_MC_TOTAL_WORDS, cs);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(totals)");
  }
  const uint64_t wpb = block / 32;
  const uint64_t grid = (nblocks + wpb - 1) / wpb;
  if (grid > 0x7fffffffull) return set_error(RNG_ERANGE, "too many blocks for one launch");
  void* args[] = {&p};
  const void* fn = mc_kernel_fn(conv == CV_FP64);
  e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(block), args, 0, cs);
  if (e != cudaSuccess) return cuda_error(e, "mc kernel launch");
  return RNG_OK;
}

static_assert(kMcSumWords + kMcSqWords == RNG_MC_TOTAL_WORDS, "totals layout");

// Round sum_k words[k] * 2^(32k) * 2^-scale to the nearest double, ties to
// even: the words are first carried into 64-bit limbs (6 limbs hold any
// value the word arrays can reach), then the top 53 bits are kept and the
// rest decides the rounding.
static double round_pieces(const uint64_t* words, uint32_t nwords, int scale) {
  uint64_t limb[6] = {0, 0, 0, 0, 0, 0};
  for (uint32_t k = 0; k < nwords; ++k) {  // add words[k] << 32k
    const uint32_t q = (32 * k) / 64, r = (32 * k) % 64;
    unsigned __int128 carry = r ? (unsigned __int128)words[k] << r : words[k];
    for (uint32_t j = q; j < 6 && carry; ++j) {
      const unsigned __int128 t = (unsigned __int128)limb[j] + (uint64_t)carry;
      limb[j] = (uint64_t)t;
      carry = (carry >> 64) + (t >> 64);
    }
  }
  int top = -1;
  for (int j = 5; j >= 0 && top < 0; --j)
    if (limb[j]) top = 64 * j + 63 - __builtin_clzll(limb[j]);
  if (top < 0) return 0.0;
  auto bit = [&](int i) -> uint64_t { return (limb[i >> 6] >> (i & 63)) & 1ull; };
  if (top <= 52) return std::ldexp((double)limb[0], -scale);  // exact
  const int low = top - 52;  // lowest kept bit
  uint64_t mant = 0;
  for (int i = top; i >= low; --i) mant = (mant << 1) | bit(i);
  const uint64_t guard = bit(low - 1);
  bool sticky = false;
  for (int i = low - 2; i >= 0 && !sticky; --i) sticky = bit(i) != 0;
  if (guard && (sticky || (mant & 1ull))) mant += 1;  // a carry to 2^53 stays exact
  return std::ldexp((double)mant, low - scale);
}

rng_status rng_mc_round_totals(const uint64_t* totals, double* sum, double* sumsq) {
  if (!totals || !sum || !sumsq) return set_error(RNG_EINVAL, "NULL argument");
  *sum = round_pieces(totals, kMcSumWords, 105);
  *sumsq = round_pieces(totals + kMcSumWords, kMcSqWords, 157);
  return RNG_OK;
}

}  // extern "C"
