// bcn_mc.cuh -- the fused consumer kernel's parameter block and kernel
// selection, shared by the kernel (bcn_mc.cu) and its host-side launcher
// (bcn_mc_api.cu).
#pragma once
#include "bcn_internal.h"

namespace bcn {

// Where the squares run when tune.conv is 0 (measured on GB300).
constexpr uint32_t kMcDefaultConv = CV_FP64;

struct McParams {
  uint64_t ebase;       // (a - 3^33) mod P
  uint64_t block0;      // global number of the first block
  uint64_t nblocks;
  uint64_t len;         // variates per block (even)
  unsigned long long* hits_total;
  uint64_t* hits;       // per block, nullable
  double* sum;
  double* sumsq;
  unsigned long long* totals;  // nullable: the call's exact totals, in 32-bit pieces
  uint32_t skip;
};

// Words of the exact totals: 5 pieces of the sum on the 2^-105 grid (below
// 2^138 per block), then 6 of the sum of squares on the 2^-157 grid (below
// 2^190 per block).
constexpr uint32_t kMcSumWords = 5, kMcSqWords = 6;

// The fused kernel forming each RN(v*v) on the FP64 pipe (true) or on the
// integer pipes (false).
const void* mc_kernel_fn(bool fp64_squares);

}  // namespace bcn
