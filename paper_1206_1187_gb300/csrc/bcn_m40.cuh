// bcn_m40.cuh -- the 3^40 kernels' parameter block and kernel selection,
// shared by the kernels (bcn_m40.cu) and their host-side launcher
// (bcn_m40_api.cu).
#pragma once
#include "bcn_internal.h"

namespace bcn {

struct M40Params {
  unsigned char* out;
  uint64_t n, head, ntiles, ebase;
  // tile-to-tile jumps of the backward chains, Montgomery form of 2^(53 j),
  // h = c/2, lead = 1 for variates (0 for states):
  uint64_t jump;    // one chain: j = 33c + lead (one-product FP32 runs: 32c)
  uint64_t jump_a;  // two chains: j = 32c + h + 1 + lead and
  uint64_t jump_b;  //             j = 33c - h - 1 + lead
  uint32_t depth, nbuf;
};

// Whether one-chain FP32 runs of this depth are made from one product each
// (the compiled depths; bcn_m40.cu).
__host__ __device__ constexpr bool digit_run40_depth(uint64_t c) { return c == 15 || c == 31 || c == 44; }

// The 3^40 kernel for an output type, layout, chains per lane and tile depth
// (nullptr if there is none).
const void* pick40(int dt, int layout, uint32_t chains, uint32_t depth);

}  // namespace bcn
