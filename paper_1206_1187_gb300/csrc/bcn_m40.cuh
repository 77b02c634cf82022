// bcn_m40.cuh -- the 3^40 kernels' parameter block and kernel selection,
// shared by the kernels (bcn_m40.cu) and their host-side launcher
// (bcn_m40_api.cu).
#pragma once
#include "bcn_internal.h"

namespace bcn {

struct M40Params {
  unsigned char* out;
  uint64_t n, head, ntiles, ebase;
  uint64_t jump;    // one chain: Montgomery form of 2^(53 (31c - ahead))
  uint64_t jump_a;  // two chains: 2^(53 (32c - h - 1 - ahead)) and
  uint64_t jump_b;  //             2^(53 (31c + h + 1 - ahead)), h = c/2
  uint32_t depth, nbuf;
};

// The 3^40 kernel for an output type, layout, chains per lane and tile depth
// (nullptr if there is none).
const void* pick40(int dt, int layout, uint32_t chains, uint32_t depth);

}  // namespace bcn
