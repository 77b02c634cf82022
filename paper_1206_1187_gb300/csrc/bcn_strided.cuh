// bcn_strided.cuh -- the paper's coalesced (strided) layout: parameter block
// and kernel selection, shared by the kernels (bcn_strided.cu) and the bulk
// launcher (bcn_bulk_api.cu).
#pragma once
#include "bcn_internal.h"

namespace bcn {

struct StridedParams {
  unsigned char* out;  // position 0 of the call
  uint64_t nthreads;   // T: threads, one block of the sequence each
  uint64_t per;        // W: variates per thread (n = T * W)
  uint64_t ebase;      // (seed - 3^33 + 53*i0) mod P
  uint64_t cbits;      // ST_CONST: the word written
  uint32_t skip;
};

// The strided kernel for an output type, step variant, conversion and unroll
// factor (1 or 8); nullptr if there is none.
const void* pick_strided(int dt, int st, int cv, uint32_t unroll);

}  // namespace bcn
