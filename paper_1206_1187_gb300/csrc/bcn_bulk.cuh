// bcn_bulk.cuh -- the single-stream kernels' parameter blocks and kernel
// selection, shared by the kernels (bcn_bulk.cu) and their host-side
// launcher (bcn_bulk_api.cu).
#pragma once
#include "bcn_internal.h"

namespace bcn {

struct TiledParams {
  unsigned char* out;  // element 0 of the call
  uint64_t n;          // elements in the call
  uint64_t head;       // elements before the first 16-byte boundary
  uint64_t ntiles;     // full tiles of 32*depth elements after the head
  uint64_t ebase;      // (seed - 3^33 + 53*i0) mod P
  uint64_t jump;       // 2^(53*31*depth) (Barrett) / 2^(53*33*depth) (Montgomery)
  uint64_t jump_q;     // floor(jump * 2^64 / m), for the precomputed-quotient product
  uint64_t jump_a;     // two chains: 2^(53*(32c-h-1)) and 2^(53*(31c+h+1)), h = depth/2
  uint64_t jump_aq;
  uint64_t jump_b;
  uint64_t jump_bq;
  uint64_t cbits;      // ST_CONST: the word written
  uint32_t depth;
  uint32_t skip;
  uint32_t nbuf;       // tile buffers per warp (1 or 2)
};

struct DirectParams {
  unsigned char* out;
  uint64_t n;
  uint64_t ebase;
  uint64_t cbits;
  uint32_t skip;
};

// Whether one-chain FP32 runs of this depth are made from one product each
// (bcn_digits.cuh; the depths with a compiled kernel).
constexpr bool digit_run_depth(uint64_t c) { return c == 44; }

// The kernel for a layout, output type, step variant, conversion, chains per
// lane and tile depth (nullptr if there is none).
const void* pick_kernel(int layout, int dt, int st, int cv, int ilp, uint32_t depth);

}  // namespace bcn
