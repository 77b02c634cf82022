// bcn_batch.cuh -- the work table of the batched kernel, shared by the batch
// plans, the allocation-free batch entry point and the serving loop.
#pragma once
#include "bcn_internal.h"

namespace bcn {

struct BatchDesc {
  uint64_t ebase;       // (seed - 3^33 + 53*offset) mod P
  uint64_t n;           // elements
  unsigned char* out;   // element 0
  uint64_t unit0;       // first unit number
  uint32_t dt;          // DT_F64 / DT_F32 / DT_U64
  uint32_t head;        // elements before the first 16-byte boundary
};

struct BatchParams {
  const BatchDesc* desc;
  const uint64_t* prefix;  // nstreams + 1 unit counts, prefix[s] = desc[s].unit0
  unsigned long long* counter;
  uint64_t total_units;
  uint64_t jump;
  uint64_t jump_q;       // floor(jump * 2^64 / m)
  uint32_t nstreams;
  uint32_t depth;
  uint32_t unit_tiles;
  uint32_t skip;
};

// The batched kernel for a step variant and conversion (nullptr if none), and
// the dynamic shared memory one block of it needs.
const void* batch_kernel_fn(int step, int conv);
inline size_t batch_smem_bytes(uint32_t block, uint32_t depth) {
  return (size_t)(block / 32) * 2 * 32 * depth * 8;
}

}  // namespace bcn
