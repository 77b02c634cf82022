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
  uint64_t jump_a, jump_aq, jump_b, jump_bq;  // two chains per lane
  uint64_t back_a, back_aq, back_b, back_bq;  // two backward FP32 chains per lane
  uint32_t nstreams;
  uint32_t depth;
  uint32_t unit_tiles;
  uint32_t skip;
  uint32_t nbuf;         // tile buffers per warp (1 or 2)
};

// The batched kernel for a step variant, conversion, chains per lane and tile
// depth (nullptr if none), and the dynamic shared memory one block needs.
const void* batch_kernel_fn(int step, int conv, int chains, uint32_t depth);

// Chains per lane a batched launch uses for this tuning (2 only for the forward
// steps with depth >= 3; 0 in the tuning means 2 for the shared step).
inline uint32_t batch_chains(const rng_tune& t) {
  const bool forward = (t.step == ST_SHARED && t.conv != CV_FP64) || t.step == ST_BARRETT;
  const uint32_t want = t.chains ? t.chains : (t.step == ST_SHARED ? 2u : 1u);
  return (forward && want == 2 && t.depth >= 3) ? 2u : 1u;
}

// Fill the tile-jump multipliers (and their precomputed quotients) of p.
void batch_fill_jumps(BatchParams& p, int step, uint32_t depth);
// Tile buffers per warp for this tuning: tune.buffers, 0 meaning 2.
inline uint32_t batch_buffers(const rng_tune& t) { return t.buffers ? t.buffers : 2u; }
inline size_t batch_smem_bytes(uint32_t block, uint32_t depth, uint32_t nbuf) {
  return (size_t)(block / 32) * nbuf * 32 * depth * 8;
}

}  // namespace bcn
