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
  uint64_t jump_q;       // floor(jump * 2^64 / m); one chain per lane
  // two chains per lane, by element type (DT_F64, DT_F32, DT_U64): the FP32
  // entries are the backward chains' jumps when FP32 runs the backward step,
  // and ja alone the 32c-element jump when its runs come from one product
  uint64_t ja[3], jaq[3], jb[3], jbq[3];
  uint32_t depth[3];     // tile depth by element type
  uint32_t warp_bytes;   // one tile buffer of a warp, the largest type's tile
  uint32_t nstreams;
  uint32_t unit_tiles;
  uint32_t skip;
  uint32_t nbuf;         // tile buffers per warp (1 or 2)
};

// The tile depths of a batch by element type.  A resolved tuning's depth of 0
// (the default with the shared step on two chains) means the built-in depths
// of each type's fastest runs: FP64 30 (two variates per shared-memory
// store), FP32 44 (four, each run from one product), raw states 31; any other
// depth is the same for every type.
constexpr uint32_t kBatchDepthF64 = 30, kBatchDepthF32 = 44, kBatchDepthU64 = 31;
inline void batch_depths(const rng_tune& t, uint32_t d[3]) {
  d[DT_F64] = t.depth ? t.depth : kBatchDepthF64;
  d[DT_F32] = t.depth ? t.depth : kBatchDepthF32;
  d[DT_U64] = t.depth ? t.depth : kBatchDepthU64;
}
// Bytes of one tile buffer of a warp: the largest of the three types' tiles.
inline uint32_t batch_warp_bytes(const uint32_t d[3]) {
  const uint32_t b64 = d[DT_F64] * 8, b32 = d[DT_F32] * 4, bu = d[DT_U64] * 8;
  return 32 * (b64 > b32 ? (b64 > bu ? b64 : bu) : (b32 > bu ? b32 : bu));
}
// Elements of one work unit of a stream of element type dt.
inline uint64_t batch_unit_elems(const uint32_t d[3], uint32_t unit_tiles, int dt) {
  return 32ull * d[dt] * unit_tiles;
}

// The batched kernel for a step variant, conversion, chains per lane and tile
// depths (nullptr if none).
const void* batch_kernel_fn(int step, int conv, int chains, const uint32_t d[3]);

// Chains per lane a batched launch uses for this tuning (2 only for the forward
// steps with depth >= 3 or the built-in depths; 0 in the tuning means 2 for the
// shared step).
inline uint32_t batch_chains(const rng_tune& t) {
  const bool forward = (t.step == ST_SHARED && t.conv != CV_FP64) || t.step == ST_BARRETT;
  const uint32_t want = t.chains ? t.chains : (t.step == ST_SHARED ? 2u : 1u);
  return (forward && want == 2 && (t.depth == 0 || t.depth >= 3)) ? 2u : 1u;
}
// Whether a tuning may keep depth 0 (the built-in per-type depths): the shared
// step with the integer conversion on two chains.
inline bool batch_builtin_depths_ok(const rng_tune& t) {
  return t.step == ST_SHARED && t.conv == CV_INT && t.chains == 2;
}

// Whether the batched kernel for this tuning makes its FP32 runs from one
// product each (bcn_digits.cuh): the shared step with the integer conversion
// on two chains at the built-in depths.  Its other types keep two chains.
inline bool batch_f32_digits(int step, int conv, int chains, const uint32_t d[3]) {
  return step == ST_SHARED && conv == CV_INT && chains == 2 && d[DT_F64] == kBatchDepthF64 &&
         d[DT_F32] == kBatchDepthF32;
}

// Fill the tile-jump multipliers (and their precomputed quotients) of p.
void batch_fill_jumps(BatchParams& p, int step, int conv, int chains, const uint32_t d[3]);
// Tile buffers per warp for this tuning: tune.buffers, 0 meaning 2.
inline uint32_t batch_buffers(const rng_tune& t) { return t.buffers ? t.buffers : 2u; }
inline size_t batch_smem_bytes(uint32_t block, const uint32_t d[3], uint32_t nbuf) {
  return (size_t)(block / 32) * nbuf * batch_warp_bytes(d);
}

}  // namespace bcn
