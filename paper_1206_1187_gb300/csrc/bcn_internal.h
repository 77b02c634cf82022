// bcn_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "bcn_rng.h"

namespace bcn {

// Output element kinds used as template arguments.
enum { DT_F64 = 0, DT_F32 = 1, DT_U64 = 2 };
// State advance: Modified Barrett (forward), Montgomery (backward), Barrett
// with the quotient shared with the conversion (forward), or the roofline
// probe that writes a constant and computes nothing.
enum { ST_BARRETT = 1, ST_MONT = 2, ST_SHARED = 3, ST_LECUYER = 4, ST_BCLASSIC = 5,
       ST_CONST = 9 };
enum { CV_INT = 1, CV_FP64 = 2 };
enum { SK_TABLE = 1, SK_SQMUL = 2 };

constexpr uint32_t kMaxDepth = 255;

// A fully resolved bulk launch.
struct BulkLaunch {
  int dt, step, conv, layout, skip;
  uint32_t depth, block, grid, chains, buffers;
  size_t smem_bytes;  // TILED only
};

// Where a lane's run of c elements is split between its two chains: chain a
// takes elements [0, s), chain b [s, c).  Odd c: s = c/2 + 1.  The backward
// FP32 runs also take c = 4 mod 8, stored four variates at a time, where s
// is the larger half in whole groups of four (c = 44: s = 24); the forward
// FP64 runs c = 2 mod 4, stored two variates at a time, where s is the larger
// half in whole pairs (c = 30: s = 16).
__host__ __device__ constexpr uint32_t chain_split(uint64_t c) {
  return (uint32_t)(c % 2 ? c / 2 + 1
                          : c % 4 == 2 ? 2 * ((c / 2 + 1) / 2) : 4 * ((c / 4 + 1) / 2));
}
// Whether a backward FP32 run of this depth takes the four-variate stores.
__host__ __device__ constexpr bool vec4_depth(uint64_t c) { return c % 8 == 4; }
// Whether a forward FP64 run of this depth takes the two-variate stores.
__host__ __device__ constexpr bool vec2_depth(uint64_t c) { return c % 4 == 2; }

// The tile-to-tile jumps (in steps) of a lane's two chains over tiles of
// 32*c elements (s = chain_split(c)): forward chains move from elements s and
// c of the lane's run to elements 0 and s of its run in the next tile,
// backward ones (the FP32 step that runs Eq. 3 backwards) from elements 0 and
// s to s and c.
inline uint64_t chain_jump_a(bool backward, uint64_t c) {
  return backward ? 32 * c + chain_split(c) : 32 * c - chain_split(c);
}
inline uint64_t chain_jump_b(bool backward, uint64_t c) {
  return backward ? 33 * c - chain_split(c) : 31 * c + chain_split(c);
}

// Element size in bytes of an rng_dtype.
inline size_t dtype_size(int dt) { return dt == DT_F32 ? 4 : 8; }

// Elements before the first 16-byte boundary of `out` (at most n).
inline uint64_t head_elems(const void* out, size_t esz, uint64_t n) {
  const uintptr_t addr = (uintptr_t)out;
  const uint64_t h = ((16 - (addr & 15)) & 15) / esz;
  return h < n ? h : n;
}

// Set the calling thread's error message and return `st`.
rng_status set_error(rng_status st, const char* fmt, ...);
rng_status cuda_error(cudaError_t e, const char* what);

// Device properties cached per device.
struct DeviceInfo {
  int device;
  int sms;
  size_t smem_optin;  // max dynamic shared memory per block
};
rng_status device_info(DeviceInfo* out);

// Allow a kernel the device's full opt-in dynamic shared memory (once per
// kernel and device).
rng_status enable_smem(const void* fn, int device, size_t bytes);

// The tuning installed by rng_set_auto_tune for dtype dt (zeros if none), or
// the one BCN_RNG_TUNE forces for every dtype when that variable is set.
rng_tune auto_defaults(int dt);

// Fill in every zero field of `tune` for a bulk call of n elements of dt.
rng_status resolve_bulk(uint64_t n, int dt, const rng_tune* tune, BulkLaunch* out,
                        bool constant);

// Launch a bulk generation (or constant fill) of elements [0, n) of the
// call, whose element 0 is variate number i0 of the stream seeded with
// `seed`.  `out` is aligned to the element size.
rng_status launch_bulk(const BulkLaunch& L, uint64_t seed, uint64_t i0, uint64_t n,
                       void* out, uint64_t const_bits, cudaStream_t cs);

}  // namespace bcn
