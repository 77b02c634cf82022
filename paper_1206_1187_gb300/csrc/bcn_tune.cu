// bcn_tune.cu -- the measured choice of launch parameters.
//
// rng_autotune_bulk times candidate tunings of a bulk call with CUDA events
// and reports the fastest; rng_set_auto_tune installs a tuning as the
// library's default for the fields a caller leaves at zero.  The paper picks
// its threads per block by running every candidate 100 times and keeping the
// best (Sec. 3.2); this is the same procedure over this kernel's parameters
// (reduction, conversion, tile depth, block, grid).
#include <mutex>

#include "bcn_internal.h"
#include "bcn_math.cuh"

namespace bcn {

static std::mutex g_auto_mu;
static rng_tune g_auto[3] = {};  // per rng_dtype; zero fields = built-in choice

rng_tune auto_defaults(int dt) {
  std::lock_guard<std::mutex> lock(g_auto_mu);
  if (dt < 0 || dt > 2) return rng_tune{};
  return g_auto[dt];
}

}  // namespace bcn

using namespace bcn;

extern "C" {

rng_status rng_set_auto_tune(rng_dtype dt, const rng_tune* t) {
  if ((int)dt < 0 || (int)dt > 2) return set_error(RNG_EINVAL, "dtype %d", (int)dt);
  std::lock_guard<std::mutex> lock(g_auto_mu);
  if (t) {
    g_auto[dt] = *t;
    g_auto[dt].grid = 0;  // the grid follows n; never pin it globally
  } else {
    g_auto[dt] = rng_tune{};
  }
  return RNG_OK;
}

rng_status rng_autotune_bulk(uint64_t n, rng_dtype dt, void* out, void* cuda_stream,
                             const rng_tune* candidates, uint32_t ncand, uint32_t reps,
                             rng_tune* best, float* ms_out) {
  if (!candidates || ncand == 0 || !best)
    return set_error(RNG_EINVAL, "candidates and best are required");
  if (n == 0 || n > RNG_MAX_N) return set_error(RNG_ERANGE, "n out of range");
  if (!out || (uintptr_t)out % dtype_size(dt) != 0)
    return set_error(RNG_EINVAL, "output pointer NULL or misaligned");
  if (reps == 0) reps = 1;
  cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_error(e, "cudaEventCreate");
  }
  rng_status result = RNG_OK;
  float best_ms = -1.0f;
  for (uint32_t i = 0; i < ncand; ++i) {
    if (ms_out) ms_out[i] = -1.0f;
    BulkLaunch L;
    if (resolve_bulk(n, (int)dt, &candidates[i], &L, false) != RNG_OK) continue;  // invalid
    rng_status st = launch_bulk(L, kSeedMin, 0, n, out, 0, cs);  // warm-up
    if (st != RNG_OK) {
      result = st;
      break;
    }
    cudaEventRecord(e0, cs);
    for (uint32_t r = 0; r < reps && st == RNG_OK; ++r)
      st = launch_bulk(L, kSeedMin, (uint64_t)r * n, n, out, 0, cs);
    cudaEventRecord(e1, cs);
    e = cudaEventSynchronize(e1);
    if (st != RNG_OK) {
      result = st;
      break;
    }
    if (e != cudaSuccess) {
      result = cuda_error(e, "autotune timing");
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    if (ms_out) ms_out[i] = ms;
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best->step = (uint32_t)L.step;
      best->conv = (uint32_t)L.conv;
      best->layout = (uint32_t)L.layout;
      best->skip = (uint32_t)L.skip;
      best->depth = L.depth;
      best->block = L.block;
      best->grid = L.grid;
      best->unit = 0;
      best->chains = L.chains;
      best->buffers = L.buffers;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result == RNG_OK && best_ms < 0.0f)
    result = set_error(RNG_EINVAL, "no valid candidate");
  return result;
}

}  // extern "C"
