// bcn_tune.cu -- the measured choice of launch parameters.
//
// rng_autotune_bulk times candidate tunings of a bulk call with CUDA events
// and reports the fastest; rng_set_auto_tune installs a tuning as the
// library's default for the fields a caller leaves at zero.  The paper picks
// its threads per block by running every candidate 100 times and keeping the
// best (Sec. 3.2); this is the same procedure over this kernel's parameters
// (reduction, conversion, tile depth, block, grid).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "bcn_host.h"
#include "bcn_math.cuh"

namespace bcn {

static std::mutex g_auto_mu;
static rng_tune g_auto[3] = {};  // per rng_dtype; zero fields = built-in choice

// "key=value,key=value" into *out (fields not named stay 0).  On failure
// returns false with the reason in err.
static bool parse_tune(const char* text, rng_tune* out, char* err, size_t errlen) {
  static const char* const kSteps[] = {"", "barrett", "montgomery", "shared", "lecuyer",
                                       "barrett_classic"};
  static const char* const kConvs[] = {"", "int", "fp64"};
  static const char* const kLayouts[] = {"", "tiled", "direct", "strided"};
  static const char* const kSkips[] = {"", "table", "sqmul"};
  typedef uint32_t rng_tune::*Member;
  struct Field {
    const char* key;
    Member member;
    const char* const* names;
    int nnames;
  };
  static const Field kFields[] = {
      {"step", &rng_tune::step, kSteps, 6},       {"conv", &rng_tune::conv, kConvs, 3},
      {"layout", &rng_tune::layout, kLayouts, 4}, {"skip", &rng_tune::skip, kSkips, 3},
      {"depth", &rng_tune::depth, nullptr, 0},    {"block", &rng_tune::block, nullptr, 0},
      {"grid", &rng_tune::grid, nullptr, 0},      {"unit", &rng_tune::unit, nullptr, 0},
      {"chains", &rng_tune::chains, nullptr, 0},  {"buffers", &rng_tune::buffers, nullptr, 0},
  };
  rng_tune t = {};
  const char* p = text;
  while (*p) {
    while (*p == ' ' || *p == '\t' || *p == ',') ++p;
    if (!*p) break;
    const char* k0 = p;
    while (*p && *p != '=' && *p != ',' && *p != ' ' && *p != '\t') ++p;
    const size_t klen = (size_t)(p - k0);
    while (*p == ' ' || *p == '\t') ++p;
    if (*p != '=') {
      snprintf(err, errlen, "expected key=value at '%.*s'", (int)klen, k0);
      return false;
    }
    ++p;
    while (*p == ' ' || *p == '\t') ++p;
    const char* v0 = p;
    while (*p && *p != ',' && *p != ' ' && *p != '\t') ++p;
    const size_t vlen = (size_t)(p - v0);
    const Field* f = nullptr;
    for (const Field& c : kFields)
      if (strlen(c.key) == klen && strncmp(c.key, k0, klen) == 0) f = &c;
    if (!f) {
      snprintf(err, errlen, "unknown key '%.*s'", (int)klen, k0);
      return false;
    }
    bool ok = false;
    uint32_t value = 0;
    for (int i = 1; i < f->nnames && !ok; ++i)
      if (strlen(f->names[i]) == vlen && strncmp(f->names[i], v0, vlen) == 0) {
        value = (uint32_t)i;
        ok = true;
      }
    if (!ok && vlen > 0 && vlen <= 10) {  // a decimal number
      uint64_t x = 0;
      ok = true;
      for (size_t i = 0; i < vlen; ++i) {
        if (v0[i] < '0' || v0[i] > '9') {
          ok = false;
          break;
        }
        x = x * 10 + (uint64_t)(v0[i] - '0');
      }
      if (ok && x > 0xFFFFFFFFull) ok = false;
      value = (uint32_t)x;
    }
    if (!ok) {
      snprintf(err, errlen, "bad value '%.*s' for %s", (int)vlen, v0, f->key);
      return false;
    }
    t.*(f->member) = value;
  }
  *out = t;
  return true;
}

// BCN_RNG_TUNE, read once: a tuning forced on every call of the 3^33
// generator (its grid ignored, as the grid follows n).
static std::once_flag g_env_once;
static bool g_env_set = false;
static rng_tune g_env = {};
static char g_env_err[160] = "";

static void load_env_tune() {
  const char* v = getenv("BCN_RNG_TUNE");
  if (!v) return;
  g_env_set = true;
  if (!parse_tune(v, &g_env, g_env_err, sizeof g_env_err) && !g_env_err[0])
    snprintf(g_env_err, sizeof g_env_err, "does not parse");
  g_env.grid = 0;
}

rng_tune auto_defaults(int dt) {
  std::call_once(g_env_once, load_env_tune);
  if (g_env_set && !g_env_err[0]) return g_env;
  std::lock_guard<std::mutex> lock(g_auto_mu);
  if (dt < 0 || dt > 2) return rng_tune{};
  return g_auto[dt];
}

bool env_tune_sets_block() {
  std::call_once(g_env_once, load_env_tune);
  return g_env_set && !g_env_err[0] && g_env.block != 0;
}

rng_status env_tune_check() {
  std::call_once(g_env_once, load_env_tune);
  if (g_env_set && g_env_err[0]) return set_error(RNG_EINVAL, "BCN_RNG_TUNE: %s", g_env_err);
  return RNG_OK;
}

}  // namespace bcn

using namespace bcn;

extern "C" {

rng_status rng_parse_tune(const char* text, rng_tune* out) {
  if (!text || !out) return set_error(RNG_EINVAL, "NULL argument");
  char err[160];
  if (!parse_tune(text, out, err, sizeof err)) return set_error(RNG_EINVAL, "%s", err);
  return RNG_OK;
}

rng_status rng_set_auto_tune(rng_dtype dt, const rng_tune* t) {
  if ((int)dt < 0 || (int)dt > 2) return set_error(RNG_EINVAL, "dtype %d", (int)dt);
  if (t && t->layout == RNG_LAYOUT_STRIDED)
    return set_error(RNG_EINVAL, "the strided layout permutes the output and cannot be a default");
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
