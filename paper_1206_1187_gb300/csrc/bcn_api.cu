// bcn_api.cu -- the C ABI of include/bcn_rng.h: streams, argument checks,
// error reporting and device properties.  All numerical work happens in the
// kernels; this file only validates, resolves launch shapes and launches.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "bcn_host.h"
#include "bcn_math.cuh"

struct bcn_stream {
  uint64_t seed;
  uint64_t count;
  cudaStream_t cs;
  // staging for rng_generate_to_host, created on first use
  int staging_device = -1;
  uint32_t nstage = 0;
  size_t stage_bytes = 0;
  void* stage[8] = {};
  cudaStream_t stage_cs[8] = {};
};

namespace bcn {

static thread_local char g_err[512];

rng_status set_error(rng_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

rng_status cuda_error(cudaError_t e, const char* what) {
  return set_error(RNG_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e),
                   cudaGetErrorString(e));
}

rng_status device_info(DeviceInfo* out) {
  static std::mutex mu;
  static std::vector<DeviceInfo> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(mu);
  for (const DeviceInfo& d : cache)
    if (d.device == dev) {
      *out = d;
      return RNG_OK;
    }
  DeviceInfo d = {};
  d.device = dev;
  e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute(SM count)");
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute(shared memory)");
  d.smem_optin = (size_t)optin;
  cache.push_back(d);
  *out = d;
  return RNG_OK;
}

// Allocation failures injected by rng_debug_fail_allocations: after
// g_fail_skip more allocations succeed, the next g_fail_count fail.
static std::mutex g_fail_mu;
static uint64_t g_fail_skip = 0, g_fail_count = 0;

static bool injected_failure() {
  std::lock_guard<std::mutex> lock(g_fail_mu);
  if (g_fail_count == 0) return false;
  if (g_fail_skip > 0) {
    --g_fail_skip;
    return false;
  }
  --g_fail_count;
  return true;
}

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t pinned_malloc(void** p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}

static bool seed_ok(uint64_t seed) { return seed >= kSeedMin && seed <= kSeedMax; }

// Shared checks of a bulk call; returns RNG_OK when there is work to launch
// and sets *empty when n == 0.
static rng_status check_bulk(uint64_t seed, uint64_t n, int dt, const void* out,
                             bool* empty) {
  *empty = false;
  if (!seed_ok(seed))
    return set_error(RNG_ERANGE, "start index %llu outside [3^33+100, 2^53]",
                     (unsigned long long)seed);
  if (dt != RNG_F64 && dt != RNG_F32 && dt != RNG_U64)
    return set_error(RNG_EINVAL, "dtype %d is not an rng_dtype", dt);
  if (n == 0) {
    *empty = true;
    return RNG_OK;
  }
  if (n > RNG_MAX_N)
    return set_error(RNG_ERANGE, "n = %llu exceeds RNG_MAX_N", (unsigned long long)n);
  if (out == nullptr) return set_error(RNG_EINVAL, "output pointer is NULL");
  if ((uintptr_t)out % dtype_size(dt) != 0)
    return set_error(RNG_EINVAL, "output pointer is not aligned to its %zu-byte elements",
                     dtype_size(dt));
  return RNG_OK;
}

static rng_status generate_impl(uint64_t seed, uint64_t i0, uint64_t n, int dt, void* out,
                                cudaStream_t cs, const rng_tune* tune) {
  bool empty = false;
  rng_status st = check_bulk(seed, n, dt, out, &empty);
  if (st != RNG_OK || empty) return st;
  BulkLaunch L;
  st = resolve_bulk(n, dt, tune, &L, false);
  if (st != RNG_OK) return st;
  return launch_bulk(L, seed, i0, n, out, 0, cs);
}

}  // namespace bcn

using namespace bcn;

extern "C" {

rng_status rng_create(uint64_t start_index, bcn_stream** out) {
  if (!out) return set_error(RNG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!seed_ok(start_index))
    return set_error(RNG_ERANGE, "start index %llu outside [3^33+100, 2^53]",
                     (unsigned long long)start_index);
  bcn_stream* s = new (std::nothrow) bcn_stream;
  if (!s) return set_error(RNG_ENOMEM, "out of host memory");
  s->seed = start_index;
  s->count = 0;
  s->cs = nullptr;
  s->nstage = 0;
  *out = s;
  return RNG_OK;
}

static void release_staging(bcn_stream* s) {
  for (uint32_t i = 0; i < s->nstage; ++i) {
    if (s->stage_cs[i]) {
      cudaStreamSynchronize(s->stage_cs[i]);
      cudaStreamDestroy(s->stage_cs[i]);
    }
    if (s->stage[i]) cudaFree(s->stage[i]);
    s->stage[i] = nullptr;
    s->stage_cs[i] = nullptr;
  }
  s->nstage = 0;
  s->stage_bytes = 0;
  s->staging_device = -1;
}

rng_status rng_destroy(bcn_stream* s) {
  if (s) release_staging(s);
  delete s;
  return RNG_OK;
}

// rng_generate_to_host: the next n variates into host memory.  Chunks of the
// call are generated into `nbuf` rotating device staging buffers, each with
// its own CUDA stream, and copied to the host from there; the generation of one
// chunk overlaps the copies of the others.  Synchronous: returns when the data
// is in host memory.
rng_status rng_generate_to_host(bcn_stream* s, uint64_t n, rng_dtype dt, void* host_out,
                                uint64_t chunk_bytes, uint32_t nbuf) {
  if (!s) return set_error(RNG_EINVAL, "stream is NULL");
  bool empty = false;
  rng_status st = check_bulk(s->seed, n, (int)dt, host_out, &empty);
  if (st != RNG_OK || empty) return st;
  if (n > UINT64_MAX - s->count) return set_error(RNG_ERANGE, "count would pass 2^64-1");
  if (chunk_bytes > (1ull << 40)) return set_error(RNG_EINVAL, "chunk_bytes above 2^40");
  if (!chunk_bytes) chunk_bytes = 64ull << 20;
  if (!nbuf) nbuf = 4;
  if (nbuf > 8) return set_error(RNG_EINVAL, "at most 8 staging buffers");
  const size_t esz = dtype_size((int)dt);
  chunk_bytes = (chunk_bytes + 255) / 256 * 256;  // whole 256-byte blocks, >= 32 elements
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (s->nstage != nbuf || s->stage_bytes != chunk_bytes || s->staging_device != dev) {
    release_staging(s);
    for (uint32_t i = 0; i < nbuf; ++i) {
      e = dev_malloc(&s->stage[i], chunk_bytes);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stage_cs[i], cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        s->nstage = i + 1;
        release_staging(s);
        return cuda_error(e, "allocating host-transfer staging");
      }
    }
    s->nstage = nbuf;
    s->stage_bytes = chunk_bytes;
    s->staging_device = dev;
  }
  // work ordered after what the caller already queued on the stream's CUDA stream
  cudaEvent_t start = nullptr;
  e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(start, s->cs);
  for (uint32_t i = 0; i < nbuf && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(s->stage_cs[i], start, 0);
  if (start) cudaEventDestroy(start);
  if (e != cudaSuccess) return cuda_error(e, "ordering host transfer");
  const uint64_t per = chunk_bytes / esz;
  // on an error part way, the copies already queued still write into the
  // caller's buffer: wait for them before returning
  auto drain = [s, nbuf](rng_status r) {
    for (uint32_t i = 0; i < nbuf; ++i) cudaStreamSynchronize(s->stage_cs[i]);
    return r;
  };
  BulkLaunch L;
  bool resolved = false;
  uint64_t done = 0;
  for (uint64_t k = 0; done < n; ++k) {
    const uint64_t cnt = (n - done < per) ? n - done : per;
    const uint32_t b = (uint32_t)(k % nbuf);
    if (!resolved || cnt != per) {
      st = resolve_bulk(cnt, (int)dt, nullptr, &L, false);
      if (st != RNG_OK) return drain(st);
      resolved = cnt == per;
    }
    st = launch_bulk(L, s->seed, s->count + done, cnt, s->stage[b], 0, s->stage_cs[b]);
    if (st != RNG_OK) return drain(st);
    e = cudaMemcpyAsync(static_cast<unsigned char*>(host_out) + done * esz, s->stage[b],
                        cnt * esz, cudaMemcpyDeviceToHost, s->stage_cs[b]);
    if (e != cudaSuccess) return drain(cuda_error(e, "device-to-host copy"));
    done += cnt;
  }
  for (uint32_t i = 0; i < nbuf; ++i) {
    e = cudaStreamSynchronize(s->stage_cs[i]);
    if (e != cudaSuccess) return cuda_error(e, "host transfer");
  }
  s->count += n;
  return RNG_OK;
}

rng_status rng_set_cuda_stream(bcn_stream* s, void* cuda_stream) {
  if (!s) return set_error(RNG_EINVAL, "stream is NULL");
  s->cs = static_cast<cudaStream_t>(cuda_stream);
  return RNG_OK;
}

rng_status rng_generate_tuned(bcn_stream* s, uint64_t n, rng_dtype dt, void* out,
                              const rng_tune* tune) {
  if (!s) return set_error(RNG_EINVAL, "stream is NULL");
  if (n > UINT64_MAX - s->count)
    return set_error(RNG_ERANGE, "count would pass 2^64-1");
  rng_status st = generate_impl(s->seed, s->count, n, dt, out, s->cs, tune);
  if (st == RNG_OK) s->count += n;
  return st;
}

rng_status rng_generate(bcn_stream* s, uint64_t n, rng_dtype dt, void* out) {
  return rng_generate_tuned(s, n, dt, out, nullptr);
}

rng_status rng_skip(bcn_stream* s, uint64_t k) {
  if (!s) return set_error(RNG_EINVAL, "stream is NULL");
  if (k > UINT64_MAX - s->count) return set_error(RNG_ERANGE, "count would pass 2^64-1");
  s->count += k;
  return RNG_OK;
}

rng_status rng_get_state(const bcn_stream* s, uint64_t* start_index, uint64_t* count) {
  if (!s || !start_index || !count) return set_error(RNG_EINVAL, "NULL argument");
  *start_index = s->seed;
  *count = s->count;
  return RNG_OK;
}

rng_status rng_set_state(bcn_stream* s, uint64_t start_index, uint64_t count) {
  if (!s) return set_error(RNG_EINVAL, "stream is NULL");
  if (!seed_ok(start_index))
    return set_error(RNG_ERANGE, "start index %llu outside [3^33+100, 2^53]",
                     (unsigned long long)start_index);
  s->seed = start_index;
  s->count = count;
  return RNG_OK;
}

rng_status rng_sync(bcn_stream* s) {
  if (!s) return set_error(RNG_EINVAL, "stream is NULL");
  cudaError_t e = cudaStreamSynchronize(s->cs);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "asynchronous error");
  return RNG_OK;
}

rng_status rng_generate_at(uint64_t start_index, uint64_t offset, uint64_t n, rng_dtype dt,
                           void* out, void* cuda_stream, const rng_tune* tune) {
  return generate_impl(start_index, offset, n, dt, out, static_cast<cudaStream_t>(cuda_stream),
                       tune);
}

rng_status rng_fill_constant(uint64_t n, rng_dtype dt, double value, void* out,
                             void* cuda_stream, const rng_tune* tune) {
  bool empty = false;
  rng_status st = check_bulk(kSeedMin, n, dt, out, &empty);
  if (st != RNG_OK || empty) return st;
  if (dt == RNG_U64) return set_error(RNG_EINVAL, "the constant fill writes RNG_F64 or RNG_F32");
  uint64_t bits = 0;
  if (dt == RNG_F64) {
    std::memcpy(&bits, &value, 8);
  } else {
    float f = (float)value;
    uint32_t b32;
    std::memcpy(&b32, &f, 4);
    bits = b32;
  }
  BulkLaunch L;
  st = resolve_bulk(n, dt, tune, &L, true);
  if (st != RNG_OK) return st;
  return launch_bulk(L, kSeedMin, 0, n, out, bits, static_cast<cudaStream_t>(cuda_stream));
}

const char* rng_last_error(void) { return g_err; }

rng_status rng_debug_fail_allocations(uint32_t skip, uint32_t count) {
  std::lock_guard<std::mutex> lock(g_fail_mu);
  g_fail_skip = skip;
  g_fail_count = count;
  return RNG_OK;
}

rng_status rng_resolve_tune(uint64_t n, rng_dtype dt, const rng_tune* in, rng_tune* out) {
  if (!out) return set_error(RNG_EINVAL, "out is NULL");
  BulkLaunch L;
  rng_status st = resolve_bulk(n, dt, in, &L, false);
  if (st != RNG_OK) return st;
  out->step = (uint32_t)L.step;
  out->conv = (uint32_t)L.conv;
  out->layout = (uint32_t)L.layout;
  out->skip = (uint32_t)L.skip;
  out->depth = L.depth;
  out->block = L.block;
  out->grid = L.grid;
  const bool strided = L.layout == RNG_LAYOUT_STRIDED;
  out->unit = strided ? L.chains : 0;  // the strided layout's unroll factor
  out->chains = strided ? 0 : L.chains;
  out->buffers = L.buffers;
  return RNG_OK;
}

int rng_version(void) { return 103; }

}  // extern "C"
