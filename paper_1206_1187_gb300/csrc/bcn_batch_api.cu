// bcn_batch_api.cu -- host side of the batched kernel (bcn_batch.cu): batch
// plans (work table, graph replay), the allocation-free batch call and the
// tile-jump constants.
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "bcn_batch.cuh"
#include "bcn_host.h"
#include "bcn_math.cuh"

struct bcn_batch {
  uint32_t nstreams;
  uint64_t total_units;
  uint64_t total_elems;
  uint64_t total_bytes;
  rng_tune tune;       // resolved (depth 0: the built-in per-type depths)
  void* dev;           // descriptors | prefix | counter (one allocation)
  size_t dev_bytes;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int device;
};

namespace bcn {

// The work table lists the streams longest first (ties by stream number), so
// that the units taken last from the device counter are the short streams' (a
// long stream's units are then spread over the whole grid instead of ending
// the launch on a few warps).  The output does not depend on the order.  An
// in-place sort: the allocation-free entry point uses it too.
static void longest_first(uint32_t* order, uint32_t nstreams, const uint64_t* counts) {
  std::sort(order, order + nstreams, [counts](uint32_t x, uint32_t y) {
    return counts[x] != counts[y] ? counts[x] > counts[y] : x < y;
  });
}

// The tile-jump multipliers of every element type; with two chains, FP32
// runs the backward step when the step is the shared one with the integer
// conversion, or makes each run from one product (batch_f32_digits), whose
// state, one past the run, moves 32c elements to the lane's next run.  One
// chain per lane only occurs with one depth for every type.
void batch_fill_jumps(BatchParams& p, int step, int conv, int chains, const uint32_t d[3]) {
  const uint64_t stride = (step == ST_MONT) ? 33ull : 31ull;
  p.jump = host_pow2((53ull * stride * d[DT_F64]) % kP);
  p.jump_q = host_mulmod_quotient(p.jump);
  const bool digits = batch_f32_digits(step, conv, chains, d);
  for (int dt = 0; dt < 3; ++dt) {
    const bool back = dt == DT_F32 && step == ST_SHARED && conv == CV_INT;
    p.ja[dt] = host_pow2((53ull * (dt == DT_F32 && digits ? 32ull * d[dt]
                                                         : chain_jump_a(back, d[dt]))) % kP);
    p.jaq[dt] = host_mulmod_quotient(p.ja[dt]);
    p.jb[dt] = host_pow2((53ull * chain_jump_b(back, d[dt])) % kP);
    p.jbq[dt] = host_mulmod_quotient(p.jb[dt]);
    p.depth[dt] = d[dt];
  }
  p.warp_bytes = batch_warp_bytes(d);
}

static rng_status batch_launch_raw(bcn_batch* b, cudaStream_t cs) {
  uint32_t dd[3];
  batch_depths(b->tune, dd);
  const void* fn = batch_kernel_fn((int)b->tune.step, (int)b->tune.conv, (int)b->tune.chains, dd);
  if (!fn) return set_error(RNG_EINVAL, "no batch kernel for this step/conversion");
  unsigned char* base = static_cast<unsigned char*>(b->dev);
  BatchParams p;
  p.desc = reinterpret_cast<const BatchDesc*>(base);
  p.prefix = reinterpret_cast<const uint64_t*>(base + sizeof(BatchDesc) * b->nstreams);
  p.counter = reinterpret_cast<unsigned long long*>(base + sizeof(BatchDesc) * b->nstreams +
                                                    sizeof(uint64_t) * (b->nstreams + 1));
  p.total_units = b->total_units;
  batch_fill_jumps(p, (int)b->tune.step, (int)b->tune.conv, (int)b->tune.chains, dd);
  p.nstreams = b->nstreams;
  p.unit_tiles = b->tune.unit;
  p.skip = b->tune.skip;
  p.nbuf = b->tune.buffers;
  cudaError_t e = cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), cs);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(batch counter)");
  const size_t smem = batch_smem_bytes(b->tune.block, dd, b->tune.buffers);
  void* args[] = {&p};
  e = cudaLaunchKernel(fn, dim3(b->tune.grid), dim3(b->tune.block), args, smem, cs);
  if (e != cudaSuccess) return cuda_error(e, "batch kernel launch");
  return RNG_OK;
}

}  // namespace bcn

using namespace bcn;

extern "C" {

rng_status rng_batch_create(uint32_t nstreams, const uint64_t* starts, const uint64_t* offsets,
                            const uint64_t* counts, const uint8_t* dtypes, void* const* outs,
                            const rng_tune* tune, bcn_batch** out) {
  if (!out) return set_error(RNG_EINVAL, "out is NULL");
  *out = nullptr;
  if (nstreams == 0 || !starts || !counts || !dtypes || !outs)
    return set_error(RNG_EINVAL, "nstreams > 0 and the starts/counts/dtypes/outs arrays are required");
  rng_tune t = {};
  if (tune) t = *tune;
  const rng_status env = env_tune_check();
  if (env != RNG_OK) return env;
  const rng_tune d = auto_defaults(RNG_F64);
  if (!t.step) t.step = d.step ? d.step : (uint32_t)ST_SHARED;
  if (!t.conv) t.conv = d.conv ? d.conv : (uint32_t)CV_INT;
  if (!t.skip) t.skip = SK_TABLE;
  // zero fields: the plan shape the autotuner picks on GB300 for the batched
  // workload (4096 streams of 10^3..10^7 variates); depth 0 stays for the
  // built-in per-type depths where the kernel has them
  if (!t.block) t.block = 896;
  if (!t.unit) t.unit = 64;  // tiles per work unit
  if (!t.buffers) t.buffers = 1;
  t.buffers = batch_buffers(t);
  t.layout = RNG_LAYOUT_TILED;
  t.chains = batch_chains(t);
  if (!t.depth && !batch_builtin_depths_ok(t)) t.depth = 31;
  if (t.step != ST_SHARED && t.step != ST_BARRETT && t.step != ST_MONT)
    return set_error(RNG_EINVAL, "tune.step %u is not a step variant", t.step);
  if (t.conv != CV_INT && t.conv != CV_FP64)
    return set_error(RNG_EINVAL, "tune.conv %u is not a conversion", t.conv);
  if (t.skip != SK_TABLE && t.skip != SK_SQMUL)
    return set_error(RNG_EINVAL, "tune.skip %u is not a skip-ahead method", t.skip);
  if ((t.depth && t.depth % 2 == 0) || t.depth > kMaxDepth)
    return set_error(RNG_EINVAL, "tune.depth %u must be odd and at most %u", t.depth, kMaxDepth);
  if (t.block % 32 != 0 || t.block == 0 || t.block > 1024)
    return set_error(RNG_EINVAL, "tune.block %u must be a multiple of 32, <= 1024", t.block);
  if (t.unit > 4096) return set_error(RNG_EINVAL, "tune.unit (tiles per work unit) > 4096");
  if (t.buffers > 2) return set_error(RNG_EINVAL, "tune.buffers %u must be 0, 1 or 2", t.buffers);
  DeviceInfo di;
  rng_status st = device_info(&di);
  if (st != RNG_OK) return st;
  uint32_t dd[3];
  batch_depths(t, dd);
  const size_t smem = batch_smem_bytes(t.block, dd, t.buffers);
  if (smem > di.smem_optin)
    return set_error(RNG_EINVAL, "tile buffers need %zu bytes of shared memory, %zu available",
                     smem, di.smem_optin);
  const void* fn = batch_kernel_fn((int)t.step, (int)t.conv, (int)t.chains, dd);
  if (!fn) return set_error(RNG_EINVAL, "no batch kernel for this step/conversion");
  cudaError_t e =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)di.smem_optin);
  if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(batch)");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)t.block, smem);
  if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(batch)");
  const uint64_t full = (uint64_t)std::max(per_sm, 1) * (uint64_t)di.sms;

  std::vector<BatchDesc> desc(nstreams);
  std::vector<uint64_t> prefix(nstreams + 1);
  std::vector<uint32_t> order(nstreams);
  for (uint32_t s = 0; s < nstreams; ++s) {
    const uint64_t seed = starts[s], off = offsets ? offsets[s] : 0, n = counts[s];
    if (seed < kSeedMin || seed > kSeedMax)
      return set_error(RNG_ERANGE, "stream %u: start index outside [3^33+100, 2^53]", s);
    if (dtypes[s] > RNG_U64) return set_error(RNG_EINVAL, "stream %u: bad dtype %u", s, dtypes[s]);
    if (n > RNG_MAX_N) return set_error(RNG_ERANGE, "stream %u: count exceeds RNG_MAX_N", s);
    if (n > UINT64_MAX - off) return set_error(RNG_ERANGE, "stream %u: offset + count overflows", s);
    const size_t esz = dtype_size(dtypes[s]);
    if (n > 0 && (!outs[s] || (uintptr_t)outs[s] % esz != 0))
      return set_error(RNG_EINVAL, "stream %u: output NULL or not aligned to %zu bytes", s, esz);
    order[s] = s;
  }
  longest_first(order.data(), nstreams, counts);
  uint64_t units = 0, elems = 0, bytes = 0;
  for (uint32_t k = 0; k < nstreams; ++k) {
    const uint32_t s = order[k];
    const uint64_t seed = starts[s], off = offsets ? offsets[s] : 0, n = counts[s];
    const size_t esz = dtype_size(dtypes[s]);
    BatchDesc& D = desc[k];
    D.ebase = host_exponent_base(seed, off);
    D.n = n;
    D.out = static_cast<unsigned char*>(outs[s]);
    D.dt = dtypes[s];
    D.head = n ? (uint32_t)head_elems(outs[s], esz, n) : 0;
    D.unit0 = units;
    prefix[k] = units;
    uint64_t nu = 0;
    const uint64_t unit_elems = batch_unit_elems(dd, t.unit, (int)D.dt);
    if (n > 0) nu = n > D.head ? (n - D.head + unit_elems - 1) / unit_elems : 1;
    units += nu;
    elems += n;
    bytes += n * esz;
  }
  prefix[nstreams] = units;

  bcn_batch* b = new (std::nothrow) bcn_batch;
  if (!b) return set_error(RNG_ENOMEM, "out of host memory");
  b->nstreams = nstreams;
  b->total_units = units;
  b->total_elems = elems;
  b->total_bytes = bytes;
  b->graph = nullptr;
  b->exec = nullptr;
  b->device = di.device;
  b->dev = nullptr;
  const size_t desc_bytes = sizeof(BatchDesc) * nstreams;
  const size_t prefix_bytes = sizeof(uint64_t) * (nstreams + 1);
  b->dev_bytes = desc_bytes + prefix_bytes + 16;
  e = dev_malloc(&b->dev, b->dev_bytes);
  if (e != cudaSuccess) {
    delete b;
    return cuda_error(e, "cudaMalloc(batch plan)");
  }
  unsigned char* base = static_cast<unsigned char*>(b->dev);
  e = cudaMemcpy(base, desc.data(), desc_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + desc_bytes, prefix.data(), prefix_bytes,
                                       cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(base + desc_bytes + prefix_bytes, 0, 16);
  if (e != cudaSuccess) {
    cudaFree(b->dev);
    delete b;
    return cuda_error(e, "uploading the batch plan");
  }
  if (!t.grid) {
    const uint64_t need = (units + t.block / 32 - 1) / (t.block / 32);
    t.grid = (uint32_t)std::max<uint64_t>(1, std::min(full, need));
  }
  b->tune = t;
  *out = b;
  return RNG_OK;
}

rng_status rng_batch_launch(bcn_batch* b, void* cuda_stream) {
  if (!b) return set_error(RNG_EINVAL, "batch is NULL");
  if (b->total_units == 0) return RNG_OK;
  return batch_launch_raw(b, static_cast<cudaStream_t>(cuda_stream));
}

rng_status rng_batch_graph_launch(bcn_batch* b, void* cuda_stream) {
  if (!b) return set_error(RNG_EINVAL, "batch is NULL");
  if (b->total_units == 0) return RNG_OK;
  cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
  if (!b->exec) {  // capture memset + kernel once, on a private stream
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamCreate(capture)");
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_error(e, "cudaStreamBeginCapture");
    }
    rng_status st = batch_launch_raw(b, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (st != RNG_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_error(e, "cudaGraphInstantiate");
    }
    b->graph = g;
    b->exec = x;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, cs);
  if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
  return RNG_OK;
}

rng_status rng_batch_info(const bcn_batch* b, uint64_t* total_elems, uint64_t* total_bytes,
                          uint64_t* units, rng_tune* resolved) {
  if (!b) return set_error(RNG_EINVAL, "batch is NULL");
  if (total_elems) *total_elems = b->total_elems;
  if (total_bytes) *total_bytes = b->total_bytes;
  if (units) *units = b->total_units;
  if (resolved) *resolved = b->tune;
  return RNG_OK;
}

rng_status rng_batch_destroy(bcn_batch* b) {
  if (!b) return RNG_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->dev) cudaFree(b->dev);
  delete b;
  return RNG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch generation that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running under a host framework
// whose caching allocator owns all device memory (a stray cudaMalloc there can
// fail or fragment its pool), latency-critical paths that must not take the
// device-wide synchronisation cudaMalloc/cudaFree may imply, and embedded or
// sandboxed hosts where device allocation is simply not permitted.  For them
// the work table of the batched kernel (one descriptor per stream, the prefix
// of work-unit counts and the work counter) lives in this file-scope device
// array instead of a plan's cudaMalloc'd table.  The array holds at most
// kNoallocMaxStreams streams (about 49 KB) and stays resident on every device
// that loads the library until the process exits.
namespace bcn {

constexpr uint32_t kNoallocMaxStreams = 1024;
constexpr size_t kNoallocDescBytes = sizeof(BatchDesc) * kNoallocMaxStreams;
constexpr size_t kNoallocPrefixBytes = sizeof(uint64_t) * (kNoallocMaxStreams + 1);
constexpr size_t kNoallocBytes = kNoallocDescBytes + kNoallocPrefixBytes + 16;
static_assert(kNoallocDescBytes % 16 == 0 && kNoallocPrefixBytes % 8 == 0, "layout");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kNoallocMaxDevices = 64;
constexpr int kNoallocMaxKernels = 32;  // more than the batched kernel's instantiations
static std::mutex g_noalloc_mu;
static void* g_noalloc_dev[kNoallocMaxDevices];  // device address of the array, per device
// per device, the kernels whose shared-memory limit has been raised (a fixed
// table: recording them allocates nothing either)
static const void* g_noalloc_ready[kNoallocMaxDevices][kNoallocMaxKernels];
// host staging for the table (static: building it allocates nothing either)
static BatchDesc g_noalloc_desc[kNoallocMaxStreams];
static uint64_t g_noalloc_prefix[kNoallocMaxStreams + 1];
static uint32_t g_noalloc_order[kNoallocMaxStreams];

}  // namespace bcn

extern "C" rng_status rng_batch_generate_noalloc(uint32_t nstreams, const uint64_t* starts,
                                                 const uint64_t* offsets, const uint64_t* counts,
                                                 const uint8_t* dtypes, void* const* outs,
                                                 const rng_tune* tune, void* cuda_stream) {
  if (nstreams == 0) return RNG_OK;
  if (nstreams > kNoallocMaxStreams)
    return set_error(RNG_ERANGE, "%u streams exceed the no-allocation limit of %u", nstreams,
                     kNoallocMaxStreams);
  if (!starts || !counts || !dtypes || !outs)
    return set_error(RNG_EINVAL, "the starts/counts/dtypes/outs arrays are required");
  rng_tune t = {};
  if (tune) t = *tune;
  const rng_status env = env_tune_check();
  if (env != RNG_OK) return env;
  const rng_tune d = auto_defaults(RNG_F64);
  if (!t.step) t.step = d.step ? d.step : (uint32_t)ST_SHARED;
  if (!t.conv) t.conv = d.conv ? d.conv : (uint32_t)CV_INT;
  if (!t.skip) t.skip = SK_TABLE;
  // zero fields: the same shape as a batch plan's
  if (!t.block) t.block = 896;
  if (!t.unit) t.unit = 64;
  if (!t.buffers) t.buffers = 1;
  t.buffers = batch_buffers(t);
  t.chains = batch_chains(t);
  if (!t.depth && !batch_builtin_depths_ok(t)) t.depth = 31;
  if (t.step != ST_SHARED && t.step != ST_BARRETT && t.step != ST_MONT)
    return set_error(RNG_EINVAL, "tune.step %u is not a step variant", t.step);
  if (t.conv != CV_INT && t.conv != CV_FP64)
    return set_error(RNG_EINVAL, "tune.conv %u is not a conversion", t.conv);
  if (t.skip != SK_TABLE && t.skip != SK_SQMUL)
    return set_error(RNG_EINVAL, "tune.skip %u is not a skip-ahead method", t.skip);
  if ((t.depth && t.depth % 2 == 0) || t.depth > kMaxDepth)
    return set_error(RNG_EINVAL, "tune.depth %u must be odd and at most %u", t.depth, kMaxDepth);
  if (t.block % 32 != 0 || t.block == 0 || t.block > 1024)
    return set_error(RNG_EINVAL, "tune.block %u must be a multiple of 32, <= 1024", t.block);
  if (t.unit > 4096) return set_error(RNG_EINVAL, "tune.unit (tiles per work unit) > 4096");
  if (t.buffers > 2) return set_error(RNG_EINVAL, "tune.buffers %u must be 0, 1 or 2", t.buffers);
  DeviceInfo di;
  rng_status st = device_info(&di);
  if (st != RNG_OK) return st;
  if (di.device < 0 || di.device >= kNoallocMaxDevices)
    return set_error(RNG_EINVAL, "device %d beyond the no-allocation device table", di.device);
  uint32_t dd[3];
  batch_depths(t, dd);
  const size_t smem = batch_smem_bytes(t.block, dd, t.buffers);
  if (smem > di.smem_optin)
    return set_error(RNG_EINVAL, "tile buffers need %zu bytes of shared memory, %zu available",
                     smem, di.smem_optin);
  const void* fn = batch_kernel_fn((int)t.step, (int)t.conv, (int)t.chains, dd);
  if (!fn) return set_error(RNG_EINVAL, "no batch kernel for this step/conversion");
  cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);

  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  // once per device, with that device current: the array's device address
  // (in host code its name is only a host-side stand-in)
  if (!g_noalloc_dev[di.device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-allocation table)");
    g_noalloc_dev[di.device] = ptr;
  }
  // once per device and kernel: the kernel's full shared-memory allowance
  {
    const void** ready = g_noalloc_ready[di.device];
    int k = 0;
    while (k < kNoallocMaxKernels && ready[k] && ready[k] != fn) ++k;
    if (k == kNoallocMaxKernels || ready[k] != fn) {
      cudaError_t e =
          cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)di.smem_optin);
      if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(batch)");
      if (k < kNoallocMaxKernels) ready[k] = fn;
    }
  }
  unsigned char* base = static_cast<unsigned char*>(g_noalloc_dev[di.device]);

  for (uint32_t s = 0; s < nstreams; ++s) {
    const uint64_t seed = starts[s], off = offsets ? offsets[s] : 0, n = counts[s];
    if (seed < kSeedMin || seed > kSeedMax)
      return set_error(RNG_ERANGE, "stream %u: start index outside [3^33+100, 2^53]", s);
    if (dtypes[s] > RNG_U64) return set_error(RNG_EINVAL, "stream %u: bad dtype %u", s, dtypes[s]);
    if (n > RNG_MAX_N) return set_error(RNG_ERANGE, "stream %u: count exceeds RNG_MAX_N", s);
    if (n > UINT64_MAX - off) return set_error(RNG_ERANGE, "stream %u: offset + count overflows", s);
    const size_t esz = dtype_size(dtypes[s]);
    if (n > 0 && (!outs[s] || (uintptr_t)outs[s] % esz != 0))
      return set_error(RNG_EINVAL, "stream %u: output NULL or not aligned to %zu bytes", s, esz);
    g_noalloc_order[s] = s;
  }
  longest_first(g_noalloc_order, nstreams, counts);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)t.block, smem);
  if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const uint64_t full = (uint64_t)std::max(per_sm, 1) * (uint64_t)di.sms;
  uint64_t units = 0;
  for (uint32_t k = 0; k < nstreams; ++k) {
    const uint32_t s = g_noalloc_order[k];
    const uint64_t seed = starts[s], off = offsets ? offsets[s] : 0, n = counts[s];
    const size_t esz = dtype_size(dtypes[s]);
    BatchDesc& D = g_noalloc_desc[k];
    D.ebase = host_exponent_base(seed, off);
    D.n = n;
    D.out = static_cast<unsigned char*>(outs[s]);
    D.dt = dtypes[s];
    D.head = n ? (uint32_t)head_elems(outs[s], esz, n) : 0;
    D.unit0 = units;
    g_noalloc_prefix[k] = units;
    const uint64_t unit_elems = batch_unit_elems(dd, t.unit, (int)D.dt);
    if (n > 0) units += n > D.head ? (n - D.head + unit_elems - 1) / unit_elems : 1;
  }
  g_noalloc_prefix[nstreams] = units;
  if (units == 0) return RNG_OK;

  // Copies from pageable host memory return once the data is staged, so the
  // static host table may be rewritten by the next call.
  e = cudaMemcpyAsync(base, g_noalloc_desc, sizeof(BatchDesc) * nstreams,
                      cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + kNoallocDescBytes, g_noalloc_prefix,
                        sizeof(uint64_t) * (nstreams + 1), cudaMemcpyHostToDevice, cs);
  unsigned long long* counter =
      reinterpret_cast<unsigned long long*>(base + kNoallocDescBytes + kNoallocPrefixBytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), cs);
  if (e != cudaSuccess) return cuda_error(e, "staging the no-allocation table");

  uint32_t grid = t.grid;
  if (!grid) {
    const uint64_t need = (units + t.block / 32 - 1) / (t.block / 32);
    grid = (uint32_t)std::max<uint64_t>(1, std::min(full, need));
  }
  BatchParams p;
  p.desc = reinterpret_cast<const BatchDesc*>(base);
  p.prefix = reinterpret_cast<const uint64_t*>(base + kNoallocDescBytes);
  p.counter = counter;
  p.total_units = units;
  batch_fill_jumps(p, (int)t.step, (int)t.conv, (int)t.chains, dd);
  p.nstreams = nstreams;
  p.unit_tiles = t.unit;
  p.skip = t.skip;
  p.nbuf = t.buffers;
  void* args[] = {&p};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(t.block), args, smem, cs);
  if (e != cudaSuccess) return cuda_error(e, "batch kernel launch (no-allocation)");
  return RNG_OK;
}
