// bcn_serve.cu -- a continuous-batching request server for variate requests.
//
// A request asks for n variates (offset .. offset+n-1 of the sequence seeded
// with a start index) as FP64, FP32 or raw states.  The server owns one device
// output pool.  A scheduler thread runs iterations:
//   1. retire the iterations whose completion event has fired: every request
//      whose last chunk rode on one is complete (its completion time is taken
//      then), and its pool range is freed `release_after` seconds later (or
//      when the caller releases it);
//   2. admit waiting requests in arrival order while a request slot is free
//      and the pool has a free range for the request's output (memory-based
//      admission).  A request that does not fit waits; a later one that does
//      fit may pass it while the waiting one is younger than the bypass age,
//      so one large request does not hold back every small one behind it.
//      Once the oldest waiting request reaches that age, nothing passes it
//      until it is admitted, so a large request is never starved.  With
//      caller-managed release (release_after_s < 0) the order is strict by
//      default: a client that consumes its results in order would otherwise
//      hold, unreleased, the ranges of the requests that passed the one it
//      waits for;
//   3. if an iteration slot is free, pack the next chunk (chunk_elems
//      variates, up to 64 times more when few requests are active) of every
//      active request, round-robin, into one work table and launch the
//      batched kernel on that slot's CUDA stream.
// With several slots, requests admitted while earlier iterations run are
// launched on another stream and overlap them on the device; chunking keeps a
// 256 MiB request from holding back the small ones.
//
// Two kernel shapes, chosen per iteration by its size when the tuning is left
// to the server: a light iteration runs short tiles in small blocks (the
// lowest latency for small requests), a heavy one -- enough work for two
// wide tiles per warp of the whole GPU -- deep tiles in 896-thread blocks with
// one buffer per warp (the highest throughput).  The bytes never depend on the
// shape.  Every chunk is a block of
// its request's sequence reached by skip-ahead (the paper's parallel split,
// Sec. 1), so a request's bytes never depend on what it was batched with.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bcn_batch.cuh"
#include "bcn_host.h"
#include "bcn_math.cuh"
#include "bcn_pool.h"

namespace bcn {

typedef std::chrono::steady_clock Clock;
static double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

enum { RQ_QUEUED = 0, RQ_ACTIVE = 1, RQ_DONE = 2, RQ_RELEASED = 3, RQ_CANCELLED = 4 };

// Where rng_server_run_trace collects its requests' latencies: the worker
// fills it in as requests complete (under the server's lock).
struct TraceSink {
  double* latency;    // one entry per request of the trace
  uint64_t pending;   // requests of the trace not yet complete
  double last_done;   // completion time of the latest one
};

struct Request {
  uint64_t seed = 0, offset = 0, n = 0, bytes = 0, pool_off = 0, scheduled = 0;
  uint32_t dt = 0;
  int state = RQ_QUEUED;
  double t_arrive = 0, t_admit = 0, t_done = 0;
  TraceSink* sink = nullptr;  // set while a running trace waits for this request
  uint32_t sink_idx = 0;
  uint32_t readers = 0;         // rng_server_read copies in progress
  bool release_pending = false; // release asked for while a copy was in progress
};

// What is kept of a request once its pool range is released (or once it is
// dropped from the queue after a cancel): its final state and times.  Only
// the most recent kPastRequests of them are kept, so a long-running server's
// bookkeeping stays bounded.
struct PastRequest {
  int state;
  double t_arrive, t_done;
};
constexpr size_t kPastRequests = 1u << 16;

// One launch shape of the batched kernel.
struct ServeShape {
  rng_tune tune;
  const void* fn = nullptr;
  size_t smem = 0;
  uint64_t grid_full = 0;
};

struct Slot {
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  BatchDesc* h_desc = nullptr;      // pinned staging of the work table
  uint64_t* h_prefix = nullptr;
  unsigned char* d_table = nullptr;  // device: descriptors | prefix | counter
  bool busy = false;
  std::vector<uint64_t> finishing;   // requests whose last chunk is in this iteration
};

}  // namespace bcn

struct bcn_server {
  rng_server_config cfg;
  bcn::ServeShape shape[2];   // [0] light iterations, [1] heavy ones
  uint32_t nshapes = 1;
  uint64_t heavy_elems = 0;   // an iteration of at least this many elements is heavy
  int device = 0;
  unsigned char* pool_dev = nullptr;
  bcn::Pool pool;
  std::mutex mu;
  std::condition_variable cv_work;   // wakes the scheduler
  std::condition_variable cv_done;   // wakes waiters
  std::unordered_map<uint64_t, bcn::Request> reqs;        // queued, active or done
  std::unordered_map<uint64_t, bcn::PastRequest> past;   // released or dropped
  std::deque<uint64_t> past_order;                       // ids in `past`, oldest first
  std::deque<uint64_t> queue;
  std::vector<uint64_t> active;
  std::deque<std::pair<double, uint64_t>> to_release;  // (time, id)
  std::vector<bcn::Slot> slots;
  std::thread worker;
  std::atomic<bool> stop{false};
  std::atomic<uint64_t> loop_gap_max_us{0};  // scheduler stall diagnostics
  std::atomic<uint64_t> launch_max_us{0};
  std::atomic<uint64_t> call_max_us[3] = {};  // staging copies, kernel launch, event record
  rng_status err = RNG_OK;
  char errmsg[256] = {0};
  uint64_t next_id = 1, rr = 0;
  double bypass_s = -1.0;     // admission bypass age (negative: strict arrival order)
  rng_server_stats st = {};
  uint64_t lat_hist[RNG_SERVER_HIST_BINS] = {};  // completion latencies, quarter octaves
  bcn_server(uint64_t cap) : pool(cap, 256) {}
};

namespace bcn {

static void server_fail(bcn_server* s, cudaError_t e, const char* what) {
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->err == RNG_OK) {
    s->err = RNG_ECUDA;
    snprintf(s->errmsg, sizeof s->errmsg, "%s: %s", what, cudaGetErrorString(e));
  }
  s->cv_done.notify_all();
}

// Move a released or cancelled request from the live table to the bounded
// history (mu held).
static void forget(bcn_server* s, std::unordered_map<uint64_t, Request>::iterator it) {
  const uint64_t id = it->first;
  s->past.emplace(id, PastRequest{it->second.state, it->second.t_arrive, it->second.t_done});
  s->reqs.erase(it);
  s->past_order.push_back(id);
  while (s->past_order.size() > kPastRequests) {
    s->past.erase(s->past_order.front());
    s->past_order.pop_front();
  }
}

// A request's state and times, live or past (mu held); false if unknown.
static bool lookup(const bcn_server* s, uint64_t id, int* state, double* t_arrive,
                   double* t_done) {
  auto it = s->reqs.find(id);
  if (it != s->reqs.end()) {
    *state = it->second.state;
    *t_arrive = it->second.t_arrive;
    *t_done = it->second.t_done;
    return true;
  }
  auto p = s->past.find(id);
  if (p == s->past.end()) return false;
  *state = p->second.state;
  *t_arrive = p->second.t_arrive;
  *t_done = p->second.t_done;
  return true;
}

// The latency histogram's bin: k with 2^(k/4) <= latency in us < 2^((k+1)/4),
// clamped to the first and last bins.
static uint32_t latency_bin(double seconds) {
  const double us = seconds * 1e6;
  if (!(us > 1.0)) return 0;
  const double k = std::floor(4.0 * std::log2(us));
  return k >= RNG_SERVER_HIST_BINS - 1 ? RNG_SERVER_HIST_BINS - 1 : (uint32_t)k;
}

// Retire finished iterations; returns true if any finished.
static bool retire(bcn_server* s) {
  bool any = false;
  for (Slot& sl : s->slots) {
    if (!sl.busy) continue;
    cudaError_t e = cudaEventQuery(sl.ev);
    if (e == cudaErrorNotReady) continue;
    if (e != cudaSuccess) {
      server_fail(s, e, "iteration");
      sl.busy = false;
      continue;
    }
    const double t = now_s();
    std::lock_guard<std::mutex> lock(s->mu);
    for (uint64_t id : sl.finishing) {
      Request& r = s->reqs.at(id);  // an active request is never forgotten
      r.state = RQ_DONE;
      r.t_done = t;
      s->st.completed += 1;
      s->st.bytes_done += r.bytes;
      s->lat_hist[latency_bin(t - r.t_arrive)] += 1;
      if (r.sink) {
        r.sink->latency[r.sink_idx] = t - r.t_arrive;
        r.sink->last_done = std::max(r.sink->last_done, t);
        r.sink->pending -= 1;
        r.sink = nullptr;
      }
      if (s->cfg.release_after_s >= 0) s->to_release.emplace_back(t + s->cfg.release_after_s, id);
    }
    sl.finishing.clear();
    sl.busy = false;
    any = true;
    s->cv_done.notify_all();
  }
  return any;
}

// Free a done request's pool range (mu held).  While rng_server_read is
// copying the range out, the free is deferred to the end of that copy, so a
// new request cannot be given the range (and overwrite it) mid-copy.
static void release_range(bcn_server* s, std::unordered_map<uint64_t, Request>::iterator it) {
  if (it->second.readers > 0) {
    it->second.release_pending = true;
    return;
  }
  s->pool.release(it->second.pool_off);
  it->second.state = RQ_RELEASED;
  forget(s, it);
  s->cv_work.notify_one();
}

// Free pool ranges whose hold time has passed (caller holds mu).
static void release_due(bcn_server* s, double t) {
  while (!s->to_release.empty() && s->to_release.front().first <= t) {
    const uint64_t id = s->to_release.front().second;
    s->to_release.pop_front();
    auto it = s->reqs.find(id);
    if (it != s->reqs.end() && it->second.state == RQ_DONE) release_range(s, it);
  }
}

// Queued requests looked at per admission pass when earlier ones do not fit.
constexpr size_t kAdmitScan = 256;
// How long a waiting request may be passed by later ones that fit, when the
// server frees results itself and the caller leaves admit_bypass_s at 0.
// Measured on the serving trace with results held 0.2 s (the pool binds):
// strict order and ages up to 0.2 s give p50 539 ms (under sustained
// overload the oldest request is soon older than the age and the order is
// strict again); 0.5 s and 1 s give p50 362 ms with the same throughput and
// p99 (1.1 s), 1 s the lower p90 (910 against 995 ms).
constexpr double kDefaultBypassS = 1.0;

// Admit queued requests in arrival order while slots and pool space allow
// (mu held).  A request that does not fit is passed over while it is younger
// than the bypass age (s->bypass_s; negative: never), and stops the pass once
// it is older.
static bool admit(bcn_server* s, double t) {
  bool any = false;
  size_t k = 0;
  while (k < s->queue.size() && k < kAdmitScan && s->active.size() < s->cfg.max_active) {
    const uint64_t id = s->queue[k];
    auto it = s->reqs.find(id);
    Request& r = it->second;
    if (r.state == RQ_CANCELLED) {
      s->queue.erase(s->queue.begin() + (std::ptrdiff_t)k);
      forget(s, it);
      continue;
    }
    uint64_t off = 0;
    if (!s->pool.alloc(r.bytes, &off)) {  // memory-based admission
      if (s->bypass_s < 0 || t - r.t_arrive >= s->bypass_s) break;
      ++k;  // later requests may pass this one, for now
      s->st.bypassed += k == 1 ? 1 : 0;
      continue;
    }
    r.pool_off = off;
    r.state = RQ_ACTIVE;
    r.t_admit = t;
    s->active.push_back(id);
    s->queue.erase(s->queue.begin() + (std::ptrdiff_t)k);
    if (k > 0) s->st.admitted_out_of_order += 1;
    any = true;
    if (s->pool.in_use > s->st.peak_pool_bytes) s->st.peak_pool_bytes = s->pool.in_use;
    if (s->active.size() > s->st.peak_active) s->st.peak_active = s->active.size();
  }
  return any;
}

// Pack the next chunk of every active request into slot `sl` (mu held).
// Returns the number of work items; *shape_out the kernel shape to launch.
static uint32_t pack(bcn_server* s, Slot& sl, uint64_t* units_out, uint32_t* shape_out) {
  const size_t na = s->active.size();
  // the piece of each request this iteration: chunk_elems when many requests
  // share it, up to 64 x chunk_elems when few do (a lone large request then
  // runs as one heavy launch instead of many light ones: nominal-trace p99
  // 0.44 -> 0.17 ms, measured against 16x and 128x), always a multiple of 4
  // elements so that every piece starts 16-byte aligned
  const uint64_t budget =
      s->cfg.chunk_elems > UINT64_MAX / 64 ? UINT64_MAX : 64 * s->cfg.chunk_elems;
  const uint64_t share = na ? budget / std::min<uint64_t>(na, s->cfg.max_items) : budget;
  const uint64_t piece = std::max<uint64_t>(s->cfg.chunk_elems, share / 4 * 4);
  uint32_t shape = 0;
  if (s->nshapes > 1) {  // the iteration's size decides the shape
    uint64_t total = 0;
    for (size_t k = 0; k < na && k < s->cfg.max_items; ++k) {
      const Request& r = s->reqs.at(s->active[(s->rr + k) % na]);
      total += std::min<uint64_t>(r.n - r.scheduled, piece);
    }
    if (total >= s->heavy_elems) shape = 1;
  }
  const rng_tune& tn = s->shape[shape].tune;
  uint32_t dd[3];
  batch_depths(tn, dd);
  uint32_t items = 0;
  uint64_t units = 0;
  std::vector<uint64_t> still;
  still.reserve(na);
  for (size_t k = 0; k < na; ++k) {
    const uint64_t id = s->active[(s->rr + k) % na];
    Request& r = s->reqs.at(id);
    if (items >= s->cfg.max_items) {
      still.push_back(id);
      continue;
    }
    const uint64_t left = r.n - r.scheduled;
    const uint64_t chunk = std::min<uint64_t>(left, piece);
    const size_t esz = dtype_size((int)r.dt);
    BatchDesc& D = sl.h_desc[items];
    D.ebase = host_exponent_base(r.seed, r.offset + r.scheduled);
    D.n = chunk;
    D.out = s->pool_dev + r.pool_off + r.scheduled * esz;
    D.dt = r.dt;
    D.head = (uint32_t)head_elems(D.out, esz, chunk);
    D.unit0 = units;
    sl.h_prefix[items] = units;
    const uint64_t unit_elems = batch_unit_elems(dd, tn.unit, (int)D.dt);
    units += chunk > D.head ? (chunk - D.head + unit_elems - 1) / unit_elems : 1;
    r.scheduled += chunk;
    ++items;
    if (r.scheduled == r.n) sl.finishing.push_back(id);
    else still.push_back(id);
  }
  sl.h_prefix[items] = units;
  s->active.swap(still);
  s->rr = s->active.empty() ? 0 : (s->rr + 1) % s->active.size();
  *units_out = units;
  *shape_out = shape;
  return items;
}

// Wall time of one runtime call, kept as the slowest of its kind (the
// server's stall diagnostics: which call a long launch spent its time in).
static cudaError_t timed_call(bcn_server* s, int kind, cudaError_t (*fn)(void*), void* arg) {
  const double t0 = now_s();
  const cudaError_t e = fn(arg);
  const uint64_t us = (uint64_t)((now_s() - t0) * 1e6);
  if (us > s->call_max_us[kind].load(std::memory_order_relaxed))
    s->call_max_us[kind].store(us, std::memory_order_relaxed);
  return e;
}

static void launch_slot(bcn_server* s, Slot& sl, uint32_t items, uint64_t units,
                        uint32_t shape) {
  const ServeShape& sh = s->shape[shape];
  const size_t desc_bytes = sizeof(BatchDesc) * s->cfg.max_items;
  const size_t prefix_bytes = sizeof(uint64_t) * (s->cfg.max_items + 1);
  struct Stage {
    Slot* sl;
    uint32_t items;
    size_t desc_bytes, prefix_bytes;
  } stage = {&sl, items, desc_bytes, prefix_bytes};
  cudaError_t e = timed_call(s, 0, [](void* a) {
    const Stage& g = *static_cast<Stage*>(a);
    cudaError_t r = cudaMemcpyAsync(g.sl->d_table, g.sl->h_desc, sizeof(BatchDesc) * g.items,
                                    cudaMemcpyHostToDevice, g.sl->cs);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(g.sl->d_table + g.desc_bytes, g.sl->h_prefix,
                          sizeof(uint64_t) * (g.items + 1), cudaMemcpyHostToDevice, g.sl->cs);
    if (r == cudaSuccess)
      r = cudaMemsetAsync(g.sl->d_table + g.desc_bytes + g.prefix_bytes, 0,
                          sizeof(unsigned long long), g.sl->cs);
    return r;
  }, &stage);
  unsigned long long* counter =
      reinterpret_cast<unsigned long long*>(sl.d_table + desc_bytes + prefix_bytes);
  if (e != cudaSuccess) return server_fail(s, e, "staging an iteration");
  BatchParams p;
  p.desc = reinterpret_cast<const BatchDesc*>(sl.d_table);
  p.prefix = reinterpret_cast<const uint64_t*>(sl.d_table + desc_bytes);
  p.counter = counter;
  p.total_units = units;
  uint32_t sd[3];
  batch_depths(sh.tune, sd);
  batch_fill_jumps(p, (int)sh.tune.step, (int)sh.tune.conv, (int)sh.tune.chains, sd);
  p.nstreams = items;
  p.unit_tiles = sh.tune.unit;
  p.skip = sh.tune.skip;
  p.nbuf = sh.tune.buffers;
  const uint64_t wpb = sh.tune.block / 32;
  const uint64_t grid = std::max<uint64_t>(1, std::min(sh.grid_full, (units + wpb - 1) / wpb));
  struct Launch {
    const ServeShape* sh;
    uint64_t grid;
    BatchParams* p;
    Slot* sl;
  } launch = {&sh, grid, &p, &sl};
  e = timed_call(s, 1, [](void* a) {
    const Launch& g = *static_cast<Launch*>(a);
    void* args[] = {g.p};
    return cudaLaunchKernel(g.sh->fn, dim3((unsigned)g.grid), dim3(g.sh->tune.block), args,
                            g.sh->smem, g.sl->cs);
  }, &launch);
  if (e == cudaSuccess)
    e = timed_call(s, 2, [](void* a) {
      Slot* sl2 = static_cast<Slot*>(a);
      return cudaEventRecord(sl2->ev, sl2->cs);
    }, &sl);
  if (e != cudaSuccess) return server_fail(s, e, "launching an iteration");
  sl.busy = true;
}

static void worker_main(bcn_server* s) {
  cudaSetDevice(s->device);
  double t_prev = now_s();
  while (!s->stop.load(std::memory_order_relaxed)) {
    {  // the longest time between two passes of this loop, sleeps excluded
      const double t = now_s();
      const uint64_t gap = (uint64_t)((t - t_prev) * 1e6);
      if (gap > s->loop_gap_max_us.load(std::memory_order_relaxed))
        s->loop_gap_max_us.store(gap, std::memory_order_relaxed);
    }
    bool did = retire(s);
    Slot* free_slot = nullptr;
    for (Slot& sl : s->slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    uint32_t items = 0, shape = 0;
    uint64_t units = 0;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      const double t = now_s();
      release_due(s, t);
      did |= admit(s, t);
      if (free_slot && !s->active.empty() && s->err == RNG_OK) {
        items = pack(s, *free_slot, &units, &shape);
        s->st.iterations += 1;
        s->st.heavy_iterations += shape;
        s->st.items += items;
        if (items > s->st.max_items_seen) s->st.max_items_seen = items;
      }
      if (!did && items == 0) {
        bool gpu_busy = false;
        for (Slot& sl : s->slots) gpu_busy |= sl.busy;
        const bool pending_release = !s->to_release.empty();
        if (!gpu_busy) {  // nothing on the device: sleep until new work (bounded)
          const double wait = pending_release
                                  ? std::max(0.0, s->to_release.front().first - t)
                                  : 0.002;
          s->cv_work.wait_for(lock, std::chrono::duration<double>(std::min(wait, 0.002)));
        }
      }
    }
    t_prev = now_s();  // a sleep above is not a stall
    if (items > 0) {
      launch_slot(s, *free_slot, items, units, shape);
      const uint64_t us = (uint64_t)((now_s() - t_prev) * 1e6);
      if (us > s->launch_max_us.load(std::memory_order_relaxed))
        s->launch_max_us.store(us, std::memory_order_relaxed);
      did = true;
    }
    if (!did) std::this_thread::yield();  // polling completion events
  }
}

}  // namespace bcn

using namespace bcn;

extern "C" {

rng_status rng_server_create(const rng_server_config* cfg_in, bcn_server** out) {
  if (!out || !cfg_in) return set_error(RNG_EINVAL, "NULL argument");
  *out = nullptr;
  rng_server_config cfg = *cfg_in;
  if (cfg.pool_bytes == 0) return set_error(RNG_EINVAL, "pool_bytes must be > 0");
  // defaults measured on the serving trace (20k req/s, 1 KiB..256 MiB): against
  // 2^21 and two slots, the saturated trace runs 1% faster and the nominal
  // one's p99 drops from 0.164 to 0.133 ms
  if (!cfg.chunk_elems) cfg.chunk_elems = 1ull << 22;
  cfg.chunk_elems = (cfg.chunk_elems + 3) / 4 * 4;  // chunks start 16-byte aligned
  if (!cfg.max_active) cfg.max_active = 4096;
  if (!cfg.max_items) cfg.max_items = 1024;
  if (!cfg.inflight) cfg.inflight = 4;
  if (cfg.inflight > 8) return set_error(RNG_EINVAL, "inflight must be 1..8");
  DeviceInfo di;
  rng_status stt = device_info(&di);
  if (stt != RNG_OK) return stt;
  stt = env_tune_check();
  if (stt != RNG_OK) return stt;
  // the caller's tuning gives one shape; a tuning left to the server gives two
  const rng_tune zero = {};
  const bool adaptive = memcmp(&cfg.tune, &zero, sizeof zero) == 0;
  ServeShape shapes[2];
  const uint32_t nshapes = adaptive ? 2 : 1;
  for (uint32_t k = 0; k < nshapes; ++k) {
    rng_tune t = cfg.tune;
    if (adaptive && k == 1) {  // the throughput shape
      t.depth = 31;
      t.block = 896;
      t.unit = 16;
      t.buffers = 1;
      t.chains = 2;
    }
    const rng_tune d = auto_defaults(RNG_F64);
    if (!t.step) t.step = d.step ? d.step : (uint32_t)ST_SHARED;
    if (!t.conv) t.conv = d.conv ? d.conv : (uint32_t)CV_INT;
    if (!t.skip) t.skip = SK_TABLE;
    if (!t.depth) t.depth = 15;
    if (!t.block) t.block = 256;
    if (!t.unit) t.unit = 4;
    t.buffers = batch_buffers(t);
    t.chains = batch_chains(t);
    if (t.depth % 2 == 0 || t.depth > kMaxDepth || t.block % 32 || !t.block || t.block > 1024 ||
        t.buffers > 2)
      return set_error(RNG_EINVAL, "bad server tuning");
    uint32_t td[3];
    batch_depths(t, td);
    const void* fn = batch_kernel_fn((int)t.step, (int)t.conv, (int)t.chains, td);
    if (!fn) return set_error(RNG_EINVAL, "no batch kernel for this step/conversion");
    const size_t smem = batch_smem_bytes(t.block, td, t.buffers);
    if (smem > di.smem_optin) return set_error(RNG_EINVAL, "tile buffers exceed shared memory");
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)di.smem_optin);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(server)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)t.block, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    shapes[k].tune = t;
    shapes[k].fn = fn;
    shapes[k].smem = smem;
    shapes[k].grid_full = (uint64_t)std::max(per_sm, 1) * (uint64_t)di.sms;
  }
  cudaError_t e = cudaSuccess;

  bcn_server* s = new (std::nothrow) bcn_server(cfg.pool_bytes);
  if (!s) return set_error(RNG_ENOMEM, "out of host memory");
  s->cfg = cfg;
  s->nshapes = nshapes;
  for (uint32_t k = 0; k < nshapes; ++k) s->shape[k] = shapes[k];
  if (nshapes > 1) {  // two wide tiles for every warp of the GPU
    const rng_tune& w = shapes[1].tune;
    s->heavy_elems = shapes[1].grid_full * (w.block / 32) * 2ull * 32ull * w.depth;
  }
  s->device = di.device;
  // admission bypass: by default a waiting request may be passed for 1 s
  // when the server frees results itself, never when the caller does
  s->bypass_s = cfg.admit_bypass_s > 0 ? cfg.admit_bypass_s
                : cfg.admit_bypass_s < 0 || cfg.release_after_s < 0 ? -1.0
                : kDefaultBypassS;
  auto cleanup = [s]() {
    for (Slot& sl : s->slots) {
      if (sl.ev) cudaEventDestroy(sl.ev);
      if (sl.cs) cudaStreamDestroy(sl.cs);
      if (sl.h_desc) cudaFreeHost(sl.h_desc);
      if (sl.h_prefix) cudaFreeHost(sl.h_prefix);
      if (sl.d_table) cudaFree(sl.d_table);
    }
    if (s->pool_dev) cudaFree(s->pool_dev);
    delete s;
  };
  e = dev_malloc((void**)&s->pool_dev, cfg.pool_bytes);
  if (e != cudaSuccess) {
    s->pool_dev = nullptr;
    cleanup();
    return cuda_error(e, "cudaMalloc(output pool)");
  }
  s->slots.resize(cfg.inflight);
  const size_t table = sizeof(BatchDesc) * cfg.max_items + sizeof(uint64_t) * (cfg.max_items + 1) + 16;
  for (Slot& sl : s->slots) {
    e = cudaStreamCreateWithFlags(&sl.cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = pinned_malloc((void**)&sl.h_desc, sizeof(BatchDesc) * cfg.max_items);
    if (e == cudaSuccess)
      e = pinned_malloc((void**)&sl.h_prefix, sizeof(uint64_t) * (cfg.max_items + 1));
    if (e == cudaSuccess) e = dev_malloc((void**)&sl.d_table, table);
    if (e != cudaSuccess) {
      cleanup();
      return cuda_error(e, "creating server slots");
    }
  }
  // First use of each slot's stream, and one empty launch of each kernel
  // shape on it (no work units), here rather than in the first iteration:
  // lazy initialisation in the runtime would otherwise land in a request's
  // latency.
  for (Slot& sl : s->slots) {
    const size_t desc_bytes = sizeof(BatchDesc) * cfg.max_items;
    const size_t prefix_bytes = sizeof(uint64_t) * (cfg.max_items + 1);
    BatchParams p = {};
    p.desc = reinterpret_cast<const BatchDesc*>(sl.d_table);
    p.prefix = reinterpret_cast<const uint64_t*>(sl.d_table + desc_bytes);
    p.counter = reinterpret_cast<unsigned long long*>(sl.d_table + desc_bytes + prefix_bytes);
    p.total_units = 0;
    for (uint32_t k = 0; k < nshapes && e == cudaSuccess; ++k) {
      const ServeShape& sh = s->shape[k];
      uint32_t sd[3];
      batch_depths(sh.tune, sd);
      batch_fill_jumps(p, (int)sh.tune.step, (int)sh.tune.conv, (int)sh.tune.chains, sd);
      p.unit_tiles = sh.tune.unit;
      p.skip = sh.tune.skip;
      p.nbuf = sh.tune.buffers;
      void* args[] = {&p};
      e = cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), sl.cs);
      if (e == cudaSuccess)
        e = cudaLaunchKernel(sh.fn, dim3(1), dim3(sh.tune.block), args, sh.smem, sl.cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sl.cs);
    if (e != cudaSuccess) {
      cleanup();
      return cuda_error(e, "warming the server slots");
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return RNG_OK;
}

}  // extern "C"

namespace bcn {

// Queue a request arriving at t_arrive; `sink` (nullable) collects its latency.
static rng_status submit_at(bcn_server* s, uint64_t start_index, uint64_t offset, uint64_t n,
                            rng_dtype dt, uint64_t* id, double t_arrive, TraceSink* sink,
                            uint32_t sink_idx) {
  if (!s || !id) return set_error(RNG_EINVAL, "NULL argument");
  if (start_index < kSeedMin || start_index > kSeedMax)
    return set_error(RNG_ERANGE, "start index outside [3^33+100, 2^53]");
  if ((int)dt < 0 || (int)dt > 2) return set_error(RNG_EINVAL, "bad dtype");
  if (n == 0) return set_error(RNG_EINVAL, "a request needs n > 0");
  if (n > RNG_MAX_N || n > UINT64_MAX - offset) return set_error(RNG_ERANGE, "n out of range");
  const uint64_t bytes = n * dtype_size((int)dt);
  if (bytes > s->cfg.pool_bytes)
    return set_error(RNG_ENOMEM, "request of %llu bytes exceeds the pool",
                     (unsigned long long)bytes);
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->err != RNG_OK) return set_error(s->err, "server failed: %s", s->errmsg);
  Request r;
  r.seed = start_index;
  r.offset = offset;
  r.n = n;
  r.bytes = bytes;
  r.dt = (uint32_t)dt;
  r.t_arrive = t_arrive;
  r.sink = sink;
  r.sink_idx = sink_idx;
  const uint64_t rid = s->next_id++;
  s->reqs.emplace(rid, r);
  s->queue.push_back(rid);
  s->st.submitted += 1;
  *id = rid;
  s->cv_work.notify_one();
  return RNG_OK;
}

}  // namespace bcn

extern "C" {

rng_status rng_server_submit(bcn_server* s, uint64_t start_index, uint64_t offset, uint64_t n,
                             rng_dtype dt, uint64_t* id) {
  return submit_at(s, start_index, offset, n, dt, id, now_s(), nullptr, 0);
}

rng_status rng_server_cancel(bcn_server* s, uint64_t id) {
  if (!s) return set_error(RNG_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    if (s->past.count(id)) return set_error(RNG_EBUSY, "request already finished");
    return set_error(RNG_EINVAL, "unknown request %llu", (unsigned long long)id);
  }
  if (it->second.state != RQ_QUEUED) return set_error(RNG_EBUSY, "request already admitted");
  it->second.state = RQ_CANCELLED;
  return RNG_OK;
}

rng_status rng_server_status(bcn_server* s, uint64_t id, int* state, double* latency_s) {
  if (!s) return set_error(RNG_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  int st = 0;
  double ta = 0, td = 0;
  if (!lookup(s, id, &st, &ta, &td))
    return set_error(RNG_EINVAL, "unknown request %llu", (unsigned long long)id);
  if (state) *state = st;
  if (latency_s) *latency_s = st >= RQ_DONE && st != RQ_CANCELLED ? td - ta : -1.0;
  return RNG_OK;
}

rng_status rng_server_wait(bcn_server* s, uint64_t id, double timeout_s) {
  if (!s) return set_error(RNG_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lock(s->mu);
  int st = 0;
  double ta = 0, td = 0;
  if (!lookup(s, id, &st, &ta, &td))
    return set_error(RNG_EINVAL, "unknown request %llu", (unsigned long long)id);
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s));
  while (st < RQ_DONE && s->err == RNG_OK) {
    const bool timed_out = s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout;
    lookup(s, id, &st, &ta, &td);  // a queued or active request is never forgotten
    if (timed_out && st < RQ_DONE)
      return set_error(RNG_ETIMEOUT, "request %llu not done after %.3f s", (unsigned long long)id,
                       timeout_s);
  }
  if (s->err != RNG_OK) return set_error(s->err, "server failed: %s", s->errmsg);
  if (st == RQ_CANCELLED) return set_error(RNG_EINVAL, "request was cancelled");
  return RNG_OK;
}

rng_status rng_server_read(bcn_server* s, uint64_t id, void* dst, uint64_t dst_bytes) {
  if (!s || !dst) return set_error(RNG_EINVAL, "NULL argument");
  uint64_t off = 0, bytes = 0;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
      if (s->past.count(id)) return set_error(RNG_EBUSY, "request released");
      return set_error(RNG_EINVAL, "unknown request");
    }
    if (it->second.state != RQ_DONE) return set_error(RNG_EBUSY, "request not done");
    if (it->second.release_pending) return set_error(RNG_EBUSY, "request released");
    off = it->second.pool_off;
    bytes = it->second.bytes;
    if (dst_bytes < bytes) return set_error(RNG_EINVAL, "destination smaller than the result");
    it->second.readers += 1;  // the range stays this request's until the copy ends
  }
  const cudaError_t e = cudaMemcpy(dst, s->pool_dev + off, bytes, cudaMemcpyDefault);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);  // a request with readers is never forgotten
    it->second.readers -= 1;
    if (it->second.readers == 0 && it->second.release_pending) release_range(s, it);
  }
  if (e != cudaSuccess) return cuda_error(e, "reading a result");
  return RNG_OK;
}

rng_status rng_server_result_ptr(bcn_server* s, uint64_t id, void** dev_ptr) {
  if (!s || !dev_ptr) return set_error(RNG_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    if (s->past.count(id)) return set_error(RNG_EBUSY, "request released");
    return set_error(RNG_EINVAL, "unknown request");
  }
  if (it->second.state != RQ_DONE) return set_error(RNG_EBUSY, "request not done");
  if (it->second.release_pending) return set_error(RNG_EBUSY, "request released");
  *dev_ptr = s->pool_dev + it->second.pool_off;
  return RNG_OK;
}

rng_status rng_server_release(bcn_server* s, uint64_t id) {
  if (!s) return set_error(RNG_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    if (s->past.count(id)) return set_error(RNG_EBUSY, "request already released");
    return set_error(RNG_EINVAL, "unknown request");
  }
  if (it->second.state != RQ_DONE || it->second.release_pending)
    return set_error(RNG_EBUSY, it->second.state != RQ_DONE ? "request not done"
                                                            : "request already released");
  release_range(s, it);
  return RNG_OK;
}

rng_status rng_server_stats_get(bcn_server* s, rng_server_stats* out) {
  if (!s || !out) return set_error(RNG_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->st;
  out->pool_in_use = s->pool.in_use;
  out->pool_bytes = s->cfg.pool_bytes;
  out->loop_gap_max_us = s->loop_gap_max_us.load();
  out->launch_max_us = s->launch_max_us.load();
  out->stage_max_us = s->call_max_us[0].load();
  out->kernel_launch_max_us = s->call_max_us[1].load();
  out->event_record_max_us = s->call_max_us[2].load();
  return s->err;
}

rng_status rng_server_latency_histogram(bcn_server* s, uint64_t* counts) {
  if (!s || !counts) return set_error(RNG_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  memcpy(counts, s->lat_hist, sizeof s->lat_hist);
  return s->err;
}

rng_status rng_server_run_trace(bcn_server* s, uint32_t n, const double* arrival_s,
                                const uint64_t* starts, const uint64_t* offsets,
                                const uint64_t* counts, const uint8_t* dtypes, double timeout_s,
                                double* latency_s, double* wall_s) {
  if (!s || !arrival_s || !starts || !counts || !dtypes || !latency_s)
    return set_error(RNG_EINVAL, "NULL argument");
  if (s->cfg.release_after_s < 0) {  // results stay in the pool: the trace must fit it
    uint64_t total = 0;
    for (uint32_t i = 0; i < n; ++i) {
      const uint64_t b = counts[i] > RNG_MAX_N
                             ? UINT64_MAX
                             : (counts[i] * dtype_size(dtypes[i]) + 255) / 256 * 256;
      total = total > UINT64_MAX - b ? UINT64_MAX : total + b;
    }
    if (total > s->cfg.pool_bytes)
      return set_error(RNG_EINVAL,
                       "the trace needs %llu pool bytes and release_after_s < 0 never frees "
                       "them: the pool holds %llu",
                       (unsigned long long)total, (unsigned long long)s->cfg.pool_bytes);
  }
  // the worker writes each latency into the sink as its request completes;
  // on every early return the trace's requests that are still pending are
  // detached from it (they keep running; only their latency goes unrecorded)
  TraceSink sink = {latency_s, 0, 0.0};
  std::vector<uint64_t> ids;
  ids.reserve(n);
  auto detach = [&]() {  // mu held
    for (uint64_t id : ids) {
      auto it = s->reqs.find(id);
      if (it != s->reqs.end() && it->second.sink == &sink) it->second.sink = nullptr;
    }
  };
  const double t0 = now_s();
  for (uint32_t i = 0; i < n; ++i) {
    const double due = t0 + arrival_s[i];
    while (now_s() < due) {
    }  // open-loop arrivals: spin until the request's arrival time
    uint64_t id = 0;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      sink.pending += 1;  // counted before the worker can complete it
    }
    // latency counts from the scheduled arrival
    rng_status st = submit_at(s, starts[i], offsets ? offsets[i] : 0, counts[i],
                              (rng_dtype)dtypes[i], &id, due, &sink, i);
    std::lock_guard<std::mutex> lock(s->mu);
    if (st != RNG_OK) {
      sink.pending -= 1;
      detach();
      return st;
    }
    ids.push_back(id);
  }
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s));
  std::unique_lock<std::mutex> lock(s->mu);
  while (sink.pending > 0 && s->err == RNG_OK) {
    if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && sink.pending > 0) {
      detach();
      return set_error(RNG_ETIMEOUT, "%llu of %u trace requests not done after %.3f s",
                       (unsigned long long)sink.pending, n, timeout_s);
    }
  }
  if (s->err != RNG_OK) {
    detach();
    return set_error(s->err, "server failed: %s", s->errmsg);
  }
  if (wall_s) *wall_s = n ? sink.last_done - t0 : 0.0;
  return RNG_OK;
}

rng_status rng_server_destroy(bcn_server* s) {
  if (!s) return RNG_OK;
  s->stop.store(true);
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (Slot& sl : s->slots) {
    if (sl.cs) cudaStreamSynchronize(sl.cs);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.cs) cudaStreamDestroy(sl.cs);
    if (sl.h_desc) cudaFreeHost(sl.h_desc);
    if (sl.h_prefix) cudaFreeHost(sl.h_prefix);
    if (sl.d_table) cudaFree(sl.d_table);
  }
  if (s->pool_dev) cudaFree(s->pool_dev);
  delete s;
  return RNG_OK;
}

}  // extern "C"
