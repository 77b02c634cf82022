/*
 * bcn_rng.h -- C ABI of the GB300 (sm_103a) alpha_{2,3} random variate
 * generator of Beliakov, Johnstone, Creighton and Wilkin, "Parallel random
 * variates generator for GPUs based on normal numbers".
 *
 * The generator is Algorithm BB (Sec. 1): a start index a in
 * [3^33+100, 2^53] is the seed, Eq. 2 gives
 *     z_0 = 2^(a - 3^33) * floor(3^33/2)  mod 3^33,
 * Eq. 3 iterates z_k = 2^53 z_(k-1) mod 3^33 and each z_k * 3^-33 is one
 * variate in (0,1).  Variate number i (counted from 0) of a stream is
 *     z = 2^((a - 3^33 + 53*(i+1)) mod P) * floor(3^33/2)  mod 3^33,
 * P = 2*3^32 the period, so any block of the sequence is reachable directly
 * (the skip-ahead property of Sec. 1) and the output does not depend on how
 * the work is split over threads.
 *
 * Output types:
 *   RNG_F64  double, RN(z * r3i) with r3i = 1.0/5559060566555523.0 (Fig. 4),
 *            one round-to-nearest multiply, no fused multiply-add.
 *   RNG_F32  float, the RNG_F64 variate rounded toward zero (stays in (0,1)).
 *   RNG_U64  the integer state z itself.
 *
 * Conventions for every entry point:
 *   - Return value: an rng_status; RNG_OK on success.  Nothing is thrown
 *     across this boundary.  rng_last_error() gives a message for the
 *     calling thread's last failure.
 *   - Device pointers are caller-owned CUDA global-memory addresses (for
 *     example a torch tensor's data_ptr()) on the current CUDA device; the
 *     library never frees them.  A pointer must be aligned to its element
 *     size, else RNG_EINVAL.
 *   - `cuda_stream` arguments are cudaStream_t handles passed as void*
 *     (NULL = the legacy default stream).  The calls that write device
 *     memory (rng_generate, rng_generate_tuned, rng_generate_at,
 *     rng40_generate_at, rng_fill_constant, rng_consume_mc) are asynchronous
 *     on that stream: they return after the launch, and the caller orders
 *     later use of the output on the same stream.  They allocate no device
 *     memory and wait for nothing; once a kernel has been launched on the
 *     device (so its shared-memory limit is set), later launches of it can
 *     be captured into a CUDA graph (checked for rng_generate_at and
 *     rng40_generate_at).  rng_generate_to_host is the synchronous
 *     exception.
 *   - A launch failure reported by the CUDA runtime is RNG_ECUDA.
 *   - bcn_stream objects are not thread-safe; use one per host thread.
 */
#ifndef BCN_RNG_H
#define BCN_RNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bcn_stream bcn_stream;

typedef enum { RNG_F64 = 0, RNG_F32 = 1, RNG_U64 = 2 } rng_dtype;

typedef enum {
  RNG_OK = 0,
  RNG_EINVAL = 1,   /* bad pointer, alignment, dtype, size or tuning field */
  RNG_ERANGE = 2,   /* seed outside [3^33+100, 2^53], or a count overflow  */
  RNG_ENOMEM = 3,   /* host allocation failed                              */
  RNG_ECUDA = 4,    /* the CUDA runtime reported an error                  */
  RNG_ETIMEOUT = 5, /* a bounded device-side wait ran out                  */
  RNG_EBUSY = 6     /* resource in use                                     */
} rng_status;

/* The reduction that advances the state (Sec. 2.1). */
typedef enum {
  RNG_STEP_AUTO = 0,           /* the measured-fastest variant                */
  RNG_STEP_BARRETT = 1,        /* Modified Barrett, Sec. 2.1.3, forward       */
  RNG_STEP_MONTGOMERY = 2,     /* Montgomery-style, R = 2^53, blocks run back */
  RNG_STEP_BARRETT_SHARED = 3, /* Barrett quotient estimate taken from the
                                  output-conversion product z*(mu+1), forward */
  RNG_STEP_LECUYER = 4,        /* L'Ecuyer's decomposition, a = 2^25, applied
                                  twice (Sec. 2.1.1), forward                 */
  RNG_STEP_BARRETT_CLASSIC = 5 /* Barrett's algorithm, k = 53 (Sec. 2.1.2)    */
} rng_step;

/* How a state becomes an FP64 variate (the RN multiply of Algorithm BB). */
typedef enum {
  RNG_CONV_AUTO = 0,
  RNG_CONV_INT = 1,   /* exact rounding emulated on the integer pipes      */
  RNG_CONV_FP64 = 2   /* int->double conversion and DMUL on the FP64 pipe  */
} rng_conv;

/* Work layout of a bulk call. */
typedef enum {
  RNG_LAYOUT_AUTO = 0,
  RNG_LAYOUT_TILED = 1,  /* lanes of a warp own consecutive runs of `depth`
                            variates of one tile; the warp's tile is staged in
                            shared memory and written by one bulk async copy */
  RNG_LAYOUT_DIRECT = 2, /* thread t of T owns [t*n/T, (t+1)*n/T) and stores
                            each variate itself (the paper's per-thread split,
                            Sec. 1; uncoalesced) */
  RNG_LAYOUT_STRIDED = 3 /* the paper's coalesced kernels (Sec. 2.2, its
                            partial-unrolling listing): thread t of T = n/W
                            makes variates t*W .. t*W+W-1 of the call and
                            stores variate t*W+j at position j*T+t.  The output
                            is that PERMUTATION of the sequence, not the
                            sequence order: W = tune.depth (0 = 4096, the
                            paper's choice) must divide n, tune.unit is the
                            loop's unroll factor (1 or 8; 0 = 8, the paper's
                            "Unrolled" kernels).  Only taken when a call's own
                            tuning names it, never as a default. */
} rng_layout;

/* Skip-ahead method for the state at the start of a block (Eq. 2). */
typedef enum {
  RNG_SKIP_AUTO = 0,
  RNG_SKIP_TABLE = 1,  /* 2^e from a compile-time table of 2^(d*256^k) */
  RNG_SKIP_SQMUL = 2   /* binary square-and-multiply                   */
} rng_skip_method;

/* Launch tuning.  Zero in any field means "choose": the tuning installed by
 * rng_set_auto_tune for the output type if any, else the shape measured best
 * on GB300: two chains per lane, one tile buffer per warp, and tiles 30 deep
 * in 896-thread blocks for FP64, 44 deep in 1024-thread blocks for FP32, 31
 * deep in 896-thread blocks for raw states (batch plans: 896-thread blocks,
 * each stream's tiles of its type's depth, 64-tile work units).  Results never
 * depend on these fields, only speed does -- except layout =
 * RNG_LAYOUT_STRIDED, which writes the paper's permuted order. */
typedef struct {
  uint32_t step;    /* rng_step                                              */
  uint32_t conv;    /* rng_conv                                              */
  uint32_t layout;  /* rng_layout                                            */
  uint32_t skip;    /* rng_skip_method                                       */
  uint32_t depth;   /* TILED: variates per lane per tile, odd, 1..255; with
                       the shared step on two chains also FP32 depths of
                       4 mod 8 (four variates per shared-memory store) and
                       FP64 depths of 2 mod 4 (two per store);
                       STRIDED: variates per thread                          */
  uint32_t block;   /* threads per block (TILED: multiple of 32, <= 1024)    */
  uint32_t grid;    /* blocks                                                */
  uint32_t unit;    /* BATCH: tiles per work unit (0 = choose); STRIDED: loop
                       unroll factor 1 or 8 (0 = 8); else ignored            */
  uint32_t chains;  /* TILED, forward steps: independent chains per lane, 1
                       or 2 (0 = choose); 2 splits each lane's run in halves */
  uint32_t buffers; /* TILED and BATCH: shared-memory tile buffers per warp,
                       1 or 2 (0 = choose); 1 halves the shared memory, so
                       more warps fit, at the cost of waiting for each tile's
                       copy to be read */
} rng_tune;

/* Largest n accepted by one generation call. */
#define RNG_MAX_N (1ULL << 46)

/* ---------------------------------------------------------------- streams */

/* Create a stream seeded with start index `start_index` (Algorithm BB,
 * step 1: 3^33+100 <= start_index <= 2^53, else RNG_ERANGE).  The stream's
 * count starts at 0 and it launches on the default CUDA stream until
 * rng_set_cuda_stream.  *out is library-owned; free it with rng_destroy. */
rng_status rng_create(uint64_t start_index, bcn_stream **out);

/* Free a stream created by rng_create.  NULL is a no-op. */
rng_status rng_destroy(bcn_stream *s);

/* Launch this stream's work on `cuda_stream` (a cudaStream_t). */
rng_status rng_set_cuda_stream(bcn_stream *s, void *cuda_stream);

/* Write the stream's next n variates (numbers count .. count+n-1, Eq. 3)
 * to the device array `out` (n elements of `dt`) and advance count by n.
 * n = 0 is a no-op.  n > RNG_MAX_N or a count past 2^64-1 is RNG_ERANGE. */
rng_status rng_generate(bcn_stream *s, uint64_t n, rng_dtype dt, void *out);

/* rng_generate with explicit launch tuning (NULL = automatic). */
rng_status rng_generate_tuned(bcn_stream *s, uint64_t n, rng_dtype dt, void *out,
                              const rng_tune *tune);

/* The stream's next n variates written to HOST memory `host_out` (n
 * elements of dt; page-locked memory gives the full transfer rate, pageable
 * memory works but each copy is staged).  Chunks of `chunk_bytes` (0 = 64 MiB)
 * are generated into `nbuf` (0 = 4, at most 8) rotating device staging
 * buffers, each on its own CUDA stream, and copied from there, so generation
 * and the device-to-host copies overlap.  The staging buffers are allocated on
 * the first call (and again if chunk_bytes or nbuf change) and kept until
 * rng_destroy.  Ordered after the work already queued on the stream's CUDA
 * stream; synchronous: returns when the data is in host memory.  Advances
 * count by n. */
rng_status rng_generate_to_host(bcn_stream *s, uint64_t n, rng_dtype dt, void *host_out,
                                uint64_t chunk_bytes, uint32_t nbuf);

/* Advance the count by k without generating (skip-ahead, Sec. 1; O(1)). */
rng_status rng_skip(bcn_stream *s, uint64_t k);

/* Checkpoint: the stream's seed and count.  The pair fully determines every
 * later variate; rng_set_state restores it (seed range as rng_create). */
rng_status rng_get_state(const bcn_stream *s, uint64_t *start_index, uint64_t *count);
rng_status rng_set_state(bcn_stream *s, uint64_t start_index, uint64_t count);

/* Wait for the stream's CUDA stream and report any asynchronous error. */
rng_status rng_sync(bcn_stream *s);

/* ------------------------------------------------------------- stateless */

/* Variates offset .. offset+n-1 of the sequence seeded with start_index,
 * written to `out` on `cuda_stream`.  Same rules as rng_generate. */
rng_status rng_generate_at(uint64_t start_index, uint64_t offset, uint64_t n,
                           rng_dtype dt, void *out, void *cuda_stream,
                           const rng_tune *tune);

/* Roofline probe (the paper's "Constant" kernel, Sec. 3.2): write the FP64
 * (dt = RNG_F64) or FP32 constant `value` n times to `out` with the same
 * tiled shared-memory + bulk-copy store path as generation.  Its rate is the
 * write ceiling the generator is measured against. */
rng_status rng_fill_constant(uint64_t n, rng_dtype dt, double value, void *out,
                             void *cuda_stream, const rng_tune *tune);

/* --------------------------------------------------------------- batches */

/* A batch: many independent streams of uneven length generated by one
 * persistent launch (the paper's parallel split of Sec. 1 applied to many
 * sequences at once).  Stream s writes variates offsets[s] ..
 * offsets[s]+counts[s]-1 of the sequence seeded with starts[s] to the device
 * array outs[s] as dtypes[s] (rng_dtype values); offsets may be NULL (all 0).
 * Each seed must satisfy Algorithm BB, step 1 (else RNG_ERANGE); each non-empty
 * output must be aligned to its element size (else RNG_EINVAL).  The host
 * arrays are copied; the output arrays stay caller-owned and must outlive the
 * plan's launches.  tune (NULL = choose) sets step, conversion, tile depth,
 * block, grid, chains, buffers and `unit` (tiles per work unit).  Creation
 * allocates a small
 * device table (about 48 bytes per stream) and synchronises the device, so it
 * is not capturable; launches are. */
typedef struct bcn_batch bcn_batch;
rng_status rng_batch_create(uint32_t nstreams, const uint64_t *starts, const uint64_t *offsets,
                            const uint64_t *counts, const uint8_t *dtypes, void *const *outs,
                            const rng_tune *tune, bcn_batch **out);

/* Generate every stream of the plan on `cuda_stream` (asynchronous: one
 * memset of the plan's work counter and one kernel launch).  Launches of one
 * plan must not overlap on the device: they share the work counter. */
rng_status rng_batch_launch(bcn_batch *b, void *cuda_stream);

/* The same work replayed as a CUDA graph (captured on first use, then one
 * cudaGraphLaunch per call on `cuda_stream`). */
rng_status rng_batch_graph_launch(bcn_batch *b, void *cuda_stream);

/* Totals of the plan and its resolved tuning (each pointer nullable); a
 * resolved depth of 0 means each stream's tiles take its type's built-in depth
 * (FP64 30, FP32 44, raw states 31). */
rng_status rng_batch_info(const bcn_batch *b, uint64_t *total_elems, uint64_t *total_bytes,
                          uint64_t *units, rng_tune *resolved);

/* Free the plan (its device table and graph).  NULL is a no-op. */
rng_status rng_batch_destroy(bcn_batch *b);

/* Batch generation that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * running under a framework whose caching allocator owns all device memory,
 * latency-critical paths that must not take the synchronisation an
 * allocation can imply, or hosts where device allocation is not permitted.
 * It generates the same streams, with the same meaning of every argument, as
 * rng_batch_create + rng_batch_launch, but its work table (descriptors, unit
 * prefix, work counter) lives in one fixed device array inside the library
 * instead of a cudaMalloc'd plan, and it allocates no device or host memory.
 *   - At most 1024 streams per call; more is RNG_ERANGE.  The array (about
 *     49 KB) is held by every device that loads the library until exit.
 *   - Zero tuning fields take a batch plan's shape (tiles 30 deep for FP64
 *     streams, 44 for FP32, 31 for raw states; 896-thread blocks, one buffer
 *     per warp, 64-tile work units).
 *   - The first call on a device, with that device current, looks up the
 *     array's device address, and the first call with each kernel shape
 *     (step, conversion, chains, depth) sets that kernel's shared-memory
 *     limit.  Make that first call on each device before any stream capture
 *     begins.
 *   - Every call rewrites the one shared table and clears its work counter:
 *     calls whose work overlaps on the GPU (on different streams, or from
 *     different host threads' streams) race and must be serialised by the
 *     caller.  Calls from several host threads are serialised on the host.
 *   - The table is copied from the library's host memory with
 *     cudaMemcpyAsync on `cuda_stream`; from pageable memory that copy may
 *     wait for earlier work on the stream before it returns.
 *   - Output arrays are caller-owned; the call is otherwise asynchronous. */
rng_status rng_batch_generate_noalloc(uint32_t nstreams, const uint64_t *starts,
                                      const uint64_t *offsets, const uint64_t *counts,
                                      const uint8_t *dtypes, void *const *outs,
                                      const rng_tune *tune, void *cuda_stream);

/* ------------------------------------------------ modulus 3^40 variant */

/* The larger-modulus generator that Sec. 1 sketches: Eq. 2 and Eq. 3 with
 * 3^40 in place of 3^33, i.e.
 *   z_0 = 2^(a - 3^40) floor(3^40/2) mod 3^40,  z_k = 2^53 z_(k-1) mod 3^40,
 * period 2*3^39 (about 8.1e18), states up to 3^40 - 1 > 2^63 (128-bit
 * products inside).  Variate i of seed a has the state
 * 2^(a - 3^40 + 53(i+1)) floor(3^40/2) mod 3^40 (step, then emit).
 *   - start_index: in [3^40 + 100, 2^64 - 1], else RNG_ERANGE.
 *   - RNG_F64: z / 3^40 rounded toward zero (its 53 significant bits are
 *     consecutive binary digits of alpha_{2,3}; every value is in (0,1),
 *     down to 3^-40).  RNG_F32: that value rounded toward zero to float.
 *     RNG_U64: the state z.
 *   - Writes variates offset .. offset+n-1 to the caller-owned device array
 *     `out` (aligned to the element size), asynchronously on `cuda_stream`
 *     (NULL = the legacy default stream).  n = 0 is a no-op; n > RNG_MAX_N is
 *     RNG_ERANGE.
 *   - tune: NULL or zero fields choose; layout, depth, block, grid, chains
 *     and buffers mean what they mean for rng_generate_at; step, conv, skip
 *     and unit must be 0 (the variant has one of each), else RNG_EINVAL.
 *     Tile depths are odd, except that FP32 on one chain (the default) also
 *     takes 44, its default; any other even depth is RNG_EINVAL. */
rng_status rng40_generate_at(uint64_t start_index, uint64_t offset, uint64_t n, rng_dtype dt,
                             void *out, void *cuda_stream, const rng_tune *tune);

/* The launch rng40_generate_at would make for n elements of dt: layout,
 * depth, block, grid, chains and buffers (other fields 0). */
rng_status rng40_resolve_tune(uint64_t n, rng_dtype dt, const rng_tune *tune, rng_tune *out);

/* ----------------------------------------------------------------- serving */

/* A continuous-batching request server (a serving form; the paper
 * has none).  Requests are generation calls (offset .. offset+n-1 of the
 * sequence seeded with a start index, as rng_generate_at) whose outputs are
 * placed in one device pool the server owns.  A scheduler thread admits
 * waiting requests in arrival order when a request slot is free and the pool
 * has room for the output (memory-based admission; a request that does not
 * fit may be passed by later ones that do for up to admit_bypass_s seconds,
 * after which nothing passes it until it is admitted), packs the next chunk of
 * every admitted request into one work table per iteration and launches the
 * batched kernel, with up to `inflight` iterations on separate CUDA streams so
 * work admitted later overlaps earlier work on the device.  Each chunk is a
 * block of its request's sequence reached by skip-ahead (Sec. 1), so a
 * request's bytes are the same alone and in any mix. */
typedef struct bcn_server bcn_server;

typedef struct {
  uint64_t pool_bytes;     /* device output pool, cudaMalloc'd at creation     */
  uint64_t chunk_elems;    /* piece of one request per iteration when many
                              requests are active (0 = 2^22; rounded up to a
                              multiple of 4); with k active requests a piece
                              may grow to 64*chunk_elems/k                      */
  uint32_t max_active;     /* admitted requests at once (0 = 4096)             */
  uint32_t max_items;      /* work items per iteration (0 = 1024)              */
  uint32_t inflight;       /* iterations in flight, 1..8 (0 = 4)               */
  uint32_t pad;
  double release_after_s;  /* >= 0: free a result's pool range this long after
                              it completes; < 0: the caller releases it        */
  rng_tune tune;           /* batched-kernel tuning; all zero = the server
                              picks per iteration: short tiles in small blocks
                              for light iterations, deep tiles in wide blocks
                              (one buffer per warp) once an iteration holds two
                              such tiles for every warp of the GPU            */
  double admit_bypass_s;   /* how long a queued request that does not fit the
                              pool may be passed by later requests that do:
                              > 0 that many seconds; < 0 never (strict arrival
                              order); 0 = 1 s when release_after_s >= 0,
                              never when the caller releases results (a client
                              consuming results in order could otherwise wait
                              on a request whose space is held by unreleased
                              requests that passed it)                       */
} rng_server_config;

typedef struct {
  uint64_t submitted, completed, iterations, items, max_items_seen;
  uint64_t peak_active, peak_pool_bytes, bytes_done, pool_in_use, pool_bytes;
  uint64_t heavy_iterations;  /* iterations launched with the throughput shape */
  uint64_t admitted_out_of_order; /* admissions that passed a waiting request  */
  uint64_t bypassed;          /* admission passes that found the oldest waiting
                                 request too large for the pool and went on   */
  uint64_t loop_gap_max_us;   /* longest interval between two passes of the
                                 scheduler loop, its own idle waits excluded  */
  uint64_t launch_max_us;     /* longest staging + launch of one iteration    */
  uint64_t stage_max_us;      /* of which: longest work-table copy + memset   */
  uint64_t kernel_launch_max_us; /* longest kernel launch call               */
  uint64_t event_record_max_us;  /* longest completion-event record          */
} rng_server_stats;

/* Request states reported by rng_server_status. */
enum { RNG_REQ_QUEUED = 0, RNG_REQ_ACTIVE = 1, RNG_REQ_DONE = 2, RNG_REQ_RELEASED = 3,
       RNG_REQ_CANCELLED = 4 };

/* Create a server on the current device (allocates the pool, per-iteration
 * tables and streams, starts the scheduler thread). */
rng_status rng_server_create(const rng_server_config *cfg, bcn_server **out);
/* Queue a request; thread-safe.  Rejected at once (and nothing else disturbed)
 * for a bad seed (RNG_ERANGE), dtype or n == 0 (RNG_EINVAL), or an output larger
 * than the pool (RNG_ENOMEM).  *id identifies it afterwards. */
rng_status rng_server_submit(bcn_server *s, uint64_t start_index, uint64_t offset, uint64_t n,
                             rng_dtype dt, uint64_t *id);
/* Withdraw a request that is still queued (RNG_EBUSY once admitted). */
rng_status rng_server_cancel(bcn_server *s, uint64_t id);
/* Request ids stay known while the request is queued, active or done; after
 * its pool range is released (or a cancelled request leaves the queue) the
 * server keeps its final state and times for the 65536 most recent such
 * requests only, so its bookkeeping stays bounded.  An id no longer known is
 * RNG_EINVAL in the calls below; reading or releasing a released request is
 * RNG_EBUSY. */
/* State and, once done, latency (submission or scheduled arrival to the
 * host seeing its last iteration complete, seconds; -1 before). */
rng_status rng_server_status(bcn_server *s, uint64_t id, int *state, double *latency_s);
/* Block until the request is done (RNG_ETIMEOUT after timeout_s). */
rng_status rng_server_wait(bcn_server *s, uint64_t id, double timeout_s);
/* Copy a done request's result (n elements of its dtype) to `dst` (host or
 * device memory of at least dst_bytes); synchronous.  The result's pool range
 * stays the request's until the copy returns: a release that falls due during
 * the copy (release_after_s >= 0, or rng_server_release from another thread)
 * takes effect when it ends. */
rng_status rng_server_read(bcn_server *s, uint64_t id, void *dst, uint64_t dst_bytes);
/* The device address of a done request's result inside the pool, valid until
 * the request is released.  With release_after_s >= 0 the server releases it
 * release_after_s seconds after completion, whatever the caller is doing with
 * the address; callers that keep the address use release_after_s < 0 and
 * rng_server_release, or rng_server_read, which holds the range while it
 * copies. */
rng_status rng_server_result_ptr(bcn_server *s, uint64_t id, void **dev_ptr);
/* Free a done request's pool range now. */
rng_status rng_server_release(bcn_server *s, uint64_t id);
/* Counters since creation (returns the server's error status, if any). */
rng_status rng_server_stats_get(bcn_server *s, rng_server_stats *out);
/* Latencies of the requests completed since creation (as rng_server_status
 * reports them) in quarter-octave bins: bin k counts latencies in
 * [2^(k/4), 2^((k+1)/4)) microseconds, bin 0 also everything shorter and the
 * last bin everything longer (2^(95/4) us is about 14 s).  `counts` receives
 * RNG_SERVER_HIST_BINS words.  Returns the server's error status, if any. */
#define RNG_SERVER_HIST_BINS 96
rng_status rng_server_latency_histogram(bcn_server *s, uint64_t *counts);
/* Replay a request trace in real time: request i is submitted at
 * arrival_s[i] seconds after the call starts (open loop), then every request
 * is awaited (RNG_ETIMEOUT after timeout_s).  latency_s[i] receives the time
 * from request i's scheduled arrival to its completion, written by the
 * scheduler as the request completes (any trace length); *wall_s (nullable)
 * the time from the start to the last completion.  On an error return the
 * trace's requests already submitted keep running, and entries of latency_s
 * for those not yet complete are left as they were.  With release_after_s < 0 the
 * results are never freed, so a trace whose outputs exceed the pool is
 * RNG_EINVAL before anything is submitted. */
rng_status rng_server_run_trace(bcn_server *s, uint32_t n, const double *arrival_s,
                                const uint64_t *starts, const uint64_t *offsets,
                                const uint64_t *counts, const uint8_t *dtypes, double timeout_s,
                                double *latency_s, double *wall_s);
/* Stop the scheduler (after the iterations in flight) and free everything. */
rng_status rng_server_destroy(bcn_server *s);

/* The pool sub-allocator the server admits with: aligned first-fit ranges of
 * a `capacity`-byte pool, neighbours merged on free.  Host bookkeeping only
 * (no device memory is touched), exposed so it can be driven on its own. */
typedef struct bcn_pool bcn_pool;
rng_status rng_pool_create(uint64_t capacity, uint64_t align, bcn_pool **out);
rng_status rng_pool_alloc(bcn_pool *p, uint64_t bytes, uint64_t *offset);  /* RNG_ENOMEM if none */
rng_status rng_pool_free(bcn_pool *p, uint64_t offset);
rng_status rng_pool_stats(bcn_pool *p, uint64_t *in_use, uint64_t *peak, uint64_t *live,
                          uint64_t *largest_free, uint64_t *free_ranges);
rng_status rng_pool_destroy(bcn_pool *p);

/* ---------------------------------------------------------- fused consumer */

/* A Monte-Carlo consumer fused with generation: variates are used on the
 * device and never stored (the use Sec. 2.2 of the paper anticipates).  The
 * sequence seeded with start_index is cut into blocks of `len` variates (len
 * even); block g = block0 + b (b < nblocks) covers variates g*len ..
 * (g+1)*len-1.  Its variates are paired (v_2j, v_2j+1) = (x, y) and the call
 * writes, for each b:
 *   hits[b]  (nullable) = number of pairs with RN(RN(x*x) + RN(y*y)) <= 1,
 *   sum[b]   = the exact sum of the block's variates, rounded to nearest even,
 *   sumsq[b] = the exact sum of RN(v*v) over the block, rounded likewise,
 * and *hits_total = the hit count over all nblocks blocks (the call zeroes it
 * first).  All outputs are caller-owned device arrays, 8-byte aligned.
 * Results are exact (integer arithmetic on the 2^-105 and 2^-157 grids), so
 * they do not depend on the launch shape.  Asynchronous on `cuda_stream`.
 * tune: only `block` (multiple of 32, <= 256), `skip` and `conv` are read;
 * conv = RNG_CONV_FP64 (or 0, the default) takes each RN(v*v) with one FP64
 * multiply, RNG_CONV_INT forms it on the integer pipes; the results are
 * identical. */
rng_status rng_consume_mc(uint64_t start_index, uint64_t block0, uint64_t nblocks, uint64_t len,
                          uint64_t *hits_total, uint64_t *hits, double *sum, double *sumsq,
                          void *cuda_stream, const rng_tune *tune);

/* rng_consume_mc that also returns the call's exact totals over all its
 * blocks in a form that adds without rounding across calls, GPUs and
 * processes -- the one exchange the paper's parallel split (Sec. 1) needs
 * when the blocks of one sequence are spread over ranks: the ranks add their
 * word arrays element by element (an integer all-reduce, exact and
 * order-free) and round once with rng_mc_round_totals.
 *   totals: caller-owned device array of RNG_MC_TOTAL_WORDS uint64 words,
 *   8-byte aligned (NULL: plain rng_consume_mc), zeroed by the call.  For
 *   k < 5, word k is the sum over the call's blocks of bits 32k..32k+31 of
 *   the block's exact sum of v * 2^105 (below 2^138); for k < 6, word 5+k
 *   the same of the block's exact sum of RN(v*v) * 2^157 (below 2^190).  So
 *   the words T stand for
 *     sum of v      = (T[0] + T[1] 2^32 + ... + T[4] 2^128) * 2^-105,
 *     sum of RN(v^2) = (T[5] + T[6] 2^32 + ... + T[10] 2^160) * 2^-157.
 *   Each word gains less than 2^32 per block, so word arrays stay exact for
 *   up to 2^32 blocks in all (a call of more blocks is RNG_ERANGE).
 * Other arguments, outputs and errors as rng_consume_mc. */
#define RNG_MC_TOTAL_WORDS 11
rng_status rng_consume_mc_totals(uint64_t start_index, uint64_t block0, uint64_t nblocks,
                                 uint64_t len, uint64_t *hits_total, uint64_t *hits, double *sum,
                                 double *sumsq, uint64_t *totals, void *cuda_stream,
                                 const rng_tune *tune);

/* Host only: round a totals word array (one call's, or the element-wise sum
 * of several calls' arrays, which must stay within 2^32 blocks in all) to
 * *sum = RN(exact sum of the variates) and *sumsq = RN(exact sum of their
 * RN(v*v)), round-to-nearest-even.  RNG_EINVAL for a NULL pointer. */
rng_status rng_mc_round_totals(const uint64_t *totals, double *sum, double *sumsq);

/* Run a kernel written only against the device-side API (bcn_device.cuh):
 * `threads` threads each create their own generator at their first variate
 * and write variates offset .. offset+n-1 of the sequence seeded with
 * start_index, as FP64 to out_f64, FP32 to out_f32 and, when out_state is not
 * NULL, their raw states to out_state (caller-owned device arrays of n
 * elements, aligned to their element size).  Exposes the device API to the
 * same checks as every other path.  Asynchronous on `cuda_stream`. */
rng_status rng_device_api_check(uint64_t start_index, uint64_t offset, uint64_t n,
                                double *out_f64, float *out_f32, uint64_t *out_state,
                                uint32_t threads, void *cuda_stream);

/* The device-side API used as the paper intends it for simulations on the GPU
 * (Sec. 2: each thread an independent subsequence with a 64-bit state, no
 * shared memory): `threads` threads (a positive multiple of 128, else
 * RNG_EINVAL) each take variates [t*n/T, (t+1)*n/T) of offset .. offset+n-1
 * of the sequence seeded with start_index (else RNG_ERANGE) and consume them
 * in registers; thread t writes only the sum modulo 2^64 of their bit
 * patterns to sums[t] (a caller-owned device array of `threads` words,
 * 8-byte aligned, else RNG_EINVAL).  dt = RNG_F64: one next_f64 call per
 * variate; RNG_F32: runs of 32 from f32_run, the rest from next_f32 (32-bit
 * patterns); any other dt is RNG_EINVAL.  n = 0 writes zeros.  Nothing else
 * is stored and the consumer is one integer add per variate, so the call
 * times the generator itself.  Asynchronous on `cuda_stream`. */
rng_status rng_device_api_checksum(uint64_t start_index, uint64_t offset, uint64_t n,
                                   rng_dtype dt, uint64_t *sums, uint32_t threads,
                                   void *cuda_stream);

/* The device-side FP32 runs (bcn_device::f32_run): `threads` threads (a
 * positive multiple of 128, else RNG_EINVAL) each write FP32 variates
 * [t*n/T, (t+1)*n/T) of offset .. offset+n-1 of the sequence seeded with
 * start_index (else RNG_ERANGE) to `out` (a caller-owned device array of n
 * floats, 4-byte aligned, else RNG_EINVAL), in runs of 32 made by f32_run and
 * the remainder by next_f32, so that the runs meet the same checks as every
 * other path.  n = 0 is a no-op.  Asynchronous on `cuda_stream`. */
rng_status rng_device_api_f32_runs(uint64_t start_index, uint64_t offset, uint64_t n,
                                   float *out, uint32_t threads, void *cuda_stream);

/* -------------------------------------------------------------- autotune */

/* Time each of the `ncand` candidate tunings of a bulk call (n elements of
 * dt written to the caller-owned device buffer `out`, which is overwritten)
 * on `cuda_stream`: one warm-up and `reps` timed launches each, CUDA events.
 * The fastest valid candidate, fully resolved, goes to *best; ms[i]
 * (nullable) receives candidate i's mean milliseconds per launch, or -1 if
 * the candidate is invalid (for example too much shared memory).  Blocks
 * until the timings are done.  The selection-by-measurement the paper makes
 * over threads per block (Sec. 3.2), applied to this library's parameters. */
rng_status rng_autotune_bulk(uint64_t n, rng_dtype dt, void *out, void *cuda_stream,
                             const rng_tune *candidates, uint32_t ncand, uint32_t reps,
                             rng_tune *best, float *ms);

/* Install `t` as the choice for the zero fields of later calls of dtype dt
 * (its grid is ignored: the grid follows n).  NULL restores the built-in
 * choice.  Process-wide; results never change, only speed (a tuning naming
 * RNG_LAYOUT_STRIDED, which permutes the output, is RNG_EINVAL here).
 *
 * The environment variable BCN_RNG_TUNE, when set, overrides every installed
 * tuning for the 3^33 generator's calls: it is read once, on the first call
 * that resolves a launch, in the form rng_parse_tune reads (for example
 * "step=barrett,conv=fp64,depth=15,block=256"); its fields fill the zero
 * fields of bulk calls, and its step and conversion those of batch plans and
 * the server (grid is ignored).  If it does not parse, every such call fails
 * with RNG_EINVAL naming the problem. */
rng_status rng_set_auto_tune(rng_dtype dt, const rng_tune *t);

/* Read a tuning from text: comma-separated key=value pairs with the keys
 * step (barrett, montgomery, shared, lecuyer, barrett_classic), conv (int,
 * fp64), layout (tiled, direct, strided), skip (table, sqmul), depth, block, grid,
 * unit, chains and buffers (decimal; enum fields also accept their numbers).
 * Fields not named are 0; spaces around pairs are allowed.  RNG_EINVAL for an
 * unknown key or a bad value.  Host-only; checks no ranges (a launch does). */
rng_status rng_parse_tune(const char *text, rng_tune *out);

/* ------------------------------------------------------------- utilities */

/* The calling thread's last error message ("" if none). */
const char *rng_last_error(void);

/* The choices an automatic call makes for (n, dt) on the current device. */
rng_status rng_resolve_tune(uint64_t n, rng_dtype dt, const rng_tune *in, rng_tune *out);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int rng_version(void);

/* Testing hook: after `skip` more device or pinned-host allocations by the
 * library succeed, make the next `count` fail as if cudaMalloc (or
 * cudaMallocHost) had run out of memory (cudaErrorMemoryAllocation, reported
 * as RNG_ECUDA by the failing call, which frees what it had allocated).
 * count = 0 turns injection off.  Process-wide.  The allocating calls are
 * rng_batch_create, rng_server_create and the first rng_generate_to_host of a
 * stream (or one with a new chunk size or buffer count). */
rng_status rng_debug_fail_allocations(uint32_t skip, uint32_t count);

#ifdef __cplusplus
}
#endif

#endif /* BCN_RNG_H */
