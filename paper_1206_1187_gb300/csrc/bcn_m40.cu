// bcn_m40.cu -- bulk generation for the larger-modulus variant (modulus 3^40,
// Sec. 1; arithmetic in bcn_math40.cuh) on sm_103a.
//
// Layout and data movement are those of the 3^33 tiled kernel: the output
// is cut into tiles of 32*c elements (c odd), each warp owns a contiguous
// range of tiles, lane l of a tile produces its elements [l*c, (l+1)*c) into
// the warp's shared-memory tile buffer, and one lane hands the tile to the
// bulk async-copy engine.  Head (before the first 16-byte boundary) and tail
// (less than a tile) are stored directly by the grid's last warp.
//
// Per variate: one quotient floor(2^53 z / 3^40) (three 64-bit partial
// products), one remainder (one product), and a shift-and-or that joins two
// consecutive quotients into the truncated FP64 variate.  A chain therefore
// runs one quotient ahead of the variate it emits: it holds the state after
// the next variate's state and that variate's quotient.
#include <mutex>
#include <set>
#include <utility>

#include "bcn_gen.cuh"
#include "bcn_math40.cuh"

namespace bcn {

// One chain.  Variates (F64/F32): z is the state after the next variate's
// state, q the next variate's quotient.  States (U64): z is the next state.
template <int DT>
struct Chain40 {
  uint64_t z, q;
  // Begin at the variate whose state is s.
  __device__ __forceinline__ void start(uint64_t s) {
    if constexpr (DT == DT_U64) {
      z = s;
    } else {
      q = quot40(s);
      z = rem40(s, q);
    }
  }
  // A variate by the fast quotient and conversion (F64/F32 only).  qmin
  // tracks the smallest high word of the quotients used as a variate's
  // leading window (0 means a variate below 2^-21); fmax the largest high
  // word of the estimates' fractions (>= 0xFFFFFFFC means undecided).
  __device__ __forceinline__ typename Word<DT>::type next_fast(uint32_t& qmin, uint32_t& fmax) {
    uint32_t fhi;
    const uint64_t q1 = quot40_fast(z, fhi);
    fmax = max(fmax, fhi);
    const uint64_t bits = bits40_fast(q, q1);
    z = rem40(z, q1);
    q = q1;
    qmin = min(qmin, (uint32_t)(q1 >> 32));
    if constexpr (DT == DT_F64) return bits;
    else return f32_bits_from_f64_bits(bits);
  }
  __device__ __forceinline__ typename Word<DT>::type next() {
    if constexpr (DT == DT_U64) {
      const uint64_t w = z;
      z = rem40(z, quot40(z));
      return w;
    } else {
      const uint64_t q1 = quot40(z);
      const uint64_t bits = q != 0 ? bits40(q, q1) : bits40_small(z, q1);
      z = rem40(z, q1);
      q = q1;
      if constexpr (DT == DT_F64) return bits;
      else return f32_bits_from_f64_bits(bits);
    }
  }
};

// Steps between what a chain holds after emitting the variate before index
// i and the state of variate i: one for variates (the look-ahead), none for
// states.
template <int DT>
constexpr uint64_t kAhead40 = DT == DT_U64 ? 0 : 1;

__device__ __forceinline__ uint64_t state_of40(uint64_t ebase, uint64_t idx) {
  return seed_state40(exponent_add40(ebase, idx + 1));
}

struct M40Params {
  unsigned char* out;
  uint64_t n, head, ntiles, ebase;
  uint64_t jump;    // one chain: Montgomery form of 2^(53 (31c - ahead))
  uint64_t jump_a;  // two chains: 2^(53 (32c - h - 1 - ahead)) and
  uint64_t jump_b;  //             2^(53 (31c + h + 1 - ahead)), h = c/2
  uint32_t depth, nbuf;
};

template <int DT>
__device__ void run_direct40(typename Word<DT>::type* __restrict__ out, uint64_t ebase,
                             uint64_t a, uint64_t b) {
  if (a >= b) return;
  Chain40<DT> g;
  g.start(state_of40(ebase, a));
  for (uint64_t i = a; i < b; ++i) out[i] = g.next();
}

template <int DT, int ILP, int CDEPTH>
__global__ void __launch_bounds__(1024) tiled40_kernel(const M40Params p) {
  typedef typename Word<DT>::type W;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t wpb = blockDim.x >> 5;
  const uint64_t gw = (uint64_t)blockIdx.x * wpb + warp;
  const uint64_t nw = (uint64_t)gridDim.x * wpb;
  const uint32_t c = CDEPTH > 0 ? (uint32_t)CDEPTH : p.depth;
  const uint32_t tile_elems = 32u * c;
  const uint32_t tile_bytes = tile_elems * (uint32_t)sizeof(W);
  W* const buf0 = reinterpret_cast<W*>(smem + (size_t)warp * p.nbuf * tile_elems * sizeof(W));
  W* const out = reinterpret_cast<W*>(p.out);

  const uint64_t t0 = gw * p.ntiles / nw;
  const uint64_t t1 = (gw + 1) * p.ntiles / nw;
  if (t0 < t1) {
    const uint64_t first = p.head + t0 * tile_elems + (uint64_t)lane * c;
    const uint32_t h = c >> 1;
    Chain40<DT> a, b;
    a.start(state_of40(p.ebase, first));
    if constexpr (ILP == 2) b.start(state_of40(p.ebase, first + h + 1));
    uint32_t issued = 0;
    for (uint64_t t = t0; t < t1; ++t) {
      W* const buf = buf0 + (issued % p.nbuf) * tile_elems;
      wait_buffer_free(issued, p.nbuf, lane);
      W* const mine = buf + lane * c;
      if constexpr (DT == DT_U64) {
        if constexpr (ILP == 2) {
#pragma unroll
          for (uint32_t i = 0; i < (CDEPTH > 0 ? (uint32_t)CDEPTH / 2 : h); ++i) {
            mine[i] = a.next();
            mine[h + 1 + i] = b.next();
          }
          mine[h] = a.next();
        } else {
#pragma unroll
          for (uint32_t i = 0; i < (CDEPTH > 0 ? (uint32_t)CDEPTH : c); ++i) mine[i] = a.next();
        }
      } else {
        // fast path for the whole run; a lane whose run met an undecided
        // quotient or a variate below 2^-21 redoes it exactly
        const Chain40<DT> a0 = a, b0 = b;
        uint32_t qmin = (uint32_t)(a.q >> 32), fmax = 0;
        if constexpr (ILP == 2) {
          qmin = min(qmin, (uint32_t)(b.q >> 32));
#pragma unroll
          for (uint32_t i = 0; i < (CDEPTH > 0 ? (uint32_t)CDEPTH / 2 : h); ++i) {
            mine[i] = a.next_fast(qmin, fmax);
            mine[h + 1 + i] = b.next_fast(qmin, fmax);
          }
          mine[h] = a.next_fast(qmin, fmax);
        } else {
#pragma unroll
          for (uint32_t i = 0; i < (CDEPTH > 0 ? (uint32_t)CDEPTH : c); ++i)
            mine[i] = a.next_fast(qmin, fmax);
        }
        const bool rare = qmin == 0 || fmax >= 0xFFFFFFFCu;
        if (__any_sync(0xffffffffu, rare)) {
          if (rare) {
            a = a0;
            b = b0;
            if constexpr (ILP == 2) {
              for (uint32_t i = 0; i < h; ++i) {
                mine[i] = a.next();
                mine[h + 1 + i] = b.next();
              }
              mine[h] = a.next();
            } else {
              for (uint32_t i = 0; i < c; ++i) mine[i] = a.next();
            }
          }
          __syncwarp();
        }
      }
      fence_proxy_async_shared();
      __syncwarp();
      if (lane == 0) {
        bulk_store(out + p.head + t * tile_elems, buf, tile_bytes);
        bulk_commit();
      }
      ++issued;
      if (t + 1 < t1) {
        if constexpr (ILP == 2) {
          a.start(mont40(a.z, p.jump_a));
          b.start(mont40(b.z, p.jump_b));
        } else {
          a.start(mont40(a.z, p.jump));
        }
      }
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }

  if (gw == nw - 1) {  // head and tail, split contiguously over the lanes
    const uint64_t tail0 = p.head + p.ntiles * tile_elems;
    const uint64_t tl = p.n - tail0;
    run_direct40<DT>(out, p.ebase, lane * p.head / 32, (lane + 1) * p.head / 32);
    run_direct40<DT>(out, p.ebase, tail0 + lane * tl / 32, tail0 + (lane + 1) * tl / 32);
  }
}

template <int DT>
__global__ void __launch_bounds__(1024) direct40_kernel(unsigned char* out, uint64_t n,
                                                        uint64_t ebase) {
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t a = (uint64_t)((u128)n * t / T);
  const uint64_t b = (uint64_t)((u128)n * (t + 1) / T);
  run_direct40<DT>(reinterpret_cast<typename Word<DT>::type*>(out), ebase, a, b);
}

template <int DT>
static const void* pick40_dt(int layout, uint32_t chains, uint32_t depth) {
  if (layout == RNG_LAYOUT_DIRECT) return (const void*)direct40_kernel<DT>;
  if (chains == 2) {
    if (depth == 15) return (const void*)tiled40_kernel<DT, 2, 15>;
    if (depth == 31) return (const void*)tiled40_kernel<DT, 2, 31>;
    return (const void*)tiled40_kernel<DT, 2, 0>;
  }
  if (depth == 15) return (const void*)tiled40_kernel<DT, 1, 15>;
  if (depth == 31) return (const void*)tiled40_kernel<DT, 1, 31>;
  return (const void*)tiled40_kernel<DT, 1, 0>;
}

static const void* pick40(int dt, int layout, uint32_t chains, uint32_t depth) {
  switch (dt) {
    case DT_F64: return pick40_dt<DT_F64>(layout, chains, depth);
    case DT_F32: return pick40_dt<DT_F32>(layout, chains, depth);
    case DT_U64: return pick40_dt<DT_U64>(layout, chains, depth);
    default: return nullptr;
  }
}

// Defaults for fields left zero (measured on GB300 with the 2^28-variate
// FP64 workload).
constexpr uint32_t k40DefDepth = 31, k40DefBlock = 896, k40DefChains = 1, k40DefBuffers = 1;

struct Launch40 {
  int dt, layout;
  uint32_t depth, block, grid, chains, buffers;
  size_t smem_bytes;
};

static rng_status resolve40(uint64_t n, int dt, const rng_tune* tune, Launch40* out) {
  rng_tune t = {};
  if (tune) t = *tune;
  if (t.step || t.conv || t.skip || t.unit)
    return set_error(RNG_EINVAL,
                     "the 3^40 variant has one step, conversion and skip-ahead: tune.step, "
                     "conv, skip and unit must be 0");
  if (dt != DT_F64 && dt != DT_F32 && dt != DT_U64)
    return set_error(RNG_EINVAL, "dtype %d is not an rng_dtype", dt);
  Launch40 L = {};
  L.dt = dt;
  L.layout = t.layout ? (int)t.layout : RNG_LAYOUT_TILED;
  if (L.layout != RNG_LAYOUT_TILED && L.layout != RNG_LAYOUT_DIRECT)
    return set_error(RNG_EINVAL, "tune.layout %u is not a layout", t.layout);
  if (t.chains > 2) return set_error(RNG_EINVAL, "tune.chains %u must be 0, 1 or 2", t.chains);
  if (t.buffers > 2) return set_error(RNG_EINVAL, "tune.buffers %u must be 0, 1 or 2", t.buffers);
  DeviceInfo di;
  rng_status st = device_info(&di);
  if (st != RNG_OK) return st;
  if (L.layout == RNG_LAYOUT_TILED) {
    L.depth = t.depth ? t.depth : k40DefDepth;
    L.block = t.block ? t.block : k40DefBlock;
    if (L.depth % 2 == 0 || L.depth > kMaxDepth)
      return set_error(RNG_EINVAL, "tune.depth %u must be odd and at most %u", L.depth,
                       kMaxDepth);
    if (L.block % 32 != 0 || L.block == 0 || L.block > 1024)
      return set_error(RNG_EINVAL, "tune.block %u must be a multiple of 32, <= 1024", L.block);
    L.chains = t.chains ? t.chains : k40DefChains;
    if (L.depth < 3) L.chains = 1;
    L.buffers = t.buffers ? t.buffers : k40DefBuffers;
    L.smem_bytes = (size_t)(L.block / 32) * L.buffers * 32 * L.depth * dtype_size(dt);
    while (!t.block && L.smem_bytes > di.smem_optin && L.block > 32) {
      L.block /= 2;
      L.smem_bytes /= 2;
    }
    if (L.smem_bytes > di.smem_optin)
      return set_error(RNG_EINVAL, "tile buffers need %zu bytes of shared memory, %zu available",
                       L.smem_bytes, di.smem_optin);
    const void* fn = pick40(dt, L.layout, L.chains, L.depth);
    st = enable_smem(fn, di.device, L.smem_bytes);
    if (st != RNG_OK) return st;
    if (t.grid) {
      L.grid = t.grid;
    } else {
      int per_sm = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)L.block,
                                                                    L.smem_bytes);
      if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (per_sm < 1) per_sm = 1;
      const uint64_t full = (uint64_t)per_sm * (uint64_t)di.sms;
      const uint64_t tiles = n / (32ull * L.depth);
      uint64_t need = (tiles + L.block / 32 - 1) / (L.block / 32);
      if (need < 1) need = 1;
      L.grid = (uint32_t)(need < full ? need : full);
    }
  } else {
    L.chains = 1;
    L.block = t.block ? t.block : 256;
    if (L.block == 0 || L.block > 1024)
      return set_error(RNG_EINVAL, "tune.block %u must be in 1..1024", L.block);
    if (t.grid) {
      L.grid = t.grid;
    } else {
      const uint64_t threads = (n + 4095) / 4096;
      uint64_t g = (threads + L.block - 1) / L.block;
      if (g < 1) g = 1;
      if (g > (1u << 30)) g = 1u << 30;
      L.grid = (uint32_t)g;
    }
  }
  if (L.grid == 0 || L.grid > (1u << 30))
    return set_error(RNG_EINVAL, "tune.grid %u out of range", L.grid);
  *out = L;
  return RNG_OK;
}

static uint64_t jump40(uint64_t steps) {
  return host40_mont_form(host40_pow2((uint64_t)(((u128)53 * steps) % k40P)));
}

static rng_status launch40(const Launch40& L, uint64_t seed, uint64_t i0, uint64_t n, void* out,
                           cudaStream_t cs) {
  const void* fn = pick40(L.dt, L.layout, L.chains, L.depth);
  if (!fn) return set_error(RNG_EINVAL, "no kernel for this combination");
  const uint64_t ebase = host40_exponent_base(seed, i0);
  cudaError_t e;
  if (L.layout == RNG_LAYOUT_TILED) {
    const uint64_t ahead = L.dt == DT_U64 ? 0 : 1;
    const uint64_t c = L.depth, h = c / 2;
    M40Params p;
    p.out = static_cast<unsigned char*>(out);
    p.n = n;
    p.head = head_elems(out, dtype_size(L.dt), n);
    p.ntiles = n > p.head ? (n - p.head) / (32ull * c) : 0;
    p.ebase = ebase;
    p.jump = jump40(31 * c - ahead);
    p.jump_a = jump40(32 * c - h - 1 - ahead);
    p.jump_b = jump40(31 * c + h + 1 - ahead);
    p.depth = L.depth;
    p.nbuf = L.buffers;
    void* args[] = {&p};
    e = cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block), args, L.smem_bytes, cs);
  } else {
    unsigned char* o = static_cast<unsigned char*>(out);
    uint64_t nn = n, eb = ebase;
    void* args[] = {&o, &nn, &eb};
    e = cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block), args, 0, cs);
  }
  if (e != cudaSuccess) return cuda_error(e, "3^40 kernel launch");
  return RNG_OK;
}

}  // namespace bcn

using namespace bcn;

extern "C" {

rng_status rng40_generate_at(uint64_t start_index, uint64_t offset, uint64_t n, rng_dtype dt,
                             void* out, void* cuda_stream, const rng_tune* tune) {
  if (start_index < k40SeedMin)
    return set_error(RNG_ERANGE, "start index %llu below 3^40+100",
                     (unsigned long long)start_index);
  if (dt != RNG_F64 && dt != RNG_F32 && dt != RNG_U64)
    return set_error(RNG_EINVAL, "dtype %d is not an rng_dtype", (int)dt);
  if (n == 0) return RNG_OK;
  if (n > RNG_MAX_N)
    return set_error(RNG_ERANGE, "n = %llu exceeds RNG_MAX_N", (unsigned long long)n);
  if (out == nullptr) return set_error(RNG_EINVAL, "output pointer is NULL");
  if ((uintptr_t)out % dtype_size((int)dt) != 0)
    return set_error(RNG_EINVAL, "output pointer is not aligned to its %zu-byte elements",
                     dtype_size((int)dt));
  Launch40 L;
  rng_status st = resolve40(n, (int)dt, tune, &L);
  if (st != RNG_OK) return st;
  return launch40(L, start_index, offset, n, out, static_cast<cudaStream_t>(cuda_stream));
}

rng_status rng40_resolve_tune(uint64_t n, rng_dtype dt, const rng_tune* tune, rng_tune* out) {
  if (!out) return set_error(RNG_EINVAL, "out is NULL");
  Launch40 L;
  rng_status st = resolve40(n, (int)dt, tune, &L);
  if (st != RNG_OK) return st;
  rng_tune r = {};
  r.layout = (uint32_t)L.layout;
  r.depth = L.depth;
  r.block = L.block;
  r.grid = L.grid;
  r.chains = L.chains;
  r.buffers = L.buffers;
  *out = r;
  return RNG_OK;
}

}  // extern "C"
