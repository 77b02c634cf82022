// bcn_gen.cuh -- the per-lane generator shared by the bulk, batched and
// fused kernels: output words, one chain of Eq. 3 under each reduction,
// block-start states (Eq. 2), plain-store runs and the bulk async-copy
// primitives that move a warp's shared-memory tile to global memory.
#pragma once
#include "bcn_internal.h"
#include "bcn_math.cuh"

namespace bcn {

template <int DT> struct Word { typedef uint64_t type; };
template <> struct Word<DT_F32> { typedef uint32_t type; };

// The output word of state z.  (phi, plo) is the product z*mu when the
// caller has it (Barrett) -- the integer conversion reuses it.
template <int DT, int CONV>
__device__ __forceinline__ typename Word<DT>::type to_word(uint64_t z, uint64_t phi,
                                                           uint64_t plo) {
  if constexpr (DT == DT_U64) {
    return z;
  } else {
    uint64_t bits;
    if constexpr (CONV == CV_INT) {
      uint64_t qh, ql;
      p_from_barrett_product(z, phi, plo, qh, ql);
      bits = f64_bits_from_p(qh, ql);
    } else {
      bits = f64_bits_fp64_fma(z);  // every conversion on the FP64 pipe
    }
    if constexpr (DT == DT_F64) return bits;
    else return f32_bits_from_f64_bits(bits);
  }
}

// One chain of the generator.  Barrett runs forward (z is the state of the
// next variate to emit); Montgomery runs backward (z is the state of the
// variate emitted next, going down).
template <int DT, int STEP, int CONV>
struct Gen {
  uint64_t z;
  __device__ __forceinline__ typename Word<DT>::type next() {
    if constexpr (STEP == ST_SHARED) {
      if constexpr (DT == DT_U64) {
        const uint64_t w = z;
        z = shared_advance(z);
        return w;
      } else if constexpr (CONV == CV_FP64) {
        const uint64_t bits = f64_bits_fp64_fma(z);
        z = shared_advance(z);
        if constexpr (DT == DT_F64) return bits;
        else return f32_bits_from_f64_bits(bits);
      } else {
        const uint64_t bits = shared_step_f64(z);
        if constexpr (DT == DT_F64) return bits;
        else return f32_bits_from_f64_bits(bits);
      }
    } else if constexpr (STEP == ST_BARRETT) {
      uint64_t plo = z * kMu, phi = umulhi(z, kMu);
      auto w = to_word<DT, CONV>(z, phi, plo);
      z = barrett_from_product(phi, plo);
      return w;
    } else if constexpr (STEP == ST_LECUYER || STEP == ST_BCLASSIC) {
      uint64_t plo = 0, phi = 0;
      if constexpr (DT != DT_U64 && CONV == CV_INT) {
        plo = z * kMu;
        phi = umulhi(z, kMu);
      }
      auto w = to_word<DT, CONV>(z, phi, plo);
      if constexpr (STEP == ST_LECUYER) z = lecuyer_step(z);
      else z = barrett_classic_step(z);
      return w;
    } else {
      uint64_t plo = 0, phi = 0;
      if constexpr (DT != DT_U64 && CONV == CV_INT) {
        plo = z * kMu;
        phi = umulhi(z, kMu);
      }
      auto w = to_word<DT, CONV>(z, phi, plo);
      z = montgomery_back(z);
      return w;
    }
  }
};

__device__ __forceinline__ uint64_t seed_state(uint64_t e, uint32_t skip) {
  return skip == SK_SQMUL ? seed_state_sqmul(e) : seed_state_table(e);
}

// State of element idx of the call: exponent ebase + 53*(idx+1)  (mod P).
__device__ __forceinline__ uint64_t state_of(uint64_t ebase, uint64_t idx, uint32_t skip) {
  return seed_state(exponent_add(ebase, idx + 1), skip);
}

// Elements [a, b) with plain global stores.
template <int DT, int STEP, int CONV>
__device__ void run_direct(typename Word<DT>::type* __restrict__ out, uint64_t ebase,
                           uint32_t skip, uint64_t a, uint64_t b, uint64_t cbits) {
  typedef typename Word<DT>::type W;
  if (a >= b) return;
  if constexpr (STEP == ST_CONST) {
    for (uint64_t i = a; i < b; ++i) out[i] = (W)cbits;
  } else if constexpr (STEP != ST_MONT) {
    Gen<DT, STEP, CONV> g{state_of(ebase, a, skip)};
    for (uint64_t i = a; i < b; ++i) out[i] = g.next();
  } else {
    Gen<DT, STEP, CONV> g{state_of(ebase, b - 1, skip)};
    for (uint64_t i = b; i-- > a;) out[i] = g.next();
  }
}

// ------------------------------------------------------- bulk async copies
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
  const uint64_t g = (uint64_t)__cvta_generic_to_global(gdst);
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(ssrc);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
               :: "l"(g), "r"(s), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Before a warp refills a tile buffer: with two buffers, the copy committed
// two tiles ago (the last reader of this buffer) must be done reading; with
// one buffer, the previous copy must be.
__device__ __forceinline__ void wait_buffer_free(uint32_t issued, uint32_t nbuf, uint32_t lane) {
  if (issued >= nbuf) {
    if (lane == 0) {
      if (nbuf == 1) bulk_wait_read_0();
      else bulk_wait_read_1();
    }
    __syncwarp();
  }
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// The buffer a warp fills next (one or two buffers per warp; no division).
__device__ __forceinline__ uint32_t tile_buffer(uint32_t issued, uint32_t nbuf) {
  return nbuf == 2 ? (issued & 1u) : 0u;
}


// The shared-quotient step's fast path for a whole run of c variates: no
// per-variate branch; a lane whose run met the rare case (a variate below
// 2^-21, probability about 2^-21 each) redoes its run exactly after a
// warp-uniform vote.
template <int DT, int CDEPTH>
__device__ __forceinline__ void shared_run_fast(typename Word<DT>::type* mine, uint32_t c,
                                                uint64_t& z) {
  typedef typename Word<DT>::type W;
  const uint64_t z_start = z;
  bool rare = false;
  if constexpr (CDEPTH > 0) {
#pragma unroll
    for (uint32_t i = 0; i < (uint32_t)CDEPTH; ++i) {
      const uint64_t b = shared_step_f64_fast(z, rare);
      if constexpr (DT == DT_F64) mine[i] = (W)b;
      else mine[i] = (W)f32_bits_from_f64_bits(b);
    }
  } else {
#pragma unroll 4
    for (uint32_t i = 0; i < c; ++i) {
      const uint64_t b = shared_step_f64_fast(z, rare);
      if constexpr (DT == DT_F64) mine[i] = (W)b;
      else mine[i] = (W)f32_bits_from_f64_bits(b);
    }
  }
  if (__any_sync(0xffffffffu, rare)) {
    if (rare) {
      uint64_t y = z_start;
      for (uint32_t i = 0; i < c; ++i) {
        const uint64_t b = shared_step_f64(y);
        if constexpr (DT == DT_F64) mine[i] = (W)b;
        else mine[i] = (W)f32_bits_from_f64_bits(b);
      }
    }
    __syncwarp();
  }
}

// `ntiles` consecutive tiles of 32*c elements, the first at element `first`
// of `out` (16-byte aligned).  Lane l produces elements [l*c, (l+1)*c) of each
// tile with c steps of chain g, writes them to one of the warp's `nbuf` tile
// buffers in shared memory, and lane 0 hands the tile to the bulk-copy engine.
// `issued` counts the warp's committed bulk groups: before a buffer is reused,
// lane 0 waits until the copy that last read it is done.  Between tiles the
// chain jumps with one product by `jump` (2^(53*31c) forward, 2^(53*33c) for
// the backward Montgomery chain, whose state is the last element of a run);
// `jump_q` is its precomputed quotient for mulmod_pre.
template <int DT, int STEP, int CONV, int CDEPTH = 0>
__device__ __forceinline__ void warp_tiles(typename Word<DT>::type* __restrict__ out,
                                           uint64_t first, uint64_t ntiles, uint32_t c_rt,
                                           uint64_t jump, uint64_t jump_q, Gen<DT, STEP, CONV>& g,
                                           typename Word<DT>::type* buf0, uint32_t& issued,
                                           uint32_t lane, uint64_t cbits, uint32_t nbuf = 2) {
  typedef typename Word<DT>::type W;
  const uint32_t c = CDEPTH > 0 ? (uint32_t)CDEPTH : c_rt;
  const uint32_t tile_elems = 32u * c;
  const uint32_t tile_bytes = tile_elems * (uint32_t)sizeof(W);
  for (uint64_t t = 0; t < ntiles; ++t) {
    W* const buf = buf0 + tile_buffer(issued, nbuf) * tile_elems;
    wait_buffer_free(issued, nbuf, lane);
    W* const mine = buf + lane * c;
    if constexpr (STEP == ST_CONST) {
      for (uint32_t i = 0; i < c; ++i) mine[i] = (W)cbits;
    } else if constexpr (STEP == ST_SHARED && CONV == CV_INT && DT != DT_U64) {
      shared_run_fast<DT, CDEPTH>(mine, c, g.z);
    } else if constexpr (STEP != ST_MONT) {
#pragma unroll 4
      for (uint32_t i = 0; i < c; ++i) mine[i] = g.next();
    } else {
#pragma unroll 4
      for (uint32_t i = c; i-- > 0;) mine[i] = g.next();
    }
    fence_proxy_async_shared();
    __syncwarp();
    if (lane == 0) {
      bulk_store(out + first + t * tile_elems, buf, tile_bytes);
      bulk_commit();
    }
    ++issued;
    if constexpr (STEP != ST_CONST) {
      if (t + 1 < ntiles) g.z = mulmod_pre(g.z, jump, jump_q);
    }
  }
}

// Two independent chains per lane: the lane's run of c elements is split at
// s = chain_split(c) into elements [0, s) (chain a) and [s, c) (chain b), and
// the two chains step alternately, so each step's latency is hidden behind
// the other chain's work.  With odd c (s = h+1, h = c/2) the stores to mine[i]
// and mine[h+1+i] keep lane stride c, so they stay bank-conflict free.
// Between tiles the forward chains jump by 32c-s and 31c+s steps, the
// backward FP32 chains by 32c+s and 33c-s (chain_jump_a / chain_jump_b).

// The FP64 output chains of the two-chain loop hold Z = z 2^10 (see
// shared_step_f64_ptx).  In runs of compile-time depth some iterations take
// their conversion on the FP64 pipe, alternating between chain a (iteration
// 0 of every K) and chain b (iteration K/2): int->double and one
// round-to-nearest multiply, the definition itself, instead of the integer
// rounding.  The FP64 pipe is otherwise idle here.  One-variate runs (odd
// depths) take K = 8, an eighth of the conversions (787 G variates/s in a
// test kernel against 787 for a sixth, 785 for a quarter and 771 for a
// third); two-variate runs (depths of 2 mod 4) take K = 6 (812 against 808
// for an eighth).  Same bits either way.
constexpr uint32_t kFp64ConvEvery = 8, kFp64ConvEveryVec2 = 6;
__device__ __forceinline__ uint64_t fp64_conv_step_scaled(uint64_t& Z) {
  const uint64_t bits = f64_bits_fp64_scaled(Z);
  Z = shared_advance_scaled(Z);
  return bits;
}

// One fast step's FP64 bits from a scaled chain; `fp64` takes the conversion
// on the FP64 pipe.
__device__ __forceinline__ uint64_t fast_word(uint64_t& Z, uint32_t& qmin, bool fp64) {
  if (fp64) return fp64_conv_step_scaled(Z);
  return shared_step_f64_ptx(Z, qmin);
}

// The two interleaved scaled chains of the branch-free shared-quotient step
// over one run of FP64 output, split at s = chain_split(c); a lane that left
// the fast path redoes its run with one exact chain on z.  Depths of 2 mod 4
// (compile-time) store two variates at a time: each lane's run then starts
// 16-byte aligned and the eight lanes of each 16-byte store phase hit
// distinct bank groups (c/2 odd); 30-deep runs split 16/14 this way measured
// 808 against 789 G variates/s for 31-deep one-variate runs in a test kernel.
template <int CDEPTH>
__device__ __forceinline__ void shared_run_fast2(uint64_t* mine, uint32_t c, uint64_t& za,
                                                 uint64_t& zb) {
  const uint64_t a_start = za;
  uint32_t qmin = 0xffffffffu;
  if constexpr (CDEPTH > 0 && vec2_depth(CDEPTH)) {
    constexpr int S = (int)chain_split(CDEPTH), GA = S / 2, GB = (CDEPTH - S) / 2;
    constexpr int G = GA > GB ? GA : GB;
    constexpr int K = (int)kFp64ConvEveryVec2;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      uint64_t va[2], vb[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int i = 2 * g + k;
        if (g < GA) va[k] = fast_word(za, qmin, i % K == 0);
        if (g < GB) vb[k] = fast_word(zb, qmin, i % K == K / 2);
      }
      if (g < GA)
        *reinterpret_cast<uint4*>(mine + 2 * g) =
            make_uint4((uint32_t)va[0], (uint32_t)(va[0] >> 32), (uint32_t)va[1],
                       (uint32_t)(va[1] >> 32));
      if (g < GB)
        *reinterpret_cast<uint4*>(mine + S + 2 * g) =
            make_uint4((uint32_t)vb[0], (uint32_t)(vb[0] >> 32), (uint32_t)vb[1],
                       (uint32_t)(vb[1] >> 32));
    }
  } else {
    const uint32_t cc = CDEPTH > 0 ? (uint32_t)CDEPTH : c;
    const uint32_t s = chain_split(cc), nb = cc - s;  // nb <= s
    constexpr uint32_t K = kFp64ConvEvery;
#pragma unroll
    for (uint32_t i = 0; i < nb; ++i) {
      mine[i] = fast_word(za, qmin, CDEPTH > 0 && i % K == 0);
      mine[s + i] = fast_word(zb, qmin, CDEPTH > 0 && i % K == K / 2);
    }
    for (uint32_t i = nb; i < s; ++i) mine[i] = fast_word(za, qmin, false);
  }
  const bool rare = qmin == 0;
  if (__any_sync(0xffffffffu, rare)) {
    if (rare) {
      const uint32_t cc = CDEPTH > 0 ? (uint32_t)CDEPTH : c;
      uint64_t y = a_start >> kZShift;
      for (uint32_t i = 0; i < cc; ++i) mine[i] = shared_step_f64(y);
    }
    __syncwarp();
  }
}

// FP32 output by the backward step with its exact quotient (two chains on
// y = z - 1): with s = chain_split(c), chain b starts one past the run and
// emits elements c-1 .. s, chain a starts at element s and emits s-1 .. 0, so
// afterwards chain a holds element 0 and chain b element s.  Every conversion
// stays on the integer pipes (taking one in six or twelve on the FP64 pipe, as
// the forward FP64 kernel does, measured 1% slower or no faster with this
// step).  Depths of 4 mod 8 (compile-time) store four variates at a time:
// each lane's run then starts 16-byte aligned, and the eight lanes of each
// 16-byte store phase hit distinct bank groups (c/4 odd); the two chains hold
// whole groups of four (for c = 44: 24 and 20 elements).  A lane whose run
// needs the exact path (see back_step_f32_ptx) redoes it forward from
// element 0.
// Element jumps of the warp's shared FP32 redo: element i of a run is
// z_0 2^(53 i) mod m (Eq. 3 applied i times), with each multiplier's
// precomputed quotient, for i up to the largest tile depth.
struct ElemJump {
  uint64_t j[kMaxDepth + 1], q[kMaxDepth + 1];
};
constexpr ElemJump make_elem_jump() {
  ElemJump t{};
  for (uint64_t i = 0; i <= kMaxDepth; ++i) {
    t.j[i] = host_pow2((53ull * i) % kP);
    t.q[i] = host_mulmod_quotient(t.j[i]);
  }
  return t;
}
static __device__ const ElemJump kElemJump = make_elem_jump();
static_assert(make_elem_jump().j[0] == 1 && make_elem_jump().j[1] == host_pow2(53) &&
                  make_elem_jump().j[kMaxDepth] == host_pow2(53ull * kMaxDepth),
              "element jumps");

// The warp's exact redo of flagged FP32 runs of c elements: for each lane
// whose bit is set in `redo`, lane l makes elements l, l + 32, ... of that
// lane's run, each from one jump of the run's element 0 (`z0`, the state of
// that element, taken from its lane), with the forward step and the exact
// conversion.  Made by its own lane alone, a redo held the other 31 lanes
// for a whole run.
__device__ __forceinline__ void warp_redo_runs_f32(uint32_t* mine, uint32_t c, uint64_t z0,
                                                   uint32_t redo) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t* const wbuf = mine - lane * c;  // the warp's tile
  __syncwarp();  // every lane's run is in shared memory before others overwrite it
  while (redo != 0) {
    const int L = __ffs(redo) - 1;
    redo &= redo - 1;
    const uint64_t zl = __shfl_sync(0xffffffffu, z0, L);
    for (uint32_t i = lane; i < c; i += 32) {
      uint64_t z = mulmod_pre(zl, __ldg(&kElemJump.j[i]), __ldg(&kElemJump.q[i]));
      wbuf[L * c + i] = f32_bits_from_f64_bits(shared_step_f64(z));
    }
  }
  __syncwarp();
}

template <int CDEPTH>
__device__ __forceinline__ void back_run_f32(uint32_t* mine, uint32_t c, uint64_t& ya,
                                             uint64_t& yb) {
  uint32_t qmin = 0xffffffffu;
  if constexpr (CDEPTH > 0 && vec4_depth(CDEPTH)) {
    constexpr int S = (int)chain_split(CDEPTH), GA = S / 4, GB = (CDEPTH - S) / 4;
    constexpr int G = GA > GB ? GA : GB;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      uint32_t va[4], vb[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (g < GB) vb[k] = back_step_f32_ptx(yb, qmin);
        if (g < GA) va[k] = back_step_f32_ptx(ya, qmin);
      }
      if (g < GB)
        *reinterpret_cast<uint4*>(mine + CDEPTH - 4 * (g + 1)) =
            make_uint4(vb[3], vb[2], vb[1], vb[0]);
      if (g < GA)
        *reinterpret_cast<uint4*>(mine + S - 4 * (g + 1)) = make_uint4(va[3], va[2], va[1], va[0]);
    }
  } else {
    const uint32_t cc = CDEPTH > 0 ? (uint32_t)CDEPTH : c;
    const uint32_t s = chain_split(cc), nb = cc - s;  // nb <= s
#pragma unroll
    for (uint32_t i = 0; i < nb; ++i) {
      mine[cc - 1 - i] = back_step_f32_ptx(yb, qmin);
      mine[s - 1 - i] = back_step_f32_ptx(ya, qmin);
    }
    for (uint32_t i = nb; i < s; ++i) mine[s - 1 - i] = back_step_f32_ptx(ya, qmin);
  }
  // A flagged run is redone exactly by the whole warp (the backward chain a
  // ends at the state of the run's element 0).
  const uint32_t redo = __ballot_sync(0xffffffffu, qmin == 0);
  if (__builtin_expect(redo != 0, 0))
    warp_redo_runs_f32(mine, CDEPTH > 0 ? (uint32_t)CDEPTH : c, ya + 1, redo);
}

// Whether a two-chain tile loop of this kind runs the backward FP32 step.
template <int DT, int STEP, int CONV>
constexpr bool kBackF32 = DT == DT_F32 && STEP == ST_SHARED && CONV == CV_INT;
// Whether it runs the forward FP64 step on chains scaled by 2^10.
template <int DT, int STEP, int CONV>
constexpr bool kScaledF64 = DT == DT_F64 && STEP == ST_SHARED && CONV == CV_INT;

template <int DT, int STEP, int CONV, int CDEPTH = 0>
__device__ __forceinline__ void warp_tiles2(typename Word<DT>::type* __restrict__ out,
                                            uint64_t first, uint64_t ntiles, uint32_t c_rt,
                                            uint64_t jump_a, uint64_t jump_aq, uint64_t jump_b,
                                            uint64_t jump_bq, Gen<DT, STEP, CONV>& a,
                                            Gen<DT, STEP, CONV>& b,
                                            typename Word<DT>::type* buf0, uint32_t& issued,
                                            uint32_t lane, uint32_t nbuf = 2) {
  typedef typename Word<DT>::type W;
  const uint32_t c = CDEPTH > 0 ? (uint32_t)CDEPTH : c_rt;
  const uint32_t tile_elems = 32u * c;
  const uint32_t tile_bytes = tile_elems * (uint32_t)sizeof(W);
  const uint32_t h = c >> 1;
  for (uint64_t t = 0; t < ntiles; ++t) {
    W* const buf = buf0 + tile_buffer(issued, nbuf) * tile_elems;
    wait_buffer_free(issued, nbuf, lane);
    W* const mine = buf + lane * c;
    if constexpr (kBackF32<DT, STEP, CONV>) {
      back_run_f32<CDEPTH>(reinterpret_cast<uint32_t*>(mine), c, a.z, b.z);
    } else if constexpr (kScaledF64<DT, STEP, CONV>) {
      shared_run_fast2<CDEPTH>(reinterpret_cast<uint64_t*>(mine), c, a.z, b.z);
    } else {
#pragma unroll 4
      for (uint32_t i = 0; i < h; ++i) {
        mine[i] = a.next();
        mine[h + 1 + i] = b.next();
      }
      mine[h] = a.next();
    }
    fence_proxy_async_shared();
    __syncwarp();
    if (lane == 0) {
      bulk_store(out + first + t * tile_elems, buf, tile_bytes);
      bulk_commit();
    }
    ++issued;
    if (t + 1 < ntiles) {
      if constexpr (kBackF32<DT, STEP, CONV>) {  // the chains hold z - 1
        a.z = mulmod_pre(a.z + 1, jump_a, jump_aq) - 1;
        b.z = mulmod_pre(b.z + 1, jump_b, jump_bq) - 1;
      } else if constexpr (kScaledF64<DT, STEP, CONV>) {  // the chains hold z 2^10
        a.z = mulmod_pre(a.z >> kZShift, jump_a, jump_aq) << kZShift;
        b.z = mulmod_pre(b.z >> kZShift, jump_b, jump_bq) << kZShift;
      } else {
        a.z = mulmod_pre(a.z, jump_a, jump_aq);
        b.z = mulmod_pre(b.z, jump_b, jump_bq);
      }
    }
  }
}

// Initial states of the two chains of a lane whose first run starts at
// element `first` (s = chain_split(c)): forward chains at elements first and
// first + s (the FP64 output chains as z 2^10); the backward FP32 chains one
// past elements s - 1 and c - 1, as z - 1.
template <int DT, int STEP, int CONV>
__device__ __forceinline__ void lane_chains2(uint64_t ebase, uint64_t first, uint32_t c,
                                             uint32_t skip, Gen<DT, STEP, CONV>& a,
                                             Gen<DT, STEP, CONV>& b) {
  const uint32_t h = c / 2;
  if constexpr (kBackF32<DT, STEP, CONV>) {
    a.z = state_of(ebase, first + chain_split(c), skip) - 1;
    b.z = state_of(ebase, first + c, skip) - 1;
  } else if constexpr (kScaledF64<DT, STEP, CONV>) {
    a.z = state_of(ebase, first, skip) << kZShift;
    b.z = state_of(ebase, first + chain_split(c), skip) << kZShift;
  } else {
    a.z = state_of(ebase, first, skip);
    b.z = state_of(ebase, first + h + 1, skip);
  }
}

// Initial chain state for a lane whose run starts at element `first` of a
// call with exponent base ebase (forward chains start at the run's first
// element, the backward Montgomery chain at its last).
template <int DT, int STEP, int CONV>
__device__ __forceinline__ Gen<DT, STEP, CONV> lane_chain(uint64_t ebase, uint64_t first,
                                                          uint32_t c, uint32_t skip) {
  Gen<DT, STEP, CONV> g{0};
  if constexpr (STEP == ST_MONT) g.z = state_of(ebase, first + c - 1, skip);
  else if constexpr (STEP != ST_CONST) g.z = state_of(ebase, first, skip);
  return g;
}

}  // namespace bcn
