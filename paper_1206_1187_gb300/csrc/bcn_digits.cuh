// bcn_digits.cuh -- the library's FP32 runs made from one product each
// (sm_103a): a tile lane's run of C variates from the state one past the run
// (the arithmetic, with its derivation, is in bcn_digits_math.cuh).
#pragma once
#include <utility>

#include "bcn_digits_math.cuh"
#include "bcn_gen.cuh"

namespace bcn {

// An FP32 run of C elements (C of 4 mod 8, four-variate shared-memory stores
// as in back_run_f32) from the state one past the run, z = s_(f+C): field i
// of z N mod 2^(53C) is the digit of element C - 1 - i.  Words are formed
// from the bottom and each digit is converted once its top word exists, so
// only a few words are live at a time.  A run that needs the exact path is
// redone by the warp from the state of its element 0, z 2^(-53C) mod m.
template <int C>
struct DigitRunF32 : DigitGeometry<C> {
  static constexpr uint64_t back = host_pow2((kP - (53ull * C) % kP) % kP);  // 2^(-53C)
  static constexpr uint64_t back_q = host_mulmod_quotient(back);
};

template <int C, int I>
__device__ __forceinline__ void digit_run_word(uint32_t z0, uint32_t z1,
                                               uint32_t (&r)[DigitRunF32<C>::W], uint32_t& v0,
                                               uint32_t& v1, uint32_t (&d)[4], uint32_t* mine,
                                               uint32_t& qmin) {
  run_product_word<DigitRunF32<C>::W, I>(z0, z1, r[I], v0, v1);
  constexpr int i = DigitRunF32<C>::digit_of_word(I);
  if constexpr (i >= 0) {
    // X = Q 2^11 for digit i: bits [53i - 11, 53i + 53) of the product
    const uint32_t u1 = run_bits32<53 * i + 21>(r);
    const uint32_t u0 = run_bits32<53 * i - 11>(r);
    d[i % 4] = f32_from_digit_words(u1, u0, qmin);
    if constexpr (i % 4 == 3)  // elements C - 4(i/4 + 1) .. C - 1 - 4(i/4)
      *reinterpret_cast<uint4*>(mine + C - 4 * (i / 4 + 1)) = make_uint4(d[3], d[2], d[1], d[0]);
  }
}

template <int C, int... I>
__device__ __forceinline__ void digit_run_words(std::integer_sequence<int, I...>, uint64_t z,
                                                uint32_t* mine, uint32_t& qmin) {
  const uint32_t z0 = (uint32_t)z, z1 = (uint32_t)(z >> 32);
  uint32_t r[DigitRunF32<C>::W];
  uint32_t v0 = 0, v1 = 0, d[4];
  (digit_run_word<C, I>(z0, z1, r, v0, v1, d, mine, qmin), ...);
}

template <int C>
__device__ __forceinline__ void digit_run_f32(uint32_t* mine, uint64_t z) {
  static_assert(vec4_depth(C), "runs of 4 mod 8 (four-variate stores)");
  uint32_t qmin = 0xffffffffu;
  digit_run_words<C>(std::make_integer_sequence<int, DigitRunF32<C>::W>{}, z, mine, qmin);
  const uint32_t redo = __ballot_sync(0xffffffffu, qmin == 0);
  if (__builtin_expect(redo != 0, 0))
    warp_redo_runs_f32(mine, C, mulmod_pre(z, DigitRunF32<C>::back, DigitRunF32<C>::back_q),
                       redo);
}

// Whether a one-chain tile loop of this kind makes its FP32 runs this way
// (compile-time depths of 4 mod 8).
template <int DT, int STEP, int CONV, int CDEPTH>
constexpr bool kDigitsF32 = DT == DT_F32 && STEP == ST_SHARED && CONV == CV_INT && CDEPTH > 0 &&
                            vec4_depth(CDEPTH);

// warp_tiles for these runs: `ntiles` consecutive tiles of 32C elements, the
// first at element `first` of `out`; z is the state one past this lane's run
// in the first tile, and `jump` = 2^(53*32C) moves it to the next tile.
template <int C>
__device__ __forceinline__ void warp_tiles_digits(uint32_t* __restrict__ out, uint64_t first,
                                                  uint64_t ntiles, uint64_t jump, uint64_t jump_q,
                                                  uint64_t z, uint32_t* buf0, uint32_t& issued,
                                                  uint32_t lane, uint32_t nbuf) {
  constexpr uint32_t tile_elems = 32u * C;
  constexpr uint32_t tile_bytes = tile_elems * 4u;
  for (uint64_t t = 0; t < ntiles; ++t) {
    uint32_t* const buf = buf0 + tile_buffer(issued, nbuf) * tile_elems;
    wait_buffer_free(issued, nbuf, lane);
    digit_run_f32<C>(buf + lane * C, z);
    fence_proxy_async_shared();
    __syncwarp();
    if (lane == 0) {
      bulk_store(out + first + t * tile_elems, buf, tile_bytes);
      bulk_commit();
    }
    ++issued;
    if (t + 1 < ntiles) z = mulmod_pre(z, jump, jump_q);
  }
}

}  // namespace bcn
