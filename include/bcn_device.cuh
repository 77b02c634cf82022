// bcn_device.cuh -- the alpha_{2,3} generator as a device-side object for your
// own kernels: a 64-bit state per thread, positioned anywhere in a sequence by
// skip-ahead, producing the same variates as the library's bulk calls.
//
// The paper points out the generator's advantage for simulations running on
// the GPU: independent subsequences per thread with only a 64-bit state and no
// shared memory (Sec. 2).  Typical use:
//
//   #include "bcn_device.cuh"
//   __global__ void sim(uint64_t seed, ...) {
//     bcn_device::Stream g = bcn_device::make_stream(seed, my_first_variate);
//     for (...) { double u = bcn_device::next_f64(g); ... }
//     float w[32];                      // or 32 floats at a time, from one product:
//     bcn_device::f32_run<32>(seed, my_first_float, w);
//   }
//
// Variate i of the sequence seeded with start index a (Algorithm BB) is
// RN(z * r3i) for z = 2^((a - 3^33 + 53*(i+1)) mod P) * floor(3^33/2) mod 3^33,
// exactly as rng_generate_at writes it, so results do not depend on how the
// work is split over threads.  Compile with nvcc for sm_103a with this
// directory on the include path.  The start index must satisfy Algorithm BB,
// step 1 (3^33+100 <= a <= 2^53); nothing is checked on the device.
#pragma once
#include <cstdint>
#include <utility>

#include "bcn_digits_math.cuh"
#include "bcn_math.cuh"

namespace bcn_device {

struct Stream {
  uint64_t Z;  // state of the next variate times 2^10 (the bulk kernels' scaled chain)
};

// A generator positioned at variate `offset` (0-based) of the sequence seeded
// with `start_index`: one fixed-base exponentiation (six modular products).
// Every 64-bit offset is exact (the sequence continues past 2^64 - 1).
__device__ inline Stream make_stream(uint64_t start_index, uint64_t offset) {
  const uint64_t e0 = (start_index - bcn::kM) % bcn::kP;
  Stream s;
  s.Z = bcn::seed_state_table(bcn::exponent_add(bcn::exponent_add(e0, offset), 1))
        << bcn::kZShift;
  return s;
}

// The generator at variate offset + extra, the sum taken without 64-bit
// wrap-around (a thread's start inside a call that began at `offset`).
__device__ inline Stream make_stream(uint64_t start_index, uint64_t offset, uint64_t extra) {
  const uint64_t e0 = (start_index - bcn::kM) % bcn::kP;
  Stream s;
  s.Z = bcn::seed_state_table(
            bcn::exponent_add(bcn::exponent_add(bcn::exponent_add(e0, offset), extra), 1))
        << bcn::kZShift;
  return s;
}

// The FP64 bits of the next variate, RN(z * r3i), and the step to the one
// after: the bulk kernels' shared-quotient step on the scaled state, with the
// exact conversion for the rare variate below 2^-21 that its fast rounding
// does not cover (the state advance is exact either way).
__device__ inline uint64_t next_bits(Stream& s) {
  const uint64_t Z0 = s.Z;
  uint32_t qmin = 0xffffffffu;
  uint64_t bits = bcn::shared_step_f64_ptx(s.Z, qmin);
  if (__builtin_expect(qmin == 0, 0)) {
    uint64_t z = Z0 >> bcn::kZShift;
    bits = bcn::shared_step_f64(z);
  }
  return bits;
}

// The next variate as a double in (0,1): RN(z * r3i), exactly.
__device__ inline double next_f64(Stream& s) {
  return __longlong_as_double((long long)next_bits(s));
}

// The next variate as a float in (0,1): the double variate rounded toward zero.
__device__ inline float next_f32(Stream& s) {
  return __uint_as_float(bcn::f32_bits_from_f64_bits(next_bits(s)));
}

// The next raw state z in [1, 3^33).
__device__ inline uint64_t next_state(Stream& s) {
  const uint64_t z = s.Z >> bcn::kZShift;
  s.Z = bcn::shared_advance_scaled(s.Z);
  return z;
}

namespace detail {
template <int C, int I>
__device__ __forceinline__ void f32_run_word(uint32_t z0, uint32_t z1,
                                             uint32_t (&r)[bcn::DigitGeometry<C>::W],
                                             uint32_t& v0, uint32_t& v1, float (&v)[C],
                                             uint32_t& qmin) {
  bcn::run_product_word<bcn::DigitGeometry<C>::W, I>(z0, z1, r[I], v0, v1);
  constexpr int i = bcn::DigitGeometry<C>::digit_of_word(I);
  if constexpr (i >= 0)
    v[C - 1 - i] = __uint_as_float(bcn::f32_from_digit_words(
        bcn::run_bits32<53 * i + 21>(r), bcn::run_bits32<53 * i - 11>(r), qmin));
}
template <int C, int... I>
__device__ __forceinline__ void f32_run_words(std::integer_sequence<int, I...>, uint64_t z,
                                              float (&v)[C], uint32_t& qmin) {
  const uint32_t z0 = (uint32_t)z, z1 = (uint32_t)(z >> 32);
  uint32_t r[bcn::DigitGeometry<C>::W];
  uint32_t v0 = 0, v1 = 0;
  (f32_run_word<C, I>(z0, z1, r, v0, v1, v, qmin), ...);
}
}  // namespace detail

// C consecutive FP32 variates, elements offset + extra .. offset + extra +
// C - 1 of the sequence seeded with start_index (the sum taken without
// 64-bit wrap-around), into v[0..C): the same values as C calls of next_f32,
// made together from one product of the state one past them
// (bcn_digits_math.cuh): measured 28.8 instructions a variate in runs of 32,
// the skip-ahead of each run included, against 42.2 for next_f64 one call at
// a time.  C is a compile-time constant; v is meant to stay in registers.  One skip-ahead per call; a run holding a digit that may round
// up or a variate below 2^-20 (about C in 2^16 runs) is made again exactly.
template <int C>
__device__ inline void f32_run(uint64_t start_index, uint64_t offset, uint64_t extra,
                               float (&v)[C]) {
  const uint64_t e0 = (start_index - bcn::kM) % bcn::kP;
  const uint64_t e = bcn::exponent_add(bcn::exponent_add(e0, offset), extra);
  const uint64_t z = bcn::seed_state_table(bcn::exponent_add(e, C + 1));  // one past the run
  uint32_t qmin = 0xffffffffu;
  detail::f32_run_words<C>(std::make_integer_sequence<int, bcn::DigitGeometry<C>::W>{}, z, v,
                           qmin);
  if (__builtin_expect(qmin == 0, 0)) {
    Stream s;
    s.Z = bcn::seed_state_table(bcn::exponent_add(e, 1)) << bcn::kZShift;  // the run's first
    for (int i = 0; i < C; ++i) v[i] = next_f32(s);
  }
}

template <int C>
__device__ inline void f32_run(uint64_t start_index, uint64_t offset, float (&v)[C]) {
  f32_run<C>(start_index, offset, 0, v);
}

}  // namespace bcn_device
