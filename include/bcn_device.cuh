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

}  // namespace bcn_device
