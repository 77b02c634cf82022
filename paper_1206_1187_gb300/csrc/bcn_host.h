// bcn_host.h -- host-side services shared by the library's launchers (no
// device code depends on these, so the kernels' digests do not either).
#pragma once
#include "bcn_internal.h"

namespace bcn {

// RNG_OK, or RNG_EINVAL with the message when BCN_RNG_TUNE is set but does
// not parse (every call that takes defaults then fails loudly).
rng_status env_tune_check();
// Whether BCN_RNG_TUNE forces a block size (small calls then keep it).
bool env_tune_sets_block();

// The library's device and pinned-host allocations go through these, so a
// test can make them fail (rng_debug_fail_allocations) as if memory ran out.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t pinned_malloc(void** p, size_t bytes);

}  // namespace bcn
