// bcn_pool.cu -- C ABI over the output-pool sub-allocator (bcn_pool.h), so
// the allocator the serving loop admits requests with can be driven and
// checked on its own.
#include <mutex>
#include <new>

#include "bcn_internal.h"
#include "bcn_pool.h"


struct bcn_pool {
  bcn::Pool pool;
  std::mutex mu;
  bcn_pool(uint64_t cap, uint64_t al) : pool(cap, al) {}
};

using namespace bcn;

extern "C" {

rng_status rng_pool_create(uint64_t capacity, uint64_t align, bcn_pool** out) {
  if (!out) return set_error(RNG_EINVAL, "out is NULL");
  *out = nullptr;
  if (capacity == 0) return set_error(RNG_EINVAL, "capacity must be > 0");
  if (align == 0 || (align & (align - 1)) != 0)
    return set_error(RNG_EINVAL, "align must be a power of two");
  bcn_pool* p = new (std::nothrow) bcn_pool(capacity, align);
  if (!p) return set_error(RNG_ENOMEM, "out of host memory");
  *out = p;
  return RNG_OK;
}

rng_status rng_pool_alloc(bcn_pool* p, uint64_t bytes, uint64_t* offset) {
  if (!p || !offset) return set_error(RNG_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(p->mu);
  if (!p->pool.alloc(bytes, offset))
    return set_error(RNG_ENOMEM, "no free range of %llu bytes", (unsigned long long)bytes);
  return RNG_OK;
}

rng_status rng_pool_free(bcn_pool* p, uint64_t offset) {
  if (!p) return set_error(RNG_EINVAL, "NULL pool");
  std::lock_guard<std::mutex> lock(p->mu);
  if (!p->pool.release(offset))
    return set_error(RNG_EINVAL, "offset %llu is not a live allocation",
                     (unsigned long long)offset);
  return RNG_OK;
}

rng_status rng_pool_stats(bcn_pool* p, uint64_t* in_use, uint64_t* peak, uint64_t* live,
                          uint64_t* largest_free, uint64_t* free_ranges) {
  if (!p) return set_error(RNG_EINVAL, "NULL pool");
  std::lock_guard<std::mutex> lock(p->mu);
  if (in_use) *in_use = p->pool.in_use;
  if (peak) *peak = p->pool.peak;
  if (live) *live = p->pool.live;
  if (largest_free) *largest_free = p->pool.largest_free();
  if (free_ranges) *free_ranges = p->pool.free_by_off.size();
  return RNG_OK;
}

rng_status rng_pool_destroy(bcn_pool* p) {
  delete p;
  return RNG_OK;
}

}  // extern "C"
