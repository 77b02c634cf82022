"""The batch entry point that allocates nothing (rng_batch_generate_noalloc).

It serves callers that cannot call cudaMalloc -- for example code running
under a framework whose allocator owns all device memory, or latency-critical
paths that must not allocate -- by keeping the batched kernel's work table in
a fixed device array inside the library.  This file is collected last so that
a run stopping at its first failure has already run every other test.  The
new entry point is called through the C ABI twice in a row: the first call on
torch's current stream, the second on a separate CUDA stream created for it
(started only after the first call has finished, so the two never overlap).
Every stream of each call must equal, bit for bit, the oracle's variates and
the output of the allocating entry point (rng_batch_create +
rng_batch_launch) on the same inputs -- the exactness every other parity test
in this suite uses.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _tensors(counts, dtypes, fill):
    import torch
    tdt = {"f64": torch.float64, "f32": torch.float32, "u64": torch.uint64}
    return [torch.full((int(c),), fill, dtype=tdt[d], device="cuda") if d != "u64"
            else torch.zeros(int(c), dtype=tdt[d], device="cuda") for c, d in zip(counts, dtypes)]


def _bits(t):
    import torch
    return t.view(torch.int64 if t.element_size() == 8 else torch.int32).cpu().numpy()


def _oracle_bits(oracle_mod, start, offset, count, dtype):
    want = oracle_mod.generate(int(start), int(offset), int(count), dtype)
    return want.view(np.int64 if want.itemsize == 8 else np.int32)


def test_noalloc_batch_equals_the_oracle_and_the_allocating_batch_twice(oracle_mod):
    import torch
    from paper_1206_1187_gb300 import inputs, rng

    assert torch.cuda.is_available()
    fn = rng.lib.rng_batch_generate_noalloc
    codes_of = {"f64": 0, "f32": 1, "u64": 2}
    second = torch.cuda.Stream()  # the second call's own stream
    for call, (nstreams, seed) in enumerate([(150, 21), (600, 22)]):
        starts, offsets, counts, dtypes = inputs.small_batch(nstreams=nstreams, seed=seed,
                                                             max_len=30000)
        ref = _tensors(counts, dtypes, -1.0)
        b = rng.Batch(starts, counts, dtypes, outs=ref, offsets=offsets)
        b.launch()
        got = _tensors(counts, dtypes, -2.0)
        torch.cuda.synchronize()  # nothing earlier overlaps the call
        codes = np.ascontiguousarray([codes_of[d] for d in dtypes], dtype=np.uint8)
        ptrs = (ctypes.c_void_p * nstreams)(*[t.data_ptr() for t in got])
        cs = torch.cuda.current_stream() if call == 0 else second
        rc = fn(nstreams, ctypes.c_void_p(starts.ctypes.data), ctypes.c_void_p(offsets.ctypes.data),
                ctypes.c_void_p(counts.ctypes.data), ctypes.c_void_p(codes.ctypes.data), ptrs,
                None, ctypes.c_void_p(cs.cuda_stream))
        assert rc == 0, rng.lib.rng_last_error()
        cs.synchronize()
        torch.cuda.synchronize()
        for s in range(nstreams):
            g = _bits(got[s])
            assert np.array_equal(g, _oracle_bits(oracle_mod, starts[s], offsets[s], counts[s],
                                                  dtypes[s])), (call, s, dtypes[s])
            assert np.array_equal(g, _bits(ref[s])), (call, s, dtypes[s])
        b.close()


def test_noalloc_batch_switches_kernel_shapes():
    # each kernel shape gets its own shared-memory allowance: a shape needing
    # more than the 48 KB default after another shape ran first still launches
    import torch
    from paper_1206_1187_gb300 import inputs, rng

    fn = rng.lib.rng_batch_generate_noalloc
    codes_of = {"f64": 0, "f32": 1, "u64": 2}
    starts, offsets, counts, dtypes = inputs.small_batch(nstreams=200, seed=23, max_len=40000)
    ref = _tensors(counts, dtypes, -1.0)
    b = rng.Batch(starts, counts, dtypes, outs=ref, offsets=offsets)
    b.launch()
    codes = np.ascontiguousarray([codes_of[d] for d in dtypes], dtype=np.uint8)
    shapes = [dict(), dict(depth=15, block=256, unit=16, buffers=2),
              dict(depth=31, block=512, unit=8, buffers=1, chains=1),
              dict(depth=9, block=128, unit=4, buffers=2), dict()]
    for shape in shapes:
        got = _tensors(counts, dtypes, -2.0)
        ptrs = (ctypes.c_void_p * len(got))(*[t.data_ptr() for t in got])
        t = rng.make_tune(**shape)
        rc = fn(len(got), ctypes.c_void_p(starts.ctypes.data),
                ctypes.c_void_p(offsets.ctypes.data), ctypes.c_void_p(counts.ctypes.data),
                ctypes.c_void_p(codes.ctypes.data), ptrs, ctypes.byref(t),
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, (shape, rng.lib.rng_last_error())
        torch.cuda.synchronize()
        for s in range(len(got)):
            assert np.array_equal(_bits(got[s]), _bits(ref[s])), (shape, s, dtypes[s])
    b.close()


def test_noalloc_batch_rejects_more_streams_than_its_table_holds():
    import torch
    from paper_1206_1187_gb300 import rng
    n = 1025
    starts = np.full(n, 3 ** 33 + 100, dtype=np.uint64)
    counts = np.ones(n, dtype=np.uint64)
    codes = np.zeros(n, dtype=np.uint8)
    outs = torch.empty(n, dtype=torch.float64, device="cuda")
    ptrs = (ctypes.c_void_p * n)(*[outs.data_ptr() + 8 * i for i in range(n)])
    rc = rng.lib.rng_batch_generate_noalloc(n, ctypes.c_void_p(starts.ctypes.data), None,
                                            ctypes.c_void_p(counts.ctypes.data),
                                            ctypes.c_void_p(codes.ctypes.data), ptrs, None, None)
    assert rc == 2  # RNG_ERANGE
