"""Seeded synthetic inputs for every workload.

This module holds no arithmetic of the generator: it only draws seeds
(start indices), lengths, element types and arrival times with numpy's PCG64,
so both the CUDA path and the oracle can be fed the same inputs.  Shapes
follow the paper's workloads ("generate n uniforms from a start index") at
the sizes the benchmarks use.
"""
from __future__ import annotations

import numpy as np

M = 3 ** 33
SEED_MIN = M + 100          # Algorithm BB, step 1
SEED_MAX = 2 ** 53


def batch_streams(nstreams: int = 4096, seed: int = 7, len_lo: float = 1e3,
                  len_hi: float = 1e7, start_hi: int = 2 ** 53 - 10 ** 8):
    """Batched workload: start indices uniform in [3^33+100, start_hi], lengths
    log-uniform in [len_lo, len_hi] (rounded), FP64 for even stream ids and
    FP32 for odd ones."""
    g = np.random.default_rng(seed)
    starts = g.integers(SEED_MIN, start_hi, size=nstreams, endpoint=True, dtype=np.uint64)
    lengths = np.rint(10.0 ** g.uniform(np.log10(len_lo), np.log10(len_hi), size=nstreams))
    lengths = lengths.astype(np.uint64)
    dtypes = ["f64" if i % 2 == 0 else "f32" for i in range(nstreams)]
    return starts, lengths, dtypes


def small_batch(nstreams: int = 200, seed: int = 3, max_len: int = 20000):
    """A parity-sized batch with empty, tiny and ragged streams and all three
    element types."""
    g = np.random.default_rng(seed)
    starts = g.integers(SEED_MIN, SEED_MAX, size=nstreams, endpoint=True, dtype=np.uint64)
    lengths = g.integers(0, max_len, size=nstreams, dtype=np.uint64)
    lengths[:8] = [0, 1, 2, 3, 4, 5, 31, 33]
    offsets = g.integers(0, 2 ** 50, size=nstreams, dtype=np.uint64)
    kinds = ["f64", "f32", "u64"]
    dtypes = [kinds[int(k)] for k in g.integers(0, 3, size=nstreams)]
    return starts, offsets, lengths, dtypes


def request_trace(n_requests: int, rate_hz: float = 20000.0, seed: int = 11,
                  min_bytes: int = 1 << 10, max_bytes: int = 256 << 20):
    """Serving workload: Poisson arrivals at `rate_hz`, request sizes
    log-uniform in [min_bytes, max_bytes], random start indices and offsets,
    FP32 and FP64 mixed 1:1.  Returns arrival times (s), element counts,
    dtypes, seeds and offsets."""
    g = np.random.default_rng(seed)
    gaps = g.exponential(1.0 / rate_hz, size=n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    nbytes = np.rint(2.0 ** g.uniform(np.log2(min_bytes), np.log2(max_bytes), size=n_requests))
    dtypes = ["f64" if k == 0 else "f32" for k in g.integers(0, 2, size=n_requests)]
    esz = np.array([8 if d == "f64" else 4 for d in dtypes], dtype=np.int64)
    counts = np.maximum(1, nbytes.astype(np.int64) // esz).astype(np.uint64)
    seeds = g.integers(SEED_MIN, SEED_MAX, size=n_requests, endpoint=True, dtype=np.uint64)
    offsets = g.integers(0, 2 ** 40, size=n_requests, dtype=np.uint64)
    return arrivals, counts, dtypes, seeds, offsets
