"""GPU parity of the batched persistent kernel against the oracle.

Every stream of a batch must equal the oracle's variates for its own seed and
offset, bit for bit, whatever the tile depth, block, work-unit size or step
variant, whether launched directly or replayed as a CUDA graph, and the bytes
between streams must stay untouched.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M = 3 ** 33
ESZ = {"f64": 8, "f32": 4, "u64": 8}
TDT = None


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_1187_gb300 import rng
    return rng


def _tdt(d):
    import torch
    return {"f64": torch.float64, "f32": torch.float32, "u64": torch.uint64}[d]


def _bits(a: np.ndarray) -> np.ndarray:
    return a.view(np.int64 if a.itemsize == 8 else np.int32)


def _dev_bits(t):
    import torch
    return t.view(torch.int64 if t.element_size() == 8 else torch.int32).cpu().numpy()


def _pool_outputs(counts, dtypes, rnd):
    """Carve every stream's output from one byte pool, at element-aligned but
    otherwise random offsets, with gaps filled by a canary byte."""
    import torch
    offs, pos = [], 64
    for c, d in zip(counts, dtypes):
        e = ESZ[d]
        pos = (pos + e - 1) // e * e + e * int(rnd.integers(0, 4))
        offs.append(pos)
        pos += int(c) * e + 24
    pool = torch.full((pos + 64,), 0xA5, dtype=torch.uint8, device="cuda")
    outs = []
    for o, c, d in zip(offs, counts, dtypes):
        outs.append(pool[o: o + int(c) * ESZ[d]].view(_tdt(d)))
    return pool, offs, outs


def test_small_batch_every_stream_exact(R, oracle_mod):
    from paper_1206_1187_gb300 import inputs
    starts, offsets, counts, dtypes = inputs.small_batch()
    rnd = np.random.default_rng(5)
    pool, offs, outs = _pool_outputs(counts, dtypes, rnd)
    b = R.Batch(starts, counts, dtypes, outs=outs, offsets=offsets)
    b.launch()
    host = pool.cpu().numpy()
    covered = np.zeros(host.size, dtype=bool)
    for s in range(len(starts)):
        n, d = int(counts[s]), dtypes[s]
        want = oracle_mod.generate(int(starts[s]), int(offsets[s]), n, d)
        got = host[offs[s]: offs[s] + n * ESZ[d]].view(want.dtype)
        assert np.array_equal(_bits(got.copy()), _bits(want)), (s, n, d)
        covered[offs[s]: offs[s] + n * ESZ[d]] = True
    assert np.all(host[~covered] == 0xA5), "bytes outside the streams were written"


def test_tuning_and_graph_never_change_the_bytes(R):
    import torch
    from paper_1206_1187_gb300 import inputs
    starts, offsets, counts, dtypes = inputs.small_batch(nstreams=120, seed=9, max_len=60000)
    rnd = np.random.default_rng(6)
    ref_pool = None
    for tune in [None, dict(depth=1, block=32, unit=1), dict(depth=7, block=128, unit=3),
                 dict(depth=31, block=256, unit=64, step="barrett"),
                 dict(depth=15, block=512, unit=2, step="montgomery"),
                 dict(depth=9, block=64, unit=5, grid=3, skip="sqmul"),
                 dict(depth=15, block=256, unit=16, conv="fp64"),
                 dict(depth=15, block=128, unit=8, chains=1),
                 dict(depth=31, block=128, unit=4, chains=2),
                 dict(depth=21, block=64, unit=3, chains=2, step="barrett"),
                 dict(depth=31, block=896, unit=4, chains=2, buffers=1),
                 dict(depth=15, block=64, unit=5, chains=1, buffers=1),
                 dict(depth=9, block=96, unit=2, chains=2, buffers=1, step="barrett")]:
        pool, offs, outs = _pool_outputs(counts, dtypes, np.random.default_rng(6))
        b = R.Batch(starts, counts, dtypes, outs=outs, offsets=offsets, tune=tune)
        b.launch()
        if ref_pool is None:
            ref_pool = pool.clone()
        else:
            assert torch.equal(pool, ref_pool), tune
        pool.fill_(0xA5)
        b.graph_launch()
        b.graph_launch()
        assert torch.equal(pool, ref_pool), ("graph", tune)
        b.close()


def test_batch_rejects_bad_streams(R):
    import torch
    out = torch.empty(10, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RNGError) as e:
        R.Batch([M + 99], [10], ["f64"], outs=[out])
    assert e.value.status == 2
    with pytest.raises(R.RNGError) as e:
        R.Batch([M + 100], [10], ["f64"], outs=[out], tune=dict(depth=4))
    assert e.value.status == 1
    with pytest.raises(R.RNGError) as e:
        R.Batch([M + 100], [10], ["f64"], outs=[out], tune=dict(buffers=3))
    assert e.value.status == 1


@pytest.mark.slow
def test_4096_stream_batch_in_a_graph(R, oracle_mod):
    """The batched workload: 4096 streams, seeds from numpy default_rng(7)
    in [3^33+100, 2^53-10^8], lengths log-uniform 10^3..10^7, FP64/FP32
    alternating, one persistent launch replayed as a CUDA graph.  Short
    streams are compared whole; every 32nd long stream on its first and last
    2048 variates and 2048 random positions."""
    import torch
    from paper_1206_1187_gb300 import inputs
    starts, counts, dtypes = inputs.batch_streams()
    total = int(sum(int(c) * ESZ[d] for c, d in zip(counts, dtypes)))
    outs = [torch.empty(int(c), dtype=_tdt(d), device="cuda") for c, d in zip(counts, dtypes)]
    b = R.Batch(starts, counts, dtypes, outs=outs)
    info = b.info()
    assert info["bytes"] == total and info["elems"] == int(sum(int(c) for c in counts))
    b.graph_launch()
    torch.cuda.synchronize()
    _check_workload(starts, counts, dtypes, outs, oracle_mod)
    # the benchmark's launch: the plan tuning measured on this workload, and the
    # shape it has picked on GB300
    from paper_1206_1187_gb300 import autotune
    best = autotune.tune_batch(workload=(starts, counts, dtypes, outs),
                               tag="batched-4096-seed7")["best"]
    for tune in (best, dict(step="shared", conv="int", depth=31, block=896, unit=64, chains=2,
                            buffers=1)):
        for o in outs:
            o.zero_()
        b2 = R.Batch(starts, counts, dtypes, outs=outs, tune=tune)
        b2.graph_launch()
        torch.cuda.synchronize()
        _check_workload(starts, counts, dtypes, outs, oracle_mod)
        b2.close()


def _check_workload(starts, counts, dtypes, outs, oracle_mod):
    import torch
    rnd = np.random.default_rng(8)
    for s in range(len(starts)):
        n, d, a = int(counts[s]), dtypes[s], int(starts[s])
        if n <= 20000:
            assert np.array_equal(_dev_bits(outs[s]), _bits(oracle_mod.generate(a, 0, n, d))), s
        elif s % 32 == 0:
            idx = np.unique(np.concatenate([np.arange(2048), np.arange(n - 2048, n),
                                            rnd.integers(0, n, size=2048)])).astype(np.int64)
            got = _dev_bits(outs[s][torch.from_numpy(idx).cuda()])
            want = _bits(oracle_mod.at(a, idx.astype(np.uint64), d))
            assert np.array_equal(got, want), s
