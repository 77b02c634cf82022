"""The continuous-batching server on the GPU.

* each request's bytes are the same served alone and served in a mix of
  concurrent requests of uneven size (and equal the oracle's);
* memory-based admission never lets the pool's in-use bytes exceed its size,
  and requests wait rather than fail when it is full;
* bad requests are rejected at submission without disturbing the others;
* a real-time trace replay completes every request with finite latency.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M = 3 ** 33


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_1187_gb300 import rng
    return rng


def _bits(t):
    import torch
    return t.view(torch.int64 if t.element_size() == 8 else torch.int32).cpu().numpy()


def _obits(a):
    return a.view(np.int64 if a.itemsize == 8 else np.int32)


def test_each_result_is_the_same_alone_and_in_the_mix(R, oracle_mod):
    from paper_1206_1187_gb300 import inputs
    arrivals, counts, dtypes, seeds, offsets = inputs.request_trace(
        240, rate_hz=20000.0, seed=5, min_bytes=1 << 10, max_bytes=8 << 20)
    n = len(arrivals)
    alone = []
    srv = R.Server(pool_bytes=64 << 20, chunk_elems=1 << 16)
    for i in range(n):
        rid = srv.submit(int(seeds[i]), int(offsets[i]), int(counts[i]), dtypes[i])
        srv.wait(rid, 30.0)
        alone.append(_bits(srv.read(rid, int(counts[i]), dtypes[i])))
        srv.release(rid)
    srv.close()

    srv = R.Server(pool_bytes=1 << 30, chunk_elems=1 << 16, inflight=3)
    lat, wall = srv.run_trace(arrivals, seeds, counts, dtypes, offsets=offsets, timeout_s=60.0)
    assert np.all(lat > 0) and np.isfinite(lat).all()
    st = srv.stats()
    assert st["completed"] == n
    assert st["max_items_seen"] > 1  # iterations carried several requests' chunks at once
    for i in range(n):
        got = _bits(srv.read(i + 1, int(counts[i]), dtypes[i]))
        assert np.array_equal(got, alone[i]), i
    for i in range(0, n, 12):
        want = oracle_mod.generate(int(seeds[i]), int(offsets[i]), int(counts[i]), dtypes[i])
        assert np.array_equal(alone[i], _obits(want)), i
    srv.close()


def test_admission_waits_for_pool_space(R, oracle_mod):
    pool = 8 << 20
    srv = R.Server(pool_bytes=pool, chunk_elems=1 << 15, release_after_s=-1.0)
    rnd = np.random.default_rng(3)
    reqs = []
    for k in range(40):
        n = int(rnd.integers(1 << 17, 3 << 17))  # 1..3 MiB of FP64
        a = int(rnd.integers(M + 100, 2 ** 53))
        reqs.append((srv.submit(a, k * 1000, n, "f64"), a, k * 1000, n))
    for rid, a, off, n in reqs:  # a client that reads, checks and releases in order
        srv.wait(rid, 30.0)
        got = _bits(srv.read(rid, n, "f64"))
        if rid % 7 == 0:
            assert np.array_equal(got, _obits(oracle_mod.generate(a, off, n, "f64")))
        srv.release(rid)
    st = srv.stats()
    assert st["completed"] == 40
    assert 0 < st["peak_pool_bytes"] <= pool
    assert st["pool_in_use"] == 0
    srv.close()


def test_bad_requests_do_not_disturb_the_others(R, oracle_mod):
    srv = R.Server(pool_bytes=16 << 20, release_after_s=-1.0)
    good = srv.submit(M + 500, 0, 100000, "f32")
    with pytest.raises(R.RNGError) as e:
        srv.submit(M + 99, 0, 10, "f64")
    assert e.value.status == 2
    with pytest.raises(R.RNGError) as e:
        srv.submit(M + 100, 0, 0, "f64")
    assert e.value.status == 1
    with pytest.raises(R.RNGError) as e:
        srv.submit(M + 100, 0, 4 << 20, "f64")  # 32 MiB > pool
    assert e.value.status == 3
    big = srv.submit(M + 700, 0, (15 << 20) // 8, "f64")  # fills the pool
    waiting = srv.submit(M + 800, 0, 1 << 20, "f64")    # cannot be admitted yet
    srv.cancel(waiting)
    assert srv.status(waiting)[0] == "cancelled"
    srv.wait(good, 30.0)
    srv.wait(big, 30.0)
    got = _bits(srv.read(good, 100000, "f32"))
    assert np.array_equal(got, _obits(oracle_mod.generate(M + 500, 0, 100000, "f32")))
    st, lat = srv.status(good)
    assert st == "done" and lat > 0
    srv.close()


def test_trace_replay_latencies(R):
    from paper_1206_1187_gb300 import inputs
    arrivals, counts, dtypes, seeds, offsets = inputs.request_trace(
        3000, rate_hz=20000.0, seed=9, min_bytes=1 << 10, max_bytes=4 << 20)
    srv = R.Server(pool_bytes=2 << 30, release_after_s=0.0)
    lat, wall = srv.run_trace(arrivals, seeds, counts, dtypes, offsets=offsets, timeout_s=60.0)
    assert np.isfinite(lat).all() and np.all(lat > 0)
    assert wall >= arrivals[-1]
    st = srv.stats()
    assert st["completed"] == 3000
    assert np.percentile(lat, 99) < 0.5
    # the server's own latency histogram holds the same latencies
    hist = srv.latency_histogram()
    assert hist.sum() == 3000
    us = lat * 1e6
    k = np.where(us > 1.0, np.floor(4.0 * np.log2(np.maximum(us, 1.0))), 0)
    want = np.bincount(np.minimum(k, R.HIST_BINS - 1).astype(np.int64), minlength=R.HIST_BINS)
    assert np.abs(hist.astype(np.int64) - want).sum() <= 4  # bin-edge rounding at most
    srv.close()


def test_released_requests_are_forgotten_beyond_the_history(R):
    """A long-running server keeps only a bounded history of released
    requests; a trace longer than that history still records every latency."""
    import time
    n = 70000  # more than the 65536 released requests the server remembers
    rnd = np.random.default_rng(17)
    seeds = rnd.integers(M + 100, 2 ** 53, size=n, endpoint=True, dtype=np.uint64)
    counts = rnd.integers(1, 65, size=n, dtype=np.uint64)
    dtypes = ["f64" if k % 2 else "f32" for k in range(n)]
    arrivals = np.zeros(n)
    srv = R.Server(pool_bytes=64 << 20, release_after_s=0.0)
    lat, wall = srv.run_trace(arrivals, seeds, counts, dtypes, timeout_s=120.0)
    assert np.isfinite(lat).all() and np.all(lat > 0) and wall > 0
    assert srv.stats()["completed"] == n
    deadline = time.time() + 10.0
    while srv.stats()["pool_in_use"] and time.time() < deadline:
        time.sleep(0.01)
    assert srv.stats()["pool_in_use"] == 0
    with pytest.raises(R.RNGError) as e:  # the oldest ids are no longer known
        srv.status(1)
    assert e.value.status == 1
    state, last_lat = srv.status(n)  # the newest are, with their latency
    assert state == "released" and last_lat == pytest.approx(lat[-1])
    with pytest.raises(R.RNGError) as e:
        srv.release(n)
    assert e.value.status == 6  # already released
    with pytest.raises(R.RNGError) as e:
        srv.read(n, int(counts[-1]), dtypes[-1])
    assert e.value.status == 6
    srv.close()


def test_trace_that_cannot_fit_a_never_releasing_pool_is_rejected(R):
    """With results held until the caller frees them, a trace whose outputs
    exceed the pool could never finish: it is refused before any submission."""
    from paper_1206_1187_gb300 import inputs
    arrivals, counts, dtypes, seeds, offsets = inputs.request_trace(
        200, rate_hz=20000.0, seed=3, min_bytes=1 << 20, max_bytes=4 << 20)
    srv = R.Server(pool_bytes=64 << 20)  # release_after_s < 0: never freed by the server
    with pytest.raises(R.RNGError) as e:
        srv.run_trace(arrivals, seeds, counts, dtypes, offsets=offsets, timeout_s=10.0)
    assert e.value.status == 1 and "never frees" in str(e.value)
    assert srv.stats()["submitted"] == 0
    srv.close()


def test_heavy_iterations_give_the_same_bytes(R, oracle_mod):
    """Iterations large enough for the throughput shape (deep tiles, wide
    blocks) give each request the bytes it gets alone (light shape)."""
    rnd = np.random.default_rng(21)
    reqs = [(int(rnd.integers(M + 100, 2 ** 53 - 10 ** 8)), int(rnd.integers(0, 2 ** 40)),
             int(rnd.integers(3 << 20, 5 << 20)), ("f64", "f32")[k % 2]) for k in range(12)]
    srv = R.Server(pool_bytes=1 << 30)
    ids = [srv.submit(a, off, n, dt) for a, off, n, dt in reqs]
    for rid in ids:
        srv.wait(rid, 60.0)
    st = srv.stats()
    assert st["heavy_iterations"] > 0
    mixed = [_bits(srv.read(rid, n, dt)) for rid, (a, off, n, dt) in zip(ids, reqs)]
    srv.close()
    srv = R.Server(pool_bytes=1 << 30, chunk_elems=1 << 20)
    for (a, off, n, dt), got in zip(reqs, mixed):
        rid = srv.submit(a, off, n, dt)
        srv.wait(rid, 60.0)
        assert np.array_equal(_bits(srv.read(rid, n, dt)), got)
        srv.release(rid)
    assert srv.stats()["heavy_iterations"] == 0
    srv.close()
    for (a, off, n, dt), got in list(zip(reqs, mixed))[:3]:
        idx = np.unique(np.concatenate([np.arange(1000), np.arange(n - 1000, n),
                                        rnd.integers(0, n, 1000)]))
        want = oracle_mod.at(a, (off + idx).astype(np.uint64), dt)
        assert np.array_equal(got[idx], _obits(want))


def test_concurrent_clients(R, oracle_mod):
    """Four host threads submit, wait for, read and release their own requests
    at once (the library's calls run without the interpreter lock); every
    result is the bytes of that request alone."""
    import threading
    srv = R.Server(pool_bytes=256 << 20, release_after_s=-1.0)
    errors, checked = [], []

    def client(k):
        try:
            rnd = np.random.default_rng(100 + k)
            for i in range(120):
                a = int(rnd.integers(M + 100, 2 ** 53))
                off = int(rnd.integers(0, 2 ** 40))
                n = int(rnd.integers(1, 200000))
                dt = ("f64", "f32", "u64")[int(rnd.integers(0, 3))]
                rid = srv.submit(a, off, n, dt)
                srv.wait(rid, 60.0)
                got = _bits(srv.read(rid, n, dt))
                srv.release(rid)
                if i % 10 == 0:
                    want = oracle_mod.generate(a, off, n, dt)
                    if not np.array_equal(got, _obits(want)):
                        errors.append((k, i, a, off, n, dt))
                    checked.append(1)
        except Exception as e:  # surfaced below
            errors.append((k, repr(e)))

    threads = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(300)
    assert not any(t.is_alive() for t in threads)
    assert not errors, errors[:3]
    assert len(checked) == 48
    st = srv.stats()
    assert st["completed"] == 480 and st["pool_in_use"] == 0
    srv.close()


def test_reads_race_automatic_release(R, oracle_mod):
    """With results freed almost at once (release_after_s = 1 ms) and other
    requests admitted into the freed space all the time, a read either finds
    the request already released (RNG_EBUSY) or returns exactly its bytes: a
    release that falls due during the copy waits for it."""
    import threading
    srv = R.Server(pool_bytes=24 << 20, release_after_s=0.001, chunk_elems=1 << 14)
    stop = threading.Event()

    def load():  # keeps the pool busy with other requests, at most 16 in flight
        rnd = np.random.default_rng(5)
        pending = []
        while not stop.is_set():
            pending.append(srv.submit(int(rnd.integers(M + 100, 2 ** 53)), 0,
                                      int(rnd.integers(1 << 12, 1 << 18)), "f64"))
            if len(pending) >= 16:
                srv.wait(pending.pop(0), 60.0)

    th = threading.Thread(target=load)
    th.start()
    rnd = np.random.default_rng(6)
    ok = busy = 0
    try:
        for i in range(150):
            a, off = int(rnd.integers(M + 100, 2 ** 53)), int(rnd.integers(0, 2 ** 40))
            n = int(rnd.integers(1 << 14, 1 << 19))
            rid = srv.submit(a, off, n, "f64")
            srv.wait(rid, 60.0)
            try:
                got = _bits(srv.read(rid, n, "f64"))
            except R.RNGError as e:
                assert e.status == 6, e  # released before the read started
                busy += 1
                continue
            ok += 1
            if i % 5 == 0:
                want = oracle_mod.generate(a, off, n, "f64")
                assert np.array_equal(got, _obits(want)), i
            else:
                idx = rnd.integers(0, n, 64)
                want = oracle_mod.at(a, (off + idx).astype(np.uint64), "f64")
                assert np.array_equal(got[idx], _obits(want)), i
    finally:
        stop.set()
        th.join(60)
    assert ok > 0
    srv.close()
