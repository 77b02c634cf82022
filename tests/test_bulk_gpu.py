"""GPU parity of the bulk generator against the CPU oracle (bit-exact).

Integer states must match exactly; FP64 variates are compared bit for bit
(one round-to-nearest multiply by r3i, no FMA); FP32 variates likewise (the
FP64 variate truncated).  Every launch layout, reduction, conversion,
skip-ahead method and tile shape must give the same bytes.
"""
import itertools
import os
import random

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M = 3 ** 33
P = 2 * 3 ** 32
NPDT = {"f64": np.int64, "f32": np.int32, "u64": np.int64}


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_1187_gb300 import rng  # raises if the library is not built
    return rng


def dev_bits(t):
    import torch
    iv = torch.int64 if t.element_size() == 8 else torch.int32
    return t.view(iv).cpu().numpy()


def host_bits(a: np.ndarray):
    return a.view(NPDT["f64"] if a.itemsize == 8 else NPDT["f32"])


def assert_same(dev, want, what=""):
    got = dev_bits(dev)
    exp = host_bits(want)
    if not np.array_equal(got, exp):
        bad = np.nonzero(got != exp)[0]
        raise AssertionError(f"{what}: {bad.size} mismatches, first at {bad[:5]}")


@pytest.mark.parametrize("dtype", ["f64", "f32", "u64"])
def test_single_stream_1e6(R, oracle_mod, dtype):
    """a = 3^33+100, n = 10^6 with the automatic launch choice."""
    a, n = M + 100, 10 ** 6
    s = R.Stream(a)
    out = s.generate(n, dtype)
    s.sync()
    assert_same(out, oracle_mod.generate(a, 0, n, dtype), dtype)
    assert s.state == (a, n)


VARIANTS = list(itertools.product(["barrett", "montgomery", "shared", "lecuyer",
                                   "barrett_classic"], ["int", "fp64"],
                                  ["tiled", "direct"], ["table", "sqmul"]))


@pytest.mark.parametrize("step,conv,layout,skip", VARIANTS)
def test_every_variant_matches_the_oracle(R, oracle_mod, step, conv, layout, skip):
    rnd = random.Random(VARIANTS.index((step, conv, layout, skip)))
    a = rnd.randint(M + 100, 2 ** 53)
    off = rnd.randint(0, 2 ** 40)
    n = 100003  # several tiles and a ragged tail
    t = R.make_tune(step=step, conv=conv, layout=layout, skip=skip)
    for dtype in ("f64", "f32", "u64"):
        out = R.generate_at(a, off, n, dtype, tune=t)
        assert_same(out, oracle_mod.generate(a, off, n, dtype), f"{step}/{conv}/{layout}/{dtype}")


def test_tile_shape_and_grid_never_change_the_output(R):
    import torch
    a, off, n = M + 4242, 12345, 3 * 10 ** 5 + 17
    ref = R.generate_at(a, off, n, "f64", tune=R.make_tune(layout="direct"))
    for depth, block, grid, step in [(1, 32, 1, "barrett"), (3, 64, 7, "montgomery"),
                                     (15, 256, 0, "barrett"), (7, 1024, 3, "barrett"), (31, 256, 0, "barrett"),
                                     (63, 128, 152, "montgomery"), (127, 64, 0, "barrett"),
                                     (255, 32, 5, "montgomery"), (9, 96, 1000, "barrett"),
                                     (5, 128, 0, "shared"), (63, 64, 77, "shared")]:
        for buffers in (1, 2):
            t = R.make_tune(step=step, layout="tiled", depth=depth, block=block, grid=grid,
                            buffers=buffers)
            out = R.generate_at(a, off, n, "f64", tune=t)
            assert torch.equal(out.view(torch.int64), ref.view(torch.int64)), (depth, block,
                                                                               grid, buffers)
    for block, grid in [(1, 1), (7, 3), (1024, 1), (33, 17)]:
        t = R.make_tune(layout="direct", block=block, grid=grid)
        out = R.generate_at(a, off, n, "f64", tune=t)
        assert torch.equal(out.view(torch.int64), ref.view(torch.int64)), (block, grid)


@pytest.mark.parametrize("step", ["shared", "barrett"])
def test_two_chains_per_lane(R, oracle_mod, step):
    """Two interleaved chains per lane (each lane's run split in halves) give
    the same bytes for every depth, block and grid."""
    import torch
    a, off, n = M + 777, 2 ** 33 + 5, 2 * 10 ** 5 + 13
    for dtype in ("f64", "f32", "u64"):
        want = oracle_mod.generate(a, off, n, dtype)
        for depth, block, grid in [(3, 32, 1), (5, 128, 0), (15, 512, 0), (31, 256, 7),
                                   (63, 64, 152), (255, 32, 0)]:
            t = R.make_tune(step=step, layout="tiled", depth=depth, block=block, grid=grid,
                            chains=2)
            out = R.generate_at(a, off, n, dtype, tune=t)
            assert_same(out, want, f"{step}/{dtype}/{depth}/{block}/{grid}")
    if step == "shared":  # FP64 runs of 2 mod 4: two variates per shared-memory store
        want = oracle_mod.generate(a, off, n, "f64")
        for depth, block, grid in [(10, 32, 1), (6, 96, 0), (30, 896, 0), (30, 640, 7),
                                   (254, 32, 0)]:
            t = R.make_tune(step=step, layout="tiled", depth=depth, block=block, grid=grid,
                            chains=2)
            assert_same(R.generate_at(a, off, n, "f64", tune=t), want,
                        f"{step}/f64/{depth}/{block}/{grid}")
    if step == "shared":  # FP32 runs of 4 mod 8: four variates per shared-memory store
        want = oracle_mod.generate(a, off, n, "f32")
        for depth, block, grid in [(4, 32, 1), (12, 96, 0), (44, 896, 0), (44, 1024, 7),
                                   (252, 32, 0)]:
            t = R.make_tune(step=step, layout="tiled", depth=depth, block=block, grid=grid,
                            chains=2)
            assert_same(R.generate_at(a, off, n, "f32", tune=t), want,
                        f"{step}/f32/{depth}/{block}/{grid}")
        # one chain, each 44-deep run from one product, one or two tile buffers
        for block, grid, buffers in [(1024, 0, 1), (32, 1, 1), (96, 7, 1), (896, 152, 1),
                                     (64, 1000, 1), (512, 0, 2), (128, 3, 2)]:
            t = R.make_tune(step=step, layout="tiled", depth=44, block=block, grid=grid,
                            chains=1, buffers=buffers)
            assert_same(R.generate_at(a, off, n, "f32", tune=t), want,
                        f"{step}/f32/44/{block}/{grid}/{buffers}/one chain")


def test_windows_around_tiny_variates(R, oracle_mod):
    """Variates below 2^-21 leave the conversion's fast path (about one in 2^21);
    windows of the sequence around such variates, found with the oracle, must
    still match for every tile depth (compile-time and run-time) and layout."""
    a = M + 100
    states = oracle_mod.generate(a, 0, 1 << 24, "u64")
    tiny = np.nonzero(states < np.uint64(M >> 21))[0]
    assert tiny.size >= 3
    for i in tiny[:6]:
        off = max(0, int(i) - 3000)
        want64 = oracle_mod.generate(a, off, 6001, "f64")
        want32 = oracle_mod.generate(a, off, 6001, "f32")
        for depth in (5, 9, 15, 31, 63):
            t = R.make_tune(step="shared", layout="tiled", depth=depth)
            assert_same(R.generate_at(a, off, 6001, "f64", tune=t), want64, f"f64 {i} {depth}")
            assert_same(R.generate_at(a, off, 6001, "f32", tune=t), want32, f"f32 {i} {depth}")
        for depth in (12, 44):
            t = R.make_tune(step="shared", layout="tiled", depth=depth)
            assert_same(R.generate_at(a, off, 6001, "f32", tune=t), want32, f"f32 {i} {depth}")
        t = R.make_tune(step="shared", layout="tiled", depth=44, chains=1)
        assert_same(R.generate_at(a, off, 6001, "f32", tune=t), want32, f"f32 {i} one product")
        for depth in (6, 30):
            t = R.make_tune(step="shared", layout="tiled", depth=depth)
            assert_same(R.generate_at(a, off, 6001, "f64", tune=t), want64, f"f64 {i} {depth}")


def test_device_side_api_matches_the_oracle(R, oracle_mod):
    """A kernel written only against include/bcn_device.cuh (per-thread
    generators positioned by skip-ahead) gives the oracle's variates."""
    # the last two start at and run across the 2^64 boundary of the index
    for a, off, n, threads in [(M + 100, 0, 100003, 1000), (2 ** 53, 2 ** 50 + 7, 4097, 1),
                               (M + 12345, 123, 250000, 65536), (M + 100, 2 ** 64 - 3000, 6000, 64),
                               (2 ** 53, 2 ** 64 - 1, 10, 3)]:
        f64, f32, st = R.device_api_check(a, off, n, threads=threads, states=True)
        assert_same(f64, oracle_mod.generate(a, off, n, "f64"), f"f64 {a} {threads}")
        assert_same(f32, oracle_mod.generate(a, off, n, "f32"), f"f32 {a} {threads}")
        assert_same(st, oracle_mod.generate(a, off, n, "u64"), f"u64 {a} {threads}")


def test_device_side_api_consumed_in_registers(R, oracle_mod):
    """The device-side API as a simulation uses it: each thread consumes its
    own variates in registers and writes only the sum mod 2^64 of their FP64
    bit patterns; every thread's word equals that sum over the oracle's
    variates of the same range (uneven ranges, a range across offset 2^64,
    and an empty call)."""
    for a, off, n, threads in [(M + 100, 0, 100003, 128), (M + 777, 12345, (1 << 20) + 5, 1024),
                               (2 ** 53, 2 ** 64 - 3000, 6000, 256), (M + 105, 7, 0, 128)]:
        sums = R.device_api_checksum(a, off, n, threads=threads).cpu().numpy().view(np.uint64)
        want = (oracle_mod.generate(a, off, n, "f64").view(np.uint64) if n
                else np.zeros(0, dtype=np.uint64))
        for t in range(threads):
            lo, hi = n * t // threads, n * (t + 1) // threads
            w = int(want[lo:hi].astype(object).sum()) % 2 ** 64 if hi > lo else 0
            assert int(sums[t]) == w, (a, off, n, t)
        # FP32: runs of 32 from f32_run, the rest from next_f32
        sums = R.device_api_checksum(a, off, n, threads=threads,
                                     dtype="f32").cpu().numpy().view(np.uint64)
        want = (oracle_mod.generate(a, off, n, "f32").view(np.uint32) if n
                else np.zeros(0, dtype=np.uint32))
        for t in range(threads):
            lo, hi = n * t // threads, n * (t + 1) // threads
            w = int(want[lo:hi].astype(object).sum()) % 2 ** 64 if hi > lo else 0
            assert int(sums[t]) == w, ("f32", a, off, n, t)


def test_device_side_f32_runs_match_the_oracle(R, oracle_mod):
    """bcn_device::f32_run (32 FP32 variates from one product) and next_f32 for
    the remainder write the oracle's FP32 variates: uneven thread ranges, a
    range across offset 2^64, ranges shorter than one run."""
    for a, off, n, threads in [(M + 100, 0, 100003, 128), (M + 777, 12345, (1 << 20) + 5, 1024),
                               (2 ** 53, 2 ** 64 - 3000, 6000, 128), (M + 5555, 3, 31, 128),
                               (M + 999, 2 ** 40 + 1, 4096 * 33, 4096)]:
        got = R.device_api_f32_runs(a, off, n, threads=threads)
        assert_same(got, oracle_mod.generate(a, off, n, "f32"), f"{a} {off} {n} {threads}")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_small_misaligned_outputs_and_canaries(R, oracle_mod, dtype):
    """n = 1..97 at every element offset inside a 16-byte line; the bytes
    around the output must stay untouched (bounds check by canary)."""
    import torch
    tdt = torch.float64 if dtype == "f64" else torch.float32
    esz = 8 if dtype == "f64" else 4
    a = M + 99991
    sentinel = -7.25
    for n in list(range(1, 98)) + [1000, 4097, 65537]:
        for shift in range(16 // esz):
            buf = torch.full((n + 64,), sentinel, dtype=tdt, device="cuda")
            view = buf[8 + shift: 8 + shift + n]
            R.generate_at(a, n, n, dtype, out=view)
            host = buf.cpu().numpy()
            assert np.all(host[: 8 + shift] == sentinel)
            assert np.all(host[8 + shift + n:] == sentinel)
            want = oracle_mod.generate(a, n, n, dtype)
            assert np.array_equal(host_bits(host[8 + shift: 8 + shift + n].copy()), host_bits(want)), (n, shift)


def test_stream_calls_concatenate(R, oracle_mod):
    import torch
    a = M + 31337
    s = R.Stream(a)
    parts = [s.generate(k, "f64") for k in (1, 2, 1000, 33333, 7)]
    s.skip(500)
    parts.append(s.generate(4096, "f64"))
    got = torch.cat(parts)
    want = np.concatenate([oracle_mod.generate(a, 0, 1 + 2 + 1000 + 33333 + 7, "f64"),
                           oracle_mod.generate(a, 1 + 2 + 1000 + 33333 + 7 + 500, 4096, "f64")])
    assert_same(got, want, "chunks")
    # checkpoint and resume
    seed, count = s.state
    cont = s.generate(1000, "f64")
    s2 = R.Stream(M + 100)
    s2.set_state(seed, count)
    assert torch.equal(s2.generate(1000, "f64").view(torch.int64), cont.view(torch.int64))


def test_generate_to_host_pipelines_chunks(R, oracle_mod):
    """Host output through rotating device staging buffers: any chunk size and
    buffer count give the oracle's variates and advance the count."""
    import torch
    a = M + 2024
    for dtype in ("f64", "f32"):
        for n, chunk, nbuf in [(1, 0, 0), (100003, 4096, 3), (1 << 21, 1 << 20, 8),
                               (777777, 256, 1)]:
            s = R.Stream(a)
            s.skip(12345)
            out = s.generate_to_host(n, dtype, chunk_bytes=chunk, nbuf=nbuf)
            assert not out.is_cuda
            want = oracle_mod.generate(a, 12345, n, dtype)
            assert np.array_equal(host_bits(out.numpy()), host_bits(want)), (dtype, n, chunk)
            assert s.state == (a, 12345 + n)
            nxt = s.generate(1000, dtype)
            assert_same(nxt, oracle_mod.generate(a, 12345 + n, 1000, dtype), "after host call")
    pageable = torch.empty(5000, dtype=torch.float64)
    s = R.Stream(a)
    s.generate_to_host(5000, "f64", out=pageable)
    assert np.array_equal(host_bits(pageable.numpy()), host_bits(oracle_mod.generate(a, 0, 5000, "f64")))


def test_offsets_across_the_period_and_far_out(R, oracle_mod):
    a = 2 ** 53
    for off in (P - 50, P, 2 * P - 7, 2 ** 60 + 11, 2 ** 64 - 5000, 2 ** 64 - 2000):
        n = 4000
        for dtype in ("u64", "f64"):
            out = R.generate_at(a, off, n, dtype)
            assert_same(out, oracle_mod.generate(a, off, n, dtype), f"off={off}")


def test_seed_bounds_on_device(R, oracle_mod):
    for a in (M + 100, 2 ** 53):
        out = R.generate_at(a, 0, 5000, "u64")
        assert_same(out, oracle_mod.generate(a, 0, 5000, "u64"), f"a={a}")
    with pytest.raises(R.RNGError):
        R.generate_at(M + 99, 0, 10, "f64")


def test_bad_tuning_is_rejected(R):
    for kw in ({"depth": 16, "layout": "tiled"}, {"block": 48, "layout": "tiled"},
               {"block": 2048}, {"step": 9}, {"conv": 5}, {"skip": 4},
               {"depth": 12, "layout": "tiled"}):
        with pytest.raises(R.RNGError) as e:
            R.generate_at(M + 100, 0, 1000, "f64", tune=R.make_tune(**kw))
        assert e.value.status == 1
    # even depths: on two chains with the shared step FP32 takes 4 mod 8 only,
    # FP64 2 mod 4 only, raw states none
    for dtype, kw in (("f32", {"depth": 16}), ("f32", {"depth": 6}), ("f32", {"depth": 30}),
                      ("f32", {"depth": 12, "chains": 1}), ("f32", {"depth": 36, "chains": 1}),
                      ("f32", {"depth": 44, "chains": 1, "conv": "fp64"}), ("f32", {"depth": 12, "step": "barrett"}),
                      ("f64", {"depth": 44}), ("f64", {"depth": 30, "chains": 1}),
                      ("f64", {"depth": 30, "step": "barrett"}), ("f64", {"depth": 30, "conv": "fp64"}),
                      ("u64", {"depth": 30}), ("u64", {"depth": 44})):
        with pytest.raises(R.RNGError) as e:
            R.generate_at(M + 100, 0, 1000, dtype, tune=R.make_tune(layout="tiled", **kw))
        assert e.value.status == 1, (dtype, kw)


def test_oversized_tiles_shrink_the_block_by_whole_warps(R, oracle_mod):
    """Tiles too large for the default block's shared memory shrink the block
    in whole warps until they fit, and the output is unchanged."""
    import torch
    optin = getattr(torch.cuda.get_device_properties(0), "shared_memory_per_block_optin",
                    232448)
    esz = {"f64": 8, "f32": 4, "u64": 8}
    for dtype in ("f64", "f32", "u64"):
        for depth in (255, 127, 63):
            tune = dict(depth=depth, buffers=2)
            r = R.resolve_tune(1 << 20, dtype, R.make_tune(**tune))
            assert r["block"] >= 32 and r["block"] % 32 == 0, (tune, r)
            assert r["block"] // 32 * r["buffers"] * 32 * r["depth"] * esz[dtype] <= optin
            n = 32 * depth * 3 + 77
            a = M + 2718281
            out = R.generate_at(a, 5, n, dtype, tune=R.make_tune(**tune))
            assert_same(out, oracle_mod.generate(a, 5, n, dtype), f"{dtype} {tune}")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fill_constant_writes_every_element(R, dtype):
    import torch
    for n in (1, 31, 4097, 10 ** 6 + 3):
        out = R.fill_constant(n, dtype, 0.375)
        assert bool(torch.all(out == 0.375))


@pytest.mark.slow
def test_two_gib_single_stream_is_thread_count_invariant(R, oracle_mod):
    """a = 3^33+12345, n = 2^28 FP64 (2 GiB): byte-identical for 1, 2^10 and
    2^16 threads of the per-thread split, for the tiled kernel the library
    picks, and to the oracle."""
    import torch
    a, n = M + 12345, 1 << 28
    tiled = R.generate_at(a, 0, n, "f64")
    want = oracle_mod.generate_mt(a, 0, n, "f64", threads=os.cpu_count() or 1)
    assert_same(tiled, want, "tiled 2^28")
    del want
    tb = tiled.view(torch.int64)
    for block, grid in [(256, 4), (256, 256), (1, 1)]:  # 2^10, 2^16, 1 thread
        out = R.generate_at(a, 0, n, "f64", tune=R.make_tune(layout="direct", block=block,
                                                             grid=grid))
        assert torch.equal(out.view(torch.int64), tb), (block, grid)
        del out
    for step, conv, chains in [("montgomery", "int", 1), ("barrett", "fp64", 1),
                               ("barrett", "int", 1), ("shared", "int", 2)]:
        out = R.generate_at(a, 0, n, "f64", tune=R.make_tune(step=step, conv=conv,
                                                             chains=chains))
        assert torch.equal(out.view(torch.int64), tb), (step, conv, chains)
        del out
    # the benchmark's launch: the autotuner's pick on this size, and the shape it
    # has picked on GB300 (depth 31, 896-thread blocks, one buffer per warp)
    from paper_1206_1187_gb300 import autotune
    best = autotune.tune_bulk("f64", n=n)["best"]
    for tune in (best, dict(step="shared", conv="int", layout="tiled", depth=31, block=896,
                            chains=2, buffers=1)):
        out = R.generate_at(a, 0, n, "f64", tune=tune)
        assert torch.equal(out.view(torch.int64), tb), tune
        del out


def test_generation_calls_replay_in_a_cuda_graph(R, oracle_mod):
    """rng_generate_at and rng40_generate_at captured into a CUDA graph (after
    one eager call) and replayed write the oracle's variates."""
    import torch
    from m40_math import M40
    n = 300007
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    out40 = torch.empty(n, dtype=torch.float32, device="cuda")
    R.generate_at(M + 777, 5, n, "f64", out=out)
    R.generate40_at(M40 + 777, 5, n, "f32", out=out40)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            R.generate_at(M + 777, 5, n, "f64", out=out, stream=s)
            R.generate40_at(M40 + 777, 5, n, "f32", out=out40, stream=s)
    out.zero_()
    out40.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert_same(out, oracle_mod.generate(M + 777, 5, n, "f64"), "graph f64")
    assert np.array_equal(out40.view(torch.int32).cpu().numpy(),
                          oracle_mod.generate40(M40 + 777, 5, n, "f32").view(np.int32))


@pytest.mark.slow
def test_full_size_fp32_and_states_sampled(R, oracle_mod):
    """2^28 FP32 variates and 2^28 raw states of the bench's stream in the
    default launch: first and last 4096 and 8192 random positions each."""
    import torch
    a, n = M + 12345, 1 << 28
    rnd = np.random.default_rng(28)
    idx = np.unique(np.concatenate([np.arange(4096), np.arange(n - 4096, n),
                                    rnd.integers(0, n, size=8192)])).astype(np.int64)
    one_product = R.make_tune(step="shared", layout="tiled", depth=44, chains=1)
    for dtype, tune in (("f32", None), ("u64", None), ("f32", one_product)):
        out = R.generate_at(a, 0, n, dtype, tune=tune)
        torch.cuda.synchronize()
        iv = torch.int32 if dtype == "f32" else torch.int64
        got = out.view(iv)[torch.from_numpy(idx).cuda()]  # index the integer view
        want = oracle_mod.at(a, idx.astype(np.uint64), dtype)
        assert np.array_equal(got.cpu().numpy(),
                              want.view(np.int32 if dtype == "f32" else np.int64)), (dtype, tune)
        del out, got


def test_host_threads_generate_concurrently(R, oracle_mod):
    """Four host threads, each with its own stream object and CUDA stream,
    generate at once (the library's shared state -- installed tunings, device
    properties, kernel attributes -- is locked); every result is exact."""
    import threading
    import torch
    results, errors = {}, []

    def work(k):
        try:
            cs = torch.cuda.Stream()
            s = R.Stream(M + 1000 * (k + 1))
            s.skip(7 * k)
            outs = []
            for j in range(5):
                outs.append(s.generate(200003 + j, ("f64", "f32", "u64")[j % 3], stream=cs))
            cs.synchronize()
            results[k] = outs
        except Exception as ex:  # reported below
            errors.append(repr(ex))

    threads = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for k in range(4):
        a, pos = M + 1000 * (k + 1), 7 * k
        for j, out in enumerate(results[k]):
            n, dt = 200003 + j, ("f64", "f32", "u64")[j % 3]
            assert_same(out, oracle_mod.generate(a, pos, n, dt), f"thread {k} call {j}")
            pos += n


@pytest.mark.parametrize("dtype", ["f64", "f32", "u64"])
def test_paper_strided_layout_matches_the_oracle(R, oracle_mod, dtype):
    """The paper's coalesced kernels (RNG_LAYOUT_STRIDED): thread t of T makes
    its block of W variates and writes them T apart.  Every step variant,
    both conversions, unrolled by 1 and by 8, gives the oracle's permuted
    order bit for bit."""
    a, off = M + 7777, 4242
    per, threads = 64, 1000
    n = per * threads
    want = oracle_mod.generate_strided(a, off, n, dtype, per=per)
    for step in ("shared", "barrett", "montgomery", "lecuyer", "barrett_classic"):
        for conv in (("int", "fp64") if dtype != "u64" else ("int",)):
            for unit in (1, 8):
                t = R.make_tune(step=step, conv=conv, layout="strided", depth=per, unit=unit,
                                block=96)
                out = R.generate_at(a, off, n, dtype, tune=t)
                assert_same(out, want, f"{step} {conv} unroll {unit}")


def test_paper_strided_layout_at_the_papers_shape(R, oracle_mod):
    """4096 variates per thread and 512-thread blocks (the paper's C2050
    configuration), the constant kernel in the same layout, and the checks:
    n must be a multiple of W, and no default may take this layout."""
    a, n = M + 12345, 1 << 22
    r = R.resolve_tune(n, "f64", R.make_tune(layout="strided"))
    assert (r["layout"], r["depth"], r["block"], r["grid"]) == ("strided", 4096, 512, 2)
    out = R.generate_at(a, 0, n, "f64", tune=R.make_tune(layout="strided"))
    assert_same(out, oracle_mod.generate_strided(a, 0, n, "f64", per=4096), "paper shape")
    import torch
    c = R.fill_constant(n, "f32", 0.25, tune=R.make_tune(layout="strided", unit=1))
    assert bool(torch.all(c == 0.25))
    with pytest.raises(R.RNGError) as e:
        R.generate_at(a, 0, n + 3, "f64", tune=R.make_tune(layout="strided"))
    assert e.value.status == 1
    with pytest.raises(R.RNGError) as e:
        R.set_auto_tune("f64", R.make_tune(layout="strided"))
    assert e.value.status == 1


def test_fp32_near_float_boundaries(R, oracle_mod):
    """FP32 variates whose quotient floor(2^53 z/m) has all ones (or all ones
    but the last one or two bits) below its leading 24 bits: the backward FP32
    step must take its exact path for the first two kinds and may not for the
    third.  Each chosen state is placed at a known output index of a seed by a
    discrete logarithm, and windows around it are generated with every FP32
    tile shape (compile-time and run-time depths, one and two chains) and in a
    batch."""
    import sys

    import torch
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from m40_math import dlog2
    rnd = random.Random(77)
    a = M + 31337
    h_inv = pow(M // 2, -1, M)
    targets = []
    for tail in (29, 28, 20, 12, 9):
        for k in (1, 2, 3):
            for _ in range(40):
                head = rnd.randrange(1 << 23, 1 << 24)
                q = (head << tail) | ((1 << tail) - k)
                z = -(-(q * M) // 2 ** 53)  # the state with this quotient, if any
                if 0 < z < M and z % 3 and (z << 53) // M == q:
                    targets.append(z)
                    break
    assert len(targets) >= 12
    shapes = [dict(), dict(depth=31), dict(depth=47, block=768), dict(depth=45, chains=2),
              dict(depth=63, chains=1), dict(depth=5, block=128), dict(depth=44, block=1024),
              dict(depth=12, block=96), dict(depth=44, chains=1), dict(depth=44, chains=1, block=64)]
    for z in targets:
        e = dlog2(z * h_inv % M, 33)
        i = ((e - (a - M)) * pow(53, -1, P) - 1) % P
        assert int(oracle_mod.generate(a, i, 1, "u64")[0]) == z
        off = i - 2000 if i >= 2000 else 0
        want = oracle_mod.generate(a, off, 4001, "f32")
        for shape in shapes:
            t = R.make_tune(step="shared", layout="tiled", **shape)
            assert_same(R.generate_at(a, off, 4001, "f32", tune=t), want, f"{z} {shape}")
        # the device-side runs (bcn_device::f32_run), whose flagged runs are made again
        assert_same(R.device_api_f32_runs(a, off, 4001, threads=128), want, f"{z} device runs")
        outs = [torch.empty(4001, dtype=torch.float32, device="cuda"),
                torch.empty(3, dtype=torch.float64, device="cuda")]
        b = R.Batch(np.array([a, a], dtype=np.uint64), np.array([4001, 3], dtype=np.uint64),
                    ["f32", "f64"], outs=outs, offsets=np.array([off, off], dtype=np.uint64))
        b.launch()
        assert_same(outs[0], want, f"batch {z}")
        b.close()


def test_small_calls_spread_their_tiles_over_every_sm(R, oracle_mod):
    """A call with too few tiles to give every SM a full block takes smaller
    blocks (unless the caller names the block or the grid); the output does
    not change."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for dtype, n in (("f64", 10 ** 6), ("f32", 10 ** 6), ("f64", 3 * 10 ** 5)):
        full = 1024 if dtype == "f32" else 896  # the default block of a large call
        auto = R.resolve_tune(n, dtype)
        tiles = n // (32 * auto["depth"])
        assert auto["block"] < full and auto["block"] % 32 == 0, (dtype, n, auto)
        assert auto["grid"] * auto["block"] // 32 >= min(tiles, sms), (dtype, n, auto)
        assert R.resolve_tune(n, dtype, R.make_tune(block=896))["block"] == 896
        assert R.resolve_tune(n, dtype, R.make_tune(grid=16))["block"] == full
        a = M + 1618
        assert_same(R.generate_at(a, 99, n, dtype), oracle_mod.generate(a, 99, n, dtype), dtype)
    assert R.resolve_tune(1 << 28, "f64")["block"] == 896
    assert R.resolve_tune(1 << 28, "f32")["block"] == 1024


def test_fp32_one_product_runs_equal_the_backward_step_at_full_size(R, oracle_mod):
    """The bench's 2^28 FP32 stream made by the default one-product runs and by
    the backward step on two chains: every element identical (two different
    computations of the same digits), and a sample equal to the oracle."""
    import torch
    a, n = M + 12345, 1 << 28
    one = R.generate_at(a, 0, n, "f32", tune=R.make_tune(step="shared", layout="tiled",
                                                        depth=44, chains=1))
    back = R.generate_at(a, 0, n, "f32", tune=R.make_tune(step="shared", layout="tiled",
                                                         depth=44, chains=2))
    torch.cuda.synchronize()
    assert torch.equal(one.view(torch.int32), back.view(torch.int32))
    idx = np.random.default_rng(44).integers(0, n, size=4096).astype(np.int64)
    got = one.view(torch.int32)[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert np.array_equal(got, oracle_mod.at(a, idx.astype(np.uint64), "f32").view(np.int32))
