"""Failure handling on the GPU, with failures made on the host.

Device and pinned allocations fail through the library's test hook
(rng_debug_fail_allocations) exactly as if memory had run out: the failing
call reports it, frees what it had taken, and the next call succeeds with the
right bytes.  The BCN_RNG_TUNE override forces a variant in a fresh process.
Nothing here faults, traps or hangs a GPU.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M = 3 ** 33
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_1187_gb300 import rng
    yield rng
    rng.debug_fail_allocations(0, 0)


def _bits(t):
    import torch
    return t.view(torch.int64 if t.element_size() == 8 else torch.int32).cpu().numpy()


def _obits(a):
    return a.view(np.int64 if a.itemsize == 8 else np.int32)


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_batch_plan_allocation_failure(R, oracle_mod):
    import torch
    from paper_1206_1187_gb300 import inputs
    starts, offsets, counts, dtypes = inputs.small_batch(nstreams=60, seed=31, max_len=5000)
    tdt = {"f64": torch.float64, "f32": torch.float32, "u64": torch.uint64}
    outs = [torch.zeros(int(c), dtype=tdt[d], device="cuda") for c, d in zip(counts, dtypes)]
    R.debug_fail_allocations(0, 1)
    with pytest.raises(R.RNGError) as e:
        R.Batch(starts, counts, dtypes, outs=outs, offsets=offsets)
    assert e.value.status == 4 and "cudaErrorMemoryAllocation" in str(e.value)
    b = R.Batch(starts, counts, dtypes, outs=outs, offsets=offsets)  # injection used up
    b.launch()
    torch.cuda.synchronize()
    for s in range(0, 60, 7):
        want = oracle_mod.generate(int(starts[s]), int(offsets[s]), int(counts[s]), dtypes[s])
        assert np.array_equal(_bits(outs[s]), _obits(want)), s
    b.close()


@pytest.mark.parametrize("skip", [0, 1, 2, 3])
def test_server_creation_failure_frees_everything(R, oracle_mod, skip):
    """The pool, then each slot's pinned tables and device table: whichever
    allocation fails, creation reports it and gives back the memory taken."""
    pool = 1 << 30
    before = _free_bytes()
    R.debug_fail_allocations(skip, 1)
    with pytest.raises(R.RNGError) as e:
        R.Server(pool_bytes=pool)
    assert e.value.status == 4
    R.debug_fail_allocations(0, 0)
    assert _free_bytes() > before - (64 << 20)  # the 1 GiB pool was released
    srv = R.Server(pool_bytes=pool, release_after_s=-1.0)
    rid = srv.submit(M + 900, 77, 50000, "f64")
    srv.wait(rid, 30.0)
    got = _bits(srv.read(rid, 50000, "f64"))
    assert np.array_equal(got, _obits(oracle_mod.generate(M + 900, 77, 50000, "f64")))
    srv.close()


def test_host_transfer_staging_failure_leaves_the_stream_usable(R, oracle_mod):
    s = R.Stream(M + 4321)
    s.skip(1000)
    n = 3 * (1 << 20) + 5
    R.debug_fail_allocations(2, 1)  # the third of four staging buffers
    with pytest.raises(R.RNGError) as e:
        s.generate_to_host(n, "f64", chunk_bytes=1 << 20, nbuf=4)
    assert e.value.status == 4
    assert s.state == (M + 4321, 1000)  # a failed call does not advance the stream
    h = s.generate_to_host(n, "f64", chunk_bytes=1 << 20, nbuf=4)
    assert s.state == (M + 4321, 1000 + n)
    want = oracle_mod.generate(M + 4321, 1000, n, "f64")
    assert np.array_equal(h.numpy().view(np.int64), _obits(want))


def test_environment_override_forces_a_variant():
    code = (
        "import numpy as np, torch\n"
        "from paper_1206_1187_gb300 import rng\n"
        "import oracle\n"
        "t = rng.resolve_tune(1 << 20, 'f64')\n"
        "print(t['step'], t['conv'], t['depth'], t['block'], t['chains'], t['buffers'])\n"
        "rng.set_auto_tune('f64', rng.make_tune(step='shared', depth=31, block=896))\n"
        "t2 = rng.resolve_tune(1 << 20, 'f64')\n"
        "print(t2['step'], t2['depth'])\n"
        "out = rng.generate_at(3**33 + 777, 12, 200001, 'f64')\n"
        "want = oracle.generate(3**33 + 777, 12, 200001, 'f64')\n"
        "print(bool(np.array_equal(out.view(torch.int64).cpu().numpy(), want.view(np.int64))))\n")
    env = dict(os.environ, BCN_RNG_TUNE="step=barrett,conv=fp64,depth=15,block=256,chains=1,"
                                        "buffers=2")
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = out.stdout.split("\n")
    assert lines[0] == "barrett fp64 15 256 1 2"
    assert lines[1] == "barrett 15"  # the override wins over an installed tuning
    assert lines[2] == "True"
