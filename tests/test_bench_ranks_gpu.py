"""bench.py's multi-rank path (the one the driver launches under torchrun,
one rank per GPU) run with two ranks on the visible GPU: each rank generates
its own block of the sequence by skip-ahead, the step time is the maximum over
ranks, and rank 0 alone prints one JSON line whose value counts every rank's
variates.  The ranks exchange nothing but the timing barrier and maxima (gloo
here; NCCL when each rank has a GPU of its own)."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_ranks_print_one_weak_scaling_line():
    n = 1 << 22
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--gpus", "2", "--steps", "5", "--warmup", "3",
           f"--variates={n}", "--no-batch", "--no-fused", "--no-serve", "--no-m40", "--no-device-api",
           "--no-cpu-baseline", "--no-autotune", "--e2e-steps", "1"]
    env = dict(os.environ, BCN_BENCH_BACKEND="gloo")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["scaling"] == "weak" and d["steps"] == 5
    # value = both ranks' variates over the slower rank's step time
    assert d["value"] == pytest.approx(2 * n / (d["ms_per_step"] / 1e3), rel=1e-9)
    assert d["e2e"]["d2h_bytes_per_step"] == 8 * n and "cpu_baseline" not in d
