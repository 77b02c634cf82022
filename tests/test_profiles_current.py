"""The profiler counters committed under profiles/ belong to the kernels as
they are: every `key[tag]: value digest <hex>` line that bench.py reads must
carry the digest of the current device sources of its kernel (host-side
launcher changes do not count).  A kernel change without a new capture fails
here rather than silently dropping the counters from the benchmark line."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the counters bench.py reads, with the kernel each one describes
READ_BY_BENCH = {
    ("traffic_bytes_per_launch", "bulk_f64_2e28"): "tiled",
    ("traffic_bytes_per_launch", "bulk_f32_2e28"): "tiled",
    ("inst_per_variate", "f32_2e26"): "tiled",
    ("traffic_bytes_per_launch", "m40_f64_2e28"): "m40",
    ("inst_per_variate", "m40_2e25"): "m40",
    ("traffic_bytes_per_launch", "m40_f32_2e28"): "m40",
    ("inst_per_variate", "m40_f32_2e25"): "m40",
    ("inst_per_variate", "mc_2e36"): "mc",
    ("alu_pipe_busy_frac", "mc_2e36"): "mc",
    ("fp64_pipe_busy_frac", "mc_2e36"): "mc",
    ("traffic_per_algorithmic_byte", "batch_512"): "batch",
    ("inst_per_variate", "batch_512"): "batch",
    ("inst_per_variate", "devapi_2e30"): "device",
    ("inst_per_variate", "devapi32_2e30"): "device",
}


def _recorded():
    pat = re.compile(r"^(\w+)\[(\w+)\]:\s*([0-9.eE+]+)\s+digest\s+([0-9a-f]+)\s*$", re.M)
    found = {}
    pdir = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(pdir)):
        if name.endswith((".md", ".txt")):
            with open(os.path.join(pdir, name)) as fh:
                for m in pat.finditer(fh.read()):
                    found[(m.group(1), m.group(2))] = (float(m.group(3)), m.group(4), name)
    return found


@pytest.mark.parametrize("key", sorted(READ_BY_BENCH))
def test_counter_matches_current_kernel(key):
    from paper_1206_1187_gb300 import _build
    rec = _recorded()
    assert key in rec, f"profiles/ has no {key[0]}[{key[1]}] line"
    value, digest, fname = rec[key]
    want = _build.kernel_digest(READ_BY_BENCH[key])
    assert digest == want, (f"{fname}: {key[0]}[{key[1]}] was taken for kernel sources "
                            f"{digest}, the sources are now {want}: re-take the capture")
    assert value > 0


def test_bench_reads_the_same_counters():
    import bench
    for (k, tag), kernel in READ_BY_BENCH.items():
        assert bench.profiled_value(k, tag, kernel) is not None, (k, tag)
