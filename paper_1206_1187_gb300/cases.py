"""Named workloads at sizes suited to a profiler capture.

    python -m paper_1206_1187_gb300.cases bulk 33554432 [reps]
    python -m paper_1206_1187_gb300.cases bulk32 33554432 [reps]
    python -m paper_1206_1187_gb300.cases batch 2048 [reps]
    python -m paper_1206_1187_gb300.cases mc 16384 [reps]
    python -m paper_1206_1187_gb300.cases m40 33554432 [reps]

Each case runs `reps` launches (default 3) of one of the library's kernels on
synthetic inputs and exits 0; nothing is checked here (the test suite does
that).  The tuning is the installed autotune result when one is cached.
"""
from __future__ import annotations

import sys


def main(argv):
    import torch

    from paper_1206_1187_gb300 import autotune, inputs, rng
    case = argv[1]
    size = int(argv[2])
    reps = int(argv[3]) if len(argv) > 3 else 3
    seed = 3 ** 33 + 12345
    if case in ("bulk", "bulk32"):
        dtype = "f64" if case == "bulk" else "f32"
        autotune.tune_bulk(dtype, n=1 << 28)  # the tuning the benchmark uses
        out = torch.empty(size, dtype=torch.float64 if dtype == "f64" else torch.float32,
                          device="cuda")
        for _ in range(reps):
            rng.generate_at(seed, 0, size, dtype, out=out)
    elif case == "batch":
        tdt = {"f64": torch.float64, "f32": torch.float32}

        def workload():  # built only if the tuning is not cached yet
            st, co, dt = inputs.batch_streams()
            return st, co, dt, [torch.empty(int(c), dtype=tdt[d], device="cuda")
                                for c, d in zip(co, dt)]
        # the benchmark's tuning, measured on the batched workload itself
        tune = autotune.tune_batch(workload=workload, tag="batched-4096-seed7")["best"]
        torch.cuda.empty_cache()
        starts, counts, dtypes = inputs.batch_streams(nstreams=size, len_hi=1e6)
        outs = [torch.empty(int(c), dtype=tdt[d], device="cuda") for c, d in zip(counts, dtypes)]
        b = rng.Batch(starts, counts, dtypes, outs=outs, tune=tune)
        for _ in range(reps):
            b.launch()
    elif case == "m40":
        out = torch.empty(size, dtype=torch.float64, device="cuda")
        for _ in range(reps):
            rng.generate40_at(3 ** 40 + 12345, 0, size, "f64", out=out)
    elif case == "mc":
        for _ in range(reps):
            rng.consume_mc(3 ** 33 + 100, size, 1 << 16)
    else:
        raise SystemExit(f"unknown case {case!r}")
    torch.cuda.synchronize()
    print(f"{case} {size} x{reps} ok")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
