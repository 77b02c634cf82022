"""Named workloads at sizes suited to a profiler capture.

    python -m paper_1206_1187_gb300.cases bulk 33554432 [reps]     # FP64, autotuned shape
    python -m paper_1206_1187_gb300.cases bulk32 67108864 [reps]   # FP32, default shape
    python -m paper_1206_1187_gb300.cases batch 512 [reps]   # first 512 streams of the batched workload
    python -m paper_1206_1187_gb300.cases batch 4096 [reps]  # the whole batched workload
    python -m paper_1206_1187_gb300.cases mc 16384 [reps]
    python -m paper_1206_1187_gb300.cases devapi 1073741824 [reps]    # device-side header
    python -m paper_1206_1187_gb300.cases devapi32 1073741824 [reps]  # its FP32 runs
    python -m paper_1206_1187_gb300.cases m40 33554432 [reps]      # 3^40, FP64
    python -m paper_1206_1187_gb300.cases m40f32 33554432 [reps]   # 3^40, FP32

Each case runs `reps` launches (default 3) of one of the library's kernels on
synthetic inputs and exits 0; nothing is checked here (the test suite does
that).  Each uses the launch shape the benchmark uses for that form: the
autotuned one for FP64 (cached per GPU model), the built-in default for FP32,
batch plans, 3^40 (both output types) and the fused consumer.
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
        if dtype == "f64":
            autotune.tune_bulk(dtype, n=1 << 28)  # the tuning the benchmark uses
        out = torch.empty(size, dtype=torch.float64 if dtype == "f64" else torch.float32,
                          device="cuda")
        for _ in range(reps):
            rng.generate_at(seed, 0, size, dtype, out=out)
    elif case == "batch":
        tdt = {"f64": torch.float64, "f32": torch.float32}
        starts, counts, dtypes = inputs.batch_streams()  # the batched workload's streams
        starts, counts, dtypes = starts[:size], counts[:size], dtypes[:size]
        outs = [torch.empty(int(c), dtype=tdt[d], device="cuda") for c, d in zip(counts, dtypes)]
        # a plan's built-in shape (the one the autotuner picks for this workload)
        b = rng.Batch(starts, counts, dtypes, outs=outs)
        for _ in range(reps):
            b.launch()
    elif case in ("m40", "m40f32"):
        f64 = case == "m40"
        out = torch.empty(size, dtype=torch.float64 if f64 else torch.float32, device="cuda")
        for _ in range(reps):
            rng.generate40_at(3 ** 40 + 12345, 0, size, "f64" if f64 else "f32", out=out)
    elif case == "mc":
        for _ in range(reps):
            rng.consume_mc(3 ** 33 + 100, size, 1 << 16)
    elif case in ("devapi", "devapi32"):  # size variates consumed by 2^18 threads
        for _ in range(reps):
            rng.device_api_checksum(seed, 0, size, threads=1 << 18,
                                    dtype="f64" if case == "devapi" else "f32")
    else:
        raise SystemExit(f"unknown case {case!r}")
    torch.cuda.synchronize()
    print(f"{case} {size} x{reps} ok")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
