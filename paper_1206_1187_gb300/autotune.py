"""The project's autotuner: picks the step variant, conversion, tile depth and
block shape by measurement (the native timing harness rng_autotune_bulk),
caches the winner per GPU model and dtype, and installs it as the library's
default for calls that leave those fields at zero.

Results never depend on the choice -- every candidate writes the same bytes
-- so tuning only changes speed.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import _build, rng

CACHE = os.path.join(_build.BUILD_DIR, "autotune.json")
_lock = threading.Lock()

STEPS = ("shared", "barrett", "montgomery")
DEPTHS = (5, 7, 9, 15, 31, 63)          # variates per lane per tile (odd)
BLOCKS = (128, 256, 512)


def bulk_candidates(dtype: str) -> list[dict]:
    cands = []
    for step in STEPS:
        for conv in ("int", "fp64"):
            if dtype == "u64" and conv == "fp64":
                continue
            for depth in DEPTHS:
                for block in BLOCKS:
                    for chains in ((1, 2) if step != "montgomery" else (1,)):
                        # one tile buffer per warp only pays where tiles are deep
                        for buffers in ((1, 2) if depth >= 15 and step == "shared" else (2,)):
                            cands.append(dict(step=step, conv=conv, layout="tiled",
                                              depth=depth, block=block, chains=chains,
                                              buffers=buffers))
    # wide blocks: with one tile buffer per warp, up to 28 warps of depth-31 tiles
    # share an SM's shared memory
    if dtype != "u64":
        wide = [(15, (768, 1024)), (31, (640, 768, 896))]
        if dtype == "f64":  # 30: 2 mod 4, two variates per shared-memory store
            wide += [(30, (640, 768, 896))]
        if dtype == "f32":  # FP32 tiles are half the bytes: deeper ones fit (44: 4 mod 8,
            # four variates per shared-memory store)
            wide += [(44, (768, 896, 1024)), (47, (768, 896, 1024)), (63, (512, 640, 768, 896))]
        for depth, blocks in wide:
            for block in blocks:
                cands.append(dict(step="shared", conv="int", layout="tiled", depth=depth,
                                  block=block, chains=2, buffers=1))
        if dtype == "f32":  # one chain: each 44-deep run from one product
            for block in (768, 896, 1024):
                cands.append(dict(step="shared", conv="int", layout="tiled", depth=44,
                                  block=block, chains=1, buffers=1))
    return cands


def _key(dtype: str, n: int) -> str:
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    return f"{name}|bulk|{dtype}|{n}|v{rng.version()}"


def _load_cache() -> dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store_cache(cache: dict) -> None:
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1)
    os.replace(tmp, CACHE)


def tune_bulk(dtype: str = "f64", n: int = 1 << 26, reps: int = 5, candidates=None,
              use_cache: bool = True, install: bool = True) -> dict:
    """Measure the candidates on an n-element buffer and return
    {"best": tuning, "table": [[candidate, ms], ...], "n": n}."""
    key = _key(dtype, n)
    with _lock:
        cache = _load_cache() if use_cache else {}
        entry = cache.get(key) if candidates is None else None
        if entry is None:
            cands = candidates or bulk_candidates(dtype)
            best, ms = rng.autotune_bulk(n, dtype, cands, reps=reps)
            torch.cuda.synchronize()
            entry = {"best": rng.tune_dict(best), "n": n, "reps": reps,
                     "table": [[c, t] for c, t in zip(cands, ms)]}
            if use_cache and candidates is None:
                cache[key] = entry
                _store_cache(cache)
    if install:
        b = dict(entry["best"])
        b.pop("grid", None)
        rng.set_auto_tune(dtype, b)
    return entry


BATCH_DEPTHS = (15, 31)
BATCH_BLOCKS = (128, 256, 512)
BATCH_UNITS = (4, 16, 64)


def batch_candidates() -> list[dict]:
    cands = [dict(step="shared", conv="int", depth=d, block=b, chains=c, unit=u)
             for d in BATCH_DEPTHS for b in BATCH_BLOCKS for c in (1, 2) for u in BATCH_UNITS]
    # one tile buffer per warp, so that more warps fit per SM
    cands += [dict(step="shared", conv="int", depth=d, block=b, chains=2, unit=u, buffers=1)
              for d, blocks in ((15, (512, 768, 1024)), (31, (512, 640, 768, 896)))
              for b in blocks for u in BATCH_UNITS]
    # the built-in per-type depths (FP64 30, FP32 44, raw states 31)
    cands += [dict(step="shared", conv="int", depth=0, block=b, chains=2, unit=u, buffers=1)
              for b in (640, 768, 896) for u in BATCH_UNITS]
    return cands


def tune_batch(nstreams: int = 512, reps: int = 3, use_cache: bool = True,
               workload=None, tag: str = "") -> dict:
    """Time batch-plan tunings and return {"best": tuning, "table": [[candidate,
    ms], ...]}; cached per GPU model.  By default on a representative batch (the
    batched workload's generator, nstreams streams of lengths log-uniform
    10^3..10^6); `workload` = (starts, counts, dtypes, outs), or a callable
    returning it (called only when the cache has no entry), tunes on that batch
    itself, cached under `tag`."""
    from . import inputs
    name = tag if workload is not None else str(nstreams)
    key = f"{torch.cuda.get_device_name(torch.cuda.current_device())}|batch|{name}" \
          f"|v{rng.version()}"
    with _lock:
        cache = _load_cache() if use_cache else {}
        if key in cache:
            return cache[key]
        if workload is not None:
            starts, counts, dtypes, outs = workload() if callable(workload) else workload
        else:
            starts, counts, dtypes = inputs.batch_streams(nstreams=nstreams, len_hi=1e6)
            tdt = {"f64": torch.float64, "f32": torch.float32}
            outs = [torch.empty(int(c), dtype=tdt[d], device="cuda")
                    for c, d in zip(counts, dtypes)]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        table = []
        for cand in batch_candidates():
            try:
                b = rng.Batch(starts, counts, dtypes, outs=outs, tune=cand)
            except rng.RNGError:
                table.append([cand, -1.0])
                continue
            b.launch()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                b.launch()
            e1.record()
            torch.cuda.synchronize()
            table.append([cand, e0.elapsed_time(e1) / reps])
            b.close()
        ranked = sorted((t for t in table if t[1] > 0), key=lambda t: t[1])
        entry = {"best": ranked[0][0], "table": table, "nstreams": nstreams}
        if use_cache:
            cache[key] = entry
            _store_cache(cache)
    return entry
