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
                        cands.append(dict(step=step, conv=conv, layout="tiled", depth=depth,
                                          block=block, chains=chains))
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
