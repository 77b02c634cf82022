"""In-tree build of the CUDA library ``libbcn_rng.so`` for sm_103a.

Each ``csrc/*.cu`` file is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically.  Run
``python -m paper_1206_1187_gb300._build`` (or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import concurrent.futures
import glob
import hashlib
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libbcn_rng.so")
STAMP = LIB + ".stamp"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
    "-Xcompiler", "-Wall", "-I", INCLUDE, "-I", CSRC,
]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"),
                 os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build the library")


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs_digest(extra_flags: list[str]) -> str:
    h = hashlib.sha256()
    files = _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + sorted(
        glob.glob(os.path.join(CSRC, "*.h"))) + sorted(glob.glob(os.path.join(INCLUDE, "*.h"))) + \
        sorted(glob.glob(os.path.join(INCLUDE, "*.cuh")))
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + extra_flags).encode())
    return h.hexdigest()


# The device-code sources of each kernel, for per-kernel digests: a profiler
# counter recorded for a kernel stays valid while these are unchanged.  The
# host-side launchers (the *_api.cu files: argument checks, launch shapes) are
# kept out of these files so that changing them does not void the counters.
KERNEL_SOURCES = {
    "tiled": ["bcn_bulk.cu", "bcn_bulk.cuh", "bcn_digits.cuh", "bcn_digits_math.cuh",
              "bcn_gen.cuh", "bcn_math.cuh", "bcn_internal.h"],
    "batch": ["bcn_batch.cu", "bcn_batch.cuh", "bcn_digits.cuh", "bcn_digits_math.cuh",
              "bcn_gen.cuh", "bcn_math.cuh", "bcn_internal.h"],
    "mc": ["bcn_mc.cu", "bcn_mc.cuh", "bcn_gen.cuh", "bcn_math.cuh", "bcn_internal.h"],
    "m40": ["bcn_m40.cu", "bcn_m40.cuh", "bcn_digits.cuh", "bcn_digits_math.cuh", "bcn_gen.cuh",
            "bcn_math.cuh", "bcn_math40.cuh", "bcn_internal.h"],
    "device": ["bcn_device_check.cu", "bcn_device.cuh", "bcn_digits_math.cuh", "bcn_math.cuh",
               "bcn_internal.h"],
}


def _source_path(name: str) -> str:
    p = os.path.join(CSRC, name)
    return p if os.path.exists(p) else os.path.join(INCLUDE, name)


def _code_only(text: str) -> str:
    """Source text without comments and with whitespace runs collapsed, so a
    digest changes with the code, not with its commentary."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_digest(kernel: str) -> str:
    """16 hex digits identifying the code (comments aside) and flags one kernel
    is built from."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(_source_path(name), encoding="utf-8") as fh:
            h.update(name.encode())
            h.update(_code_only(fh.read()).encode())
    h.update(" ".join(f for f in NVCC_FLAGS if not os.path.isabs(f)).encode())  # no paths
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile and link the library if any source changed; return its path."""
    extra_flags = list(extra_flags or [])
    digest = _inputs_digest(extra_flags)
    if not force and os.path.exists(LIB) and os.path.exists(STAMP):
        with open(STAMP) as fh:
            if fh.read().strip() == digest:
                return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    srcs = _sources()
    objs = [os.path.join(BUILD_DIR, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc] + NVCC_FLAGS + extra_flags + ["-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stderr}")
        return res.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(srcs))) as ex:
        for log in ex.map(compile_one, zip(srcs, objs)):
            if verbose and log:
                sys.stderr.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
