"""CPU oracle for the Bailey-Borwein alpha_{2,3} generator (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package.  It wraps
``bcn_oracle.c`` (plain C, ``unsigned __int128 %``), which states Algorithm BB,
Eq. 2 and Eq. 3 of Beliakov et al. directly; see that file's header for the
readings it takes.  Nothing here imports the CUDA library, and the CUDA
library never imports this.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bcn_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libbcn_oracle.so")

# 3^33, the modulus of Eq. 3, and the seed range of Algorithm BB, step 1.
M = 3 ** 33
SEED_MIN = M + 100
SEED_MAX = 2 ** 53

# The larger-modulus variant (Sec. 1): 3^40, seeds [3^40+100, 2^64-1],
# period 2*3^39.
M40 = 3 ** 40
SEED_MIN40 = M40 + 100
SEED_MAX40 = 2 ** 64 - 1
P40 = 2 * 3 ** 39

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
        ):
            os.makedirs(_BUILD_DIR, exist_ok=True)
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = [
                "gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off",
                "-fno-fast-math", "-fPIC", "-shared", "-pthread",
                "-o", tmp, _SRC, "-lm",
            ]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
    lib.oracle_seed_state.restype = u64
    lib.oracle_seed_state.argtypes = [u64, u64]
    lib.oracle_step.restype = u64
    lib.oracle_step.argtypes = [u64]
    lib.oracle_to_f64.restype = ctypes.c_double
    lib.oracle_to_f64.argtypes = [u64]
    lib.oracle_to_f32.restype = ctypes.c_float
    lib.oracle_to_f32.argtypes = [u64]
    for name in ("oracle_states", "oracle_f64", "oracle_f32"):
        fn = getattr(lib, name)
        fn.restype = i32
        fn.argtypes = [u64, u64, u64, vp]
    lib.oracle_at.restype = i32
    lib.oracle_at.argtypes = [u64, vp, u64, i32, vp]
    lib.oracle_mc.restype = i32
    lib.oracle_mc.argtypes = [u64, u64, vp, u64, vp, vp, vp]
    lib.oracle_exact_sum.restype = i32
    lib.oracle_exact_sum.argtypes = [vp, u64, vp]
    lib.oracle_generate_mt.restype = i32
    lib.oracle_generate_mt.argtypes = [u64, u64, u64, i32, vp, i32]
    lib.oracle40_seed_state.restype = u64
    lib.oracle40_seed_state.argtypes = [u64, u64]
    lib.oracle40_step.restype = u64
    lib.oracle40_step.argtypes = [u64]
    lib.oracle40_to_f64.restype = ctypes.c_double
    lib.oracle40_to_f64.argtypes = [u64]
    lib.oracle40_to_f32.restype = ctypes.c_float
    lib.oracle40_to_f32.argtypes = [u64]
    lib.oracle40_generate.restype = i32
    lib.oracle40_generate.argtypes = [u64, u64, u64, i32, vp]
    lib.oracle40_at.restype = i32
    lib.oracle40_at.argtypes = [u64, vp, u64, i32, vp]
    _lib = lib
    return lib


def _ptr(arr: np.ndarray) -> int:
    return arr.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle: {what} rejected its arguments")


def seed_state(a: int, j: int = 0) -> int:
    """Eq. 2 for the seed index a + 53*j; 0 if a is outside [3^33+100, 2^53]."""
    return int(_load().oracle_seed_state(a, j))


def step(z: int) -> int:
    """Eq. 3 once: 2^53 z mod 3^33."""
    return int(_load().oracle_step(z))


def to_f64(z: int) -> float:
    return float(_load().oracle_to_f64(z))


def to_f32(z: int) -> np.float32:
    return np.float32(_load().oracle_to_f32(z))


_DTYPES = {"f64": (np.float64, 0), "f32": (np.float32, 1), "u64": (np.uint64, 2)}


def generate(a: int, j: int, n: int, dtype: str = "f64") -> np.ndarray:
    """Variates j .. j+n-1 of the stream with seed a, one thread, in order."""
    npdt, _ = _DTYPES[dtype]
    out = np.empty(n, dtype=npdt)
    fn = {"f64": "oracle_f64", "f32": "oracle_f32", "u64": "oracle_states"}[dtype]
    _check(getattr(_load(), fn)(a, j, n, _ptr(out)), fn)
    return out


def generate_strided(a: int, j: int, n: int, dtype: str = "f64", per: int = 4096) -> np.ndarray:
    """The paper's coalesced output order (Sec. 2.2): with T = n / per threads,
    thread t makes variates j + t*per .. j + t*per + per - 1 (its block of the
    sequence) and writes variate j + t*per + k to position k*T + t, i.e. its
    k-th output at its start index plus k times the step T."""
    if per <= 0 or n % per:
        raise ValueError(f"n = {n} is not a multiple of {per} variates per thread")
    seq = generate(a, j, n, dtype)
    threads = n // per
    out = np.empty_like(seq)
    for k in range(per):  # every thread's k-th variate, threads in order
        out[k * threads:(k + 1) * threads] = seq[k::per]
    return out


def generate_mt(a: int, j: int, n: int, dtype: str = "f64", threads: int = 1,
                out: np.ndarray | None = None) -> np.ndarray:
    """Same as generate(), split over host threads by skip-ahead (timing mode)."""
    npdt, code = _DTYPES[dtype]
    if out is None:
        out = np.empty(n, dtype=npdt)
    _check(_load().oracle_generate_mt(a, j, n, code, _ptr(out), threads),
           "oracle_generate_mt")
    return out


def at(a: int, idx, dtype: str = "f64") -> np.ndarray:
    """Variates at arbitrary positions, each computed straight from Eq. 2."""
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    npdt, code = _DTYPES[dtype]
    out = np.empty(idx.size, dtype=npdt)
    _check(_load().oracle_at(a, _ptr(idx), idx.size, code, _ptr(out)), "oracle_at")
    return out


def mc(a: int, length: int, blocks) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Monte-Carlo consumer: per block hits, exact-rounded sum and sum of squares."""
    blocks = np.ascontiguousarray(blocks, dtype=np.uint64)
    hits = np.empty(blocks.size, dtype=np.uint64)
    s1 = np.empty(blocks.size, dtype=np.float64)
    s2 = np.empty(blocks.size, dtype=np.float64)
    _check(_load().oracle_mc(a, length, _ptr(blocks), blocks.size, _ptr(hits),
                             _ptr(s1), _ptr(s2)), "oracle_mc")
    return hits, s1, s2


def exact_sum(values) -> float:
    """Round-to-nearest-even of the exact sum of non-negative doubles."""
    values = np.ascontiguousarray(values, dtype=np.float64)
    out = np.zeros(1, dtype=np.float64)
    _check(_load().oracle_exact_sum(_ptr(values), values.size, _ptr(out)),
           "oracle_exact_sum")
    return float(out[0])


# ---------------------------------------------------------------- modulus 3^40
def seed_state40(a: int, j: int = 0) -> int:
    """Eq. 2 with modulus 3^40 for the seed index a + 53*j; 0 if a < 3^40+100."""
    return int(_load().oracle40_seed_state(a, j))


def step40(z: int) -> int:
    """Eq. 3 with modulus 3^40 once: 2^53 z mod 3^40."""
    return int(_load().oracle40_step(z))


def to_f64_40(z: int) -> float:
    """z / 3^40 rounded toward zero, by binary long division."""
    return float(_load().oracle40_to_f64(z))


def to_f32_40(z: int) -> np.float32:
    return np.float32(_load().oracle40_to_f32(z))


def generate40(a: int, j: int, n: int, dtype: str = "f64") -> np.ndarray:
    """Variates j .. j+n-1 of seed a under the 3^40 modulus, in order."""
    npdt, code = _DTYPES[dtype]
    out = np.empty(n, dtype=npdt)
    _check(_load().oracle40_generate(a, j, n, code, _ptr(out)), "oracle40_generate")
    return out


def at40(a: int, idx, dtype: str = "f64") -> np.ndarray:
    """Variates at arbitrary positions under the 3^40 modulus, each from Eq. 2."""
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    npdt, code = _DTYPES[dtype]
    out = np.empty(idx.size, dtype=npdt)
    _check(_load().oracle40_at(a, _ptr(idx), idx.size, code, _ptr(out)), "oracle40_at")
    return out
