"""Python binding of ``libbcn_rng.so`` (include/bcn_rng.h).

Argument marshalling only: every variate is produced by the library's CUDA
kernels.  torch provides device memory and the current CUDA stream.  There is
no fallback: if the library is missing this module raises ImportError.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import _build

M = 3 ** 33
SEED_MIN = M + 100
SEED_MAX = 2 ** 53
PERIOD = 2 * 3 ** 32
MAX_N = 1 << 46

F64, F32, U64 = 0, 1, 2
_DTYPES = {
    "f64": (F64, torch.float64),
    "f32": (F32, torch.float32),
    "u64": (U64, torch.uint64),
}
STATUS = {0: "RNG_OK", 1: "RNG_EINVAL", 2: "RNG_ERANGE", 3: "RNG_ENOMEM",
          4: "RNG_ECUDA", 5: "RNG_ETIMEOUT", 6: "RNG_EBUSY"}
STEP = {"auto": 0, "barrett": 1, "montgomery": 2, "shared": 3, "lecuyer": 4,
        "barrett_classic": 5}
CONV = {"auto": 0, "int": 1, "fp64": 2}
LAYOUT = {"auto": 0, "tiled": 1, "direct": 2, "strided": 3}
SKIP = {"auto": 0, "table": 1, "sqmul": 2}


class RNGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Tune(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in
                ("step", "conv", "layout", "skip", "depth", "block", "grid", "unit",
                 "chains", "buffers")]


def make_tune(step="auto", conv="auto", layout="auto", skip="auto", depth=0, block=0,
              grid=0, unit=0, chains=0, buffers=0) -> Tune:
    """Launch tuning; zero / "auto" lets the library choose.  Results never
    depend on it, only speed does."""
    return Tune(STEP[step] if isinstance(step, str) else step,
                CONV[conv] if isinstance(conv, str) else conv,
                LAYOUT[layout] if isinstance(layout, str) else layout,
                SKIP[skip] if isinstance(skip, str) else skip,
                depth, block, grid, unit, chains, buffers)


class ServerConfig(ctypes.Structure):
    _fields_ = [("pool_bytes", ctypes.c_uint64), ("chunk_elems", ctypes.c_uint64),
                ("max_active", ctypes.c_uint32), ("max_items", ctypes.c_uint32),
                ("inflight", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("release_after_s", ctypes.c_double), ("tune", Tune),
                ("admit_bypass_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in
                ("submitted", "completed", "iterations", "items", "max_items_seen",
                 "peak_active", "peak_pool_bytes", "bytes_done", "pool_in_use", "pool_bytes",
                 "heavy_iterations", "admitted_out_of_order", "bypassed", "loop_gap_max_us",
                 "launch_max_us", "stage_max_us", "kernel_launch_max_us",
                 "event_record_max_us")]


def _load() -> ctypes.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(
            f"the CUDA library {path} is not built; run "
            "`python -m paper_1206_1187_gb300._build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    u64, u32, i32, vp, dbl = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                              ctypes.c_void_p, ctypes.c_double)
    tp = ctypes.POINTER(Tune)
    sig = {
        "rng_create": ([u64, ctypes.POINTER(vp)], i32),
        "rng_destroy": ([vp], i32),
        "rng_set_cuda_stream": ([vp, vp], i32),
        "rng_generate": ([vp, u64, i32, vp], i32),
        "rng_generate_tuned": ([vp, u64, i32, vp, tp], i32),
        "rng_skip": ([vp, u64], i32),
        "rng_generate_to_host": ([vp, u64, i32, vp, u64, u32], i32),
        "rng_get_state": ([vp, ctypes.POINTER(u64), ctypes.POINTER(u64)], i32),
        "rng_set_state": ([vp, u64, u64], i32),
        "rng_sync": ([vp], i32),
        "rng_generate_at": ([u64, u64, u64, i32, vp, vp, tp], i32),
        "rng40_generate_at": ([u64, u64, u64, i32, vp, vp, tp], i32),
        "rng40_resolve_tune": ([u64, i32, tp, tp], i32),
        "rng_fill_constant": ([u64, i32, dbl, vp, vp, tp], i32),
        "rng_last_error": ([], ctypes.c_char_p),
        "rng_resolve_tune": ([u64, i32, tp, tp], i32),
        "rng_version": ([], i32),
        "rng_parse_tune": ([ctypes.c_char_p, tp], i32),
        "rng_debug_fail_allocations": ([u32, u32], i32),
        "rng_server_latency_histogram": ([vp, ctypes.POINTER(u64)], i32),
        "rng_autotune_bulk": ([u64, i32, vp, vp, tp, u32, u32, tp,
                               ctypes.POINTER(ctypes.c_float)], i32),
        "rng_set_auto_tune": ([i32, tp], i32),
        "rng_batch_create": ([u32, vp, vp, vp, vp, vp, tp, ctypes.POINTER(vp)], i32),
        "rng_batch_launch": ([vp, vp], i32),
        "rng_batch_graph_launch": ([vp, vp], i32),
        "rng_batch_info": ([vp, ctypes.POINTER(u64), ctypes.POINTER(u64),
                            ctypes.POINTER(u64), tp], i32),
        "rng_batch_destroy": ([vp], i32),
        "rng_consume_mc": ([u64, u64, u64, u64, vp, vp, vp, vp, vp, tp], i32),
        "rng_consume_mc_totals": ([u64, u64, u64, u64, vp, vp, vp, vp, vp, vp, tp], i32),
        "rng_mc_round_totals": ([vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)], i32),
        "rng_batch_generate_noalloc": ([u32, vp, vp, vp, vp, vp, tp, vp], i32),
        "rng_device_api_check": ([u64, u64, u64, vp, vp, vp, u32, vp], i32),
        "rng_device_api_checksum": ([u64, u64, u64, i32, vp, u32, vp], i32),
        "rng_device_api_f32_runs": ([u64, u64, u64, vp, u32, vp], i32),
        "rng_server_create": ([ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)], i32),
        "rng_server_submit": ([vp, u64, u64, u64, i32, ctypes.POINTER(u64)], i32),
        "rng_server_cancel": ([vp, u64], i32),
        "rng_server_status": ([vp, u64, ctypes.POINTER(i32), ctypes.POINTER(dbl)], i32),
        "rng_server_wait": ([vp, u64, dbl], i32),
        "rng_server_read": ([vp, u64, vp, u64], i32),
        "rng_server_result_ptr": ([vp, u64, ctypes.POINTER(vp)], i32),
        "rng_server_release": ([vp, u64], i32),
        "rng_server_stats_get": ([vp, ctypes.POINTER(ServerStats)], i32),
        "rng_server_run_trace": ([vp, u32, vp, vp, vp, vp, vp, dbl, vp,
                                  ctypes.POINTER(dbl)], i32),
        "rng_server_destroy": ([vp], i32),
        "rng_pool_create": ([u64, u64, ctypes.POINTER(vp)], i32),
        "rng_pool_alloc": ([vp, u64, ctypes.POINTER(u64)], i32),
        "rng_pool_free": ([vp, u64], i32),
        "rng_pool_stats": ([vp] + [ctypes.POINTER(u64)] * 5, i32),
        "rng_pool_destroy": ([vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


def _check(rc: int) -> None:
    if rc != 0:
        raise RNGError(rc, lib.rng_last_error().decode(errors="replace"))


def _dtype(dtype: str):
    try:
        return _DTYPES[dtype]
    except KeyError:
        raise ValueError(f"dtype must be one of {sorted(_DTYPES)}") from None


def _out_tensor(n: int, dtype: str, out):
    code, tdt = _dtype(dtype)
    if out is None:
        out = torch.empty(n, dtype=tdt, device="cuda")
    else:
        if out.dtype != tdt or not out.is_cuda or not out.is_contiguous() or out.numel() < n:
            raise ValueError(f"out must be a contiguous CUDA {tdt} tensor with >= {n} elements")
    return code, out


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _tune_ptr(tune):
    if tune is None:
        return None
    if isinstance(tune, dict):
        tune = make_tune(**tune)
    return ctypes.byref(tune)


class Stream:
    """One generator stream: a seed (start index, Algorithm BB step 1) and a
    count of variates already produced.  Launches go to torch's current CUDA
    stream at each call unless `cuda_stream` is given."""

    def __init__(self, start_index: int):
        h = ctypes.c_void_p()
        _check(lib.rng_create(start_index, ctypes.byref(h)))
        self._h = h

    def close(self) -> None:
        if self._h:
            lib.rng_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind(self, stream) -> None:
        _check(lib.rng_set_cuda_stream(self._h, ctypes.c_void_p(_stream_handle(stream))))

    def generate(self, n: int, dtype: str = "f64", out=None, tune=None, stream=None):
        code, out = _out_tensor(n, dtype, out)
        self._bind(stream)
        _check(lib.rng_generate_tuned(self._h, n, code, ctypes.c_void_p(out.data_ptr()),
                                      _tune_ptr(tune)))
        return out

    def generate_into_ptr(self, n: int, dtype: str, ptr: int, tune=None, stream=None) -> None:
        code, _ = _dtype(dtype)
        self._bind(stream)
        _check(lib.rng_generate_tuned(self._h, n, code, ctypes.c_void_p(ptr), _tune_ptr(tune)))

    def generate_to_host(self, n: int, dtype: str = "f64", out=None, chunk_bytes: int = 0,
                         nbuf: int = 0, stream=None):
        """The next n variates into a host tensor (page-locked if `out` is None),
        generation and device-to-host copies pipelined; synchronous."""
        code, tdt = _dtype(dtype)
        if out is None:
            out = torch.empty(n, dtype=tdt, pin_memory=True)
        elif out.dtype != tdt or out.is_cuda or not out.is_contiguous() or out.numel() < n:
            raise ValueError(f"out must be a contiguous host {tdt} tensor with >= {n} elements")
        self._bind(stream)
        _check(lib.rng_generate_to_host(self._h, n, code, ctypes.c_void_p(out.data_ptr()),
                                        chunk_bytes, nbuf))
        return out

    def skip(self, k: int) -> None:
        _check(lib.rng_skip(self._h, k))

    @property
    def state(self) -> tuple[int, int]:
        a, c = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib.rng_get_state(self._h, ctypes.byref(a), ctypes.byref(c)))
        return a.value, c.value

    def set_state(self, start_index: int, count: int) -> None:
        _check(lib.rng_set_state(self._h, start_index, count))

    def sync(self) -> None:
        _check(lib.rng_sync(self._h))


def generate_at(start_index: int, offset: int, n: int, dtype: str = "f64", out=None,
                tune=None, stream=None):
    """Variates offset .. offset+n-1 of the sequence seeded with start_index."""
    code, out = _out_tensor(n, dtype, out)
    _check(lib.rng_generate_at(start_index, offset, n, code, ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(_stream_handle(stream)), _tune_ptr(tune)))
    return out


def generate_at_ptr(start_index: int, offset: int, n: int, dtype: str, ptr: int, tune=None,
                    stream=None) -> None:
    code, _ = _dtype(dtype)
    _check(lib.rng_generate_at(start_index, offset, n, code, ctypes.c_void_p(ptr),
                               ctypes.c_void_p(_stream_handle(stream)), _tune_ptr(tune)))


def generate40_at(start_index: int, offset: int, n: int, dtype: str = "f64", out=None,
                  tune=None, stream=None):
    """Variates offset .. offset+n-1 of the 3^40-modulus generator seeded with
    start_index (in [3^40+100, 2^64-1])."""
    code, out = _out_tensor(n, dtype, out)
    _check(lib.rng40_generate_at(start_index, offset, n, code, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(_stream_handle(stream)), _tune_ptr(tune)))
    return out


def resolve_tune40(n: int, dtype: str = "f64", tune=None) -> dict:
    code, _ = _dtype(dtype)
    res = Tune()
    _check(lib.rng40_resolve_tune(n, code, _tune_ptr(tune), ctypes.byref(res)))
    inv = lambda d, v: next((k for k, x in d.items() if x == v), v)
    return {"layout": inv(LAYOUT, res.layout), "depth": res.depth, "block": res.block,
            "grid": res.grid, "chains": res.chains, "buffers": res.buffers}


def fill_constant(n: int, dtype: str = "f64", value: float = 0.5, out=None, tune=None,
                  stream=None):
    """The write-ceiling probe: n copies of `value` through the tiled store path."""
    code, out = _out_tensor(n, dtype, out)
    _check(lib.rng_fill_constant(n, code, value, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(_stream_handle(stream)), _tune_ptr(tune)))
    return out


def resolve_tune(n: int, dtype: str = "f64", tune=None) -> dict:
    code, _ = _dtype(dtype)
    res = Tune()
    _check(lib.rng_resolve_tune(n, code, _tune_ptr(tune), ctypes.byref(res)))
    inv = lambda d, v: next((k for k, x in d.items() if x == v), v)
    return {"step": inv(STEP, res.step), "conv": inv(CONV, res.conv),
            "layout": inv(LAYOUT, res.layout), "skip": inv(SKIP, res.skip),
            "depth": res.depth, "block": res.block, "grid": res.grid, "chains": res.chains,
            "buffers": res.buffers}


def autotune_bulk(n: int, dtype: str, candidates, reps: int = 5, out=None, stream=None):
    """Time candidate tunings (list of Tune or dicts); returns (best, ms list)."""
    code, out = _out_tensor(n, dtype, out)
    cands = [c if isinstance(c, Tune) else make_tune(**c) for c in candidates]
    arr = (Tune * len(cands))(*cands)
    ms = (ctypes.c_float * len(cands))()
    best = Tune()
    _check(lib.rng_autotune_bulk(n, code, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(_stream_handle(stream)), arr, len(cands),
                                 reps, ctypes.byref(best), ms))
    return best, [float(x) for x in ms]


def set_auto_tune(dtype: str, tune) -> None:
    """Install `tune` as the default for the zero fields of later calls."""
    code, _ = _dtype(dtype)
    _check(lib.rng_set_auto_tune(code, _tune_ptr(tune)))


def tune_dict(t: Tune) -> dict:
    inv = lambda d, v: next((k for k, x in d.items() if x == v), v)
    return {"step": inv(STEP, t.step), "conv": inv(CONV, t.conv),
            "layout": inv(LAYOUT, t.layout), "skip": inv(SKIP, t.skip),
            "depth": t.depth, "block": t.block, "grid": t.grid, "chains": t.chains,
            "buffers": t.buffers}


def consume_mc(start_index: int, nblocks: int, length: int, block0: int = 0,
               per_block_hits: bool = True, tune=None, stream=None):
    """Fused Monte-Carlo consumer (no variates stored).  Returns
    (hits_total[1], hits[nblocks] or None, sum[nblocks], sumsq[nblocks]) as
    CUDA tensors, filled asynchronously on the stream."""
    total = torch.empty(1, dtype=torch.uint64, device="cuda")
    hits = torch.empty(nblocks, dtype=torch.uint64, device="cuda") if per_block_hits else None
    s1 = torch.empty(nblocks, dtype=torch.float64, device="cuda")
    s2 = torch.empty(nblocks, dtype=torch.float64, device="cuda")
    _check(lib.rng_consume_mc(start_index, block0, nblocks, length,
                              ctypes.c_void_p(total.data_ptr()),
                              ctypes.c_void_p(hits.data_ptr()) if hits is not None else None,
                              ctypes.c_void_p(s1.data_ptr()), ctypes.c_void_p(s2.data_ptr()),
                              ctypes.c_void_p(_stream_handle(stream)), _tune_ptr(tune)))
    return total, hits, s1, s2


def consume_mc_into(start_index: int, nblocks: int, length: int, total, hits, s1, s2,
                    block0: int = 0, tune=None, stream=None) -> None:
    """consume_mc into caller-provided CUDA tensors (hits may be None)."""
    _check(lib.rng_consume_mc(start_index, block0, nblocks, length,
                              ctypes.c_void_p(total.data_ptr()),
                              ctypes.c_void_p(hits.data_ptr()) if hits is not None else None,
                              ctypes.c_void_p(s1.data_ptr()), ctypes.c_void_p(s2.data_ptr()),
                              ctypes.c_void_p(_stream_handle(stream)), _tune_ptr(tune)))


MC_TOTAL_WORDS = 11


def consume_mc_totals(start_index: int, nblocks: int, length: int, block0: int = 0,
                      tune=None, stream=None):
    """consume_mc plus the call's exact totals: returns (hits_total[1],
    hits[nblocks], sum[nblocks], sumsq[nblocks], totals[11]) as CUDA tensors.
    totals holds 32-bit pieces of the exact sums over every block of the call
    (see rng_consume_mc_totals); word arrays of several calls or ranks add
    element by element, and mc_round_totals rounds the result."""
    total = torch.empty(1, dtype=torch.uint64, device="cuda")
    hits = torch.empty(nblocks, dtype=torch.uint64, device="cuda")
    s1 = torch.empty(nblocks, dtype=torch.float64, device="cuda")
    s2 = torch.empty(nblocks, dtype=torch.float64, device="cuda")
    words = torch.empty(MC_TOTAL_WORDS, dtype=torch.uint64, device="cuda")
    _check(lib.rng_consume_mc_totals(start_index, block0, nblocks, length,
                                     ctypes.c_void_p(total.data_ptr()),
                                     ctypes.c_void_p(hits.data_ptr()),
                                     ctypes.c_void_p(s1.data_ptr()),
                                     ctypes.c_void_p(s2.data_ptr()),
                                     ctypes.c_void_p(words.data_ptr()),
                                     ctypes.c_void_p(_stream_handle(stream)), _tune_ptr(tune)))
    return total, hits, s1, s2, words


def mc_round_totals(words) -> tuple[float, float]:
    """(sum, sumsq): the totals word array (host sequence of 11 non-negative
    integers below 2^64, e.g. several ranks' arrays added) rounded to nearest."""
    import numpy as np
    w = np.ascontiguousarray([int(x) for x in words], dtype=np.uint64)
    if w.size != MC_TOTAL_WORDS:
        raise ValueError(f"need {MC_TOTAL_WORDS} words, got {w.size}")
    s1, s2 = ctypes.c_double(), ctypes.c_double()
    _check(lib.rng_mc_round_totals(ctypes.c_void_p(w.ctypes.data), ctypes.byref(s1),
                                   ctypes.byref(s2)))
    return s1.value, s2.value


def device_api_check(start_index: int, offset: int, n: int, threads: int = 4096, stream=None,
                     states: bool = False):
    """Variates from a kernel written against bcn_device.cuh: (f64, f32)
    tensors, and the raw states as a third (uint64) when `states` is set."""
    f64 = torch.empty(n, dtype=torch.float64, device="cuda")
    f32 = torch.empty(n, dtype=torch.float32, device="cuda")
    st = torch.empty(n, dtype=torch.uint64, device="cuda") if states else None
    _check(lib.rng_device_api_check(start_index, offset, n, ctypes.c_void_p(f64.data_ptr()),
                                    ctypes.c_void_p(f32.data_ptr()),
                                    ctypes.c_void_p(st.data_ptr() if states else 0), threads,
                                    ctypes.c_void_p(_stream_handle(stream))))
    return (f64, f32, st) if states else (f64, f32)


def device_api_checksum(start_index: int, offset: int, n: int, threads: int = 1 << 18,
                        stream=None, dtype: str = "f64"):
    """Per-thread sums mod 2^64 of the bit patterns of variates consumed in
    registers by a kernel written against bcn_device.cuh (thread t takes
    [t*n/T, (t+1)*n/T); FP64 by next_f64, FP32 by f32_run in runs of 32); an
    int64 tensor holding the 64-bit words."""
    code, _ = _dtype(dtype)
    sums = torch.empty(threads, dtype=torch.int64, device="cuda")
    _check(lib.rng_device_api_checksum(start_index, offset, n, code,
                                       ctypes.c_void_p(sums.data_ptr()), threads,
                                       ctypes.c_void_p(_stream_handle(stream))))
    return sums


def device_api_f32_runs(start_index: int, offset: int, n: int, threads: int = 4096,
                        stream=None):
    """FP32 variates written by a kernel using bcn_device::f32_run (runs of 32,
    the remainder by next_f32)."""
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(lib.rng_device_api_f32_runs(start_index, offset, n, ctypes.c_void_p(out.data_ptr()),
                                       threads, ctypes.c_void_p(_stream_handle(stream))))
    return out


class Batch:
    """Many streams of uneven length in one persistent launch.

    starts, counts (and optional offsets) are integer sequences; dtypes a
    sequence of "f64"/"f32"/"u64"; outs a list of CUDA tensors (or None to
    allocate).  launch() / graph_launch() enqueue on torch's current stream."""

    def __init__(self, starts, counts, dtypes, outs=None, offsets=None, tune=None):
        import numpy as np
        n = len(starts)
        self.starts = np.ascontiguousarray(starts, dtype=np.uint64)
        self.counts = np.ascontiguousarray(counts, dtype=np.uint64)
        self.offsets = (np.ascontiguousarray(offsets, dtype=np.uint64)
                        if offsets is not None else None)
        self.dtypes = list(dtypes)
        codes = np.ascontiguousarray([_dtype(d)[0] for d in self.dtypes], dtype=np.uint8)
        if outs is None:
            outs = [torch.empty(int(c), dtype=_dtype(d)[1], device="cuda")
                    for c, d in zip(self.counts, self.dtypes)]
        self.outs = outs
        ptrs = (ctypes.c_void_p * n)(*[o.data_ptr() if o is not None else 0 for o in outs])
        self._ptrs = ptrs
        h = ctypes.c_void_p()
        _check(lib.rng_batch_create(
            n, ctypes.c_void_p(self.starts.ctypes.data),
            ctypes.c_void_p(self.offsets.ctypes.data) if self.offsets is not None else None,
            ctypes.c_void_p(self.counts.ctypes.data), ctypes.c_void_p(codes.ctypes.data),
            ptrs, _tune_ptr(tune), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None) -> None:
        _check(lib.rng_batch_launch(self._h, ctypes.c_void_p(_stream_handle(stream))))

    def graph_launch(self, stream=None) -> None:
        _check(lib.rng_batch_graph_launch(self._h, ctypes.c_void_p(_stream_handle(stream))))

    def info(self) -> dict:
        e, b, u = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        t = Tune()
        _check(lib.rng_batch_info(self._h, ctypes.byref(e), ctypes.byref(b), ctypes.byref(u),
                                  ctypes.byref(t)))
        d = tune_dict(t)
        d["unit"] = t.unit
        return {"elems": e.value, "bytes": b.value, "units": u.value, "tune": d}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.rng_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (see rng_server_create)."""

    STATES = {0: "queued", 1: "active", 2: "done", 3: "released", 4: "cancelled"}

    def __init__(self, pool_bytes: int, chunk_elems: int = 0, max_active: int = 0,
                 max_items: int = 0, inflight: int = 0, release_after_s: float = -1.0,
                 tune=None, admit_bypass_s: float = 0.0):
        cfg = ServerConfig(pool_bytes, chunk_elems, max_active, max_items, inflight, 0,
                           release_after_s, Tune(), admit_bypass_s)
        if tune is not None:
            cfg.tune = tune if isinstance(tune, Tune) else make_tune(**tune)
        h = ctypes.c_void_p()
        _check(lib.rng_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, start_index: int, offset: int, n: int, dtype: str = "f64") -> int:
        rid = ctypes.c_uint64()
        _check(lib.rng_server_submit(self._h, start_index, offset, n, _dtype(dtype)[0],
                                     ctypes.byref(rid)))
        return rid.value

    def cancel(self, rid: int) -> None:
        _check(lib.rng_server_cancel(self._h, rid))

    def status(self, rid: int):
        st, lat = ctypes.c_int(), ctypes.c_double()
        _check(lib.rng_server_status(self._h, rid, ctypes.byref(st), ctypes.byref(lat)))
        return self.STATES.get(st.value, st.value), lat.value

    def wait(self, rid: int, timeout_s: float = 60.0) -> None:
        _check(lib.rng_server_wait(self._h, rid, timeout_s))

    def read(self, rid: int, n: int, dtype: str):
        _, tdt = _dtype(dtype)
        out = torch.empty(n, dtype=tdt, device="cuda")
        _check(lib.rng_server_read(self._h, rid, ctypes.c_void_p(out.data_ptr()),
                                   out.numel() * out.element_size()))
        return out

    def release(self, rid: int) -> None:
        _check(lib.rng_server_release(self._h, rid))

    def latency_histogram(self):
        """Completed-request latency counts in quarter-octave bins: bin k
        covers [2^(k/4), 2^((k+1)/4)) microseconds (first and last bins open)."""
        import numpy as np
        counts = (ctypes.c_uint64 * HIST_BINS)()
        _check(lib.rng_server_latency_histogram(self._h, counts))
        return np.array(counts[:], dtype=np.uint64)

    def stats(self) -> dict:
        st = ServerStats()
        rc = lib.rng_server_stats_get(self._h, ctypes.byref(st))
        d = {f: getattr(st, f) for f, _ in ServerStats._fields_}
        d["status"] = rc
        return d

    def run_trace(self, arrivals, starts, counts, dtypes, offsets=None, timeout_s=120.0):
        """Replay a trace in real time; returns (latencies in seconds, wall seconds)."""
        import numpy as np
        n = len(arrivals)
        arr = np.ascontiguousarray(arrivals, dtype=np.float64)
        st = np.ascontiguousarray(starts, dtype=np.uint64)
        ct = np.ascontiguousarray(counts, dtype=np.uint64)
        dt = np.ascontiguousarray([_dtype(d)[0] for d in dtypes], dtype=np.uint8)
        of = np.ascontiguousarray(offsets, dtype=np.uint64) if offsets is not None else None
        lat = np.empty(n, dtype=np.float64)
        wall = ctypes.c_double()
        _check(lib.rng_server_run_trace(
            self._h, n, ctypes.c_void_p(arr.ctypes.data), ctypes.c_void_p(st.ctypes.data),
            ctypes.c_void_p(of.ctypes.data) if of is not None else None,
            ctypes.c_void_p(ct.ctypes.data), ctypes.c_void_p(dt.ctypes.data), timeout_s,
            ctypes.c_void_p(lat.ctypes.data), ctypes.byref(wall)))
        return lat, wall.value

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.rng_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pool:
    """The host-side pool sub-allocator the server admits requests with."""

    def __init__(self, capacity: int, align: int = 256):
        h = ctypes.c_void_p()
        _check(lib.rng_pool_create(capacity, align, ctypes.byref(h)))
        self._h = h

    def alloc(self, nbytes: int):
        off = ctypes.c_uint64()
        rc = lib.rng_pool_alloc(self._h, nbytes, ctypes.byref(off))
        if rc == 3:
            return None
        _check(rc)
        return off.value

    def free(self, off: int) -> None:
        _check(lib.rng_pool_free(self._h, off))

    def stats(self) -> dict:
        v = [ctypes.c_uint64() for _ in range(5)]
        _check(lib.rng_pool_stats(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("in_use", "peak", "live", "largest_free", "free_ranges"),
                        (x.value for x in v)))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib.rng_pool_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> int:
    return lib.rng_version()


HIST_BINS = 96  # RNG_SERVER_HIST_BINS


def parse_tune(text: str) -> dict:
    """A tuning from "key=value,..." text (the form BCN_RNG_TUNE takes)."""
    res = Tune()
    _check(lib.rng_parse_tune(text.encode(), ctypes.byref(res)))
    return {f: getattr(res, f) for f, _ in Tune._fields_}


def debug_fail_allocations(skip: int, count: int) -> None:
    """Testing hook: after `skip` more library allocations succeed, fail the
    next `count` as if the device had run out of memory (0, 0 turns it off)."""
    _check(lib.rng_debug_fail_allocations(skip, count))


@dataclass
class _Info:
    path: str = _build.LIB


library_info = _Info()
