"""Python binding of libtm.so, the GB300 (sm_103a) subsampled-circulant
template matcher (include/tm.h).

Argument marshalling only: every step of the matcher runs in the library's
CUDA kernels. torch tensors supply device memory and streams; their data
pointers and the current CUDA stream are handed to the C ABI as they are.
The library must have been built (`python -m paper_1509_04863_gb300._build`
or __graft_entry__.build()); importing this package fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

from . import _build

_LIB_PATH = _build.LIB

# ---------------------------------------------------------------- constants (tm.h)
TM_OK, TM_EINVAL, TM_ENOMEM, TM_ECUDA, TM_EBUSY, TM_ETIMEDOUT, TM_EAGAIN, TM_EUNSUPPORTED = range(8)
TM_I8_PM1, TM_BITS_PM1, TM_F16, TM_F32 = range(4)
TM_MODE_AUTO, TM_MODE_PAPER, TM_MODE_EXPLICIT = range(3)
TM_ALLOW_AMBIG = 0x1
TM_THM2_SAMPLING = 0x2
TM_FINE_PIECES = 0x8
TM_SERVE_FINE_PIECES = 0x1
TM_THREE_MODULI = 0x4
TM_FOUND, TM_EMPTY, TM_RESOLVED = 0, 1, 2
TM_RF_FULL_RESCORE = 0x100
TM_RF_DEVICE_ERROR = 0x200
TM_RF_SCORE_PENDING = 0x400
TM_RF_UNCERTIFIED = 0x800
TM_BATCH_KEEP_CORR = 0x1
TM_BATCH_HOST_INPUTS = 0x2
TM_BATCH_PIPELINED = 0x4

DTYPE_CODES = {"i8": TM_I8_PM1, "bits": TM_BITS_PM1, "f16": TM_F16, "f32": TM_F32}
MODE_CODES = {"auto": TM_MODE_AUTO, "paper": TM_MODE_PAPER, "explicit": TM_MODE_EXPLICIT}


class tm_plan_desc(C.Structure):
    _fields_ = [("N", C.c_int64), ("K", C.c_int32), ("xdtype", C.c_int32), ("mode", C.c_int32),
                ("M1", C.c_int32), ("M2", C.c_int32), ("flags", C.c_uint32), ("M3", C.c_int32),
                ("reserved", C.c_int32)]


class tm_plan_info(C.Structure):
    _fields_ = [("N", C.c_int64), ("K", C.c_int32), ("xdtype", C.c_int32), ("M1", C.c_int32),
                ("M2", C.c_int32), ("L1", C.c_int64), ("L2", C.c_int64), ("P", C.c_int32),
                ("max_cand", C.c_int32), ("M3", C.c_int32), ("reserved", C.c_int32), ("L3", C.c_int64)]


class tm_result(C.Structure):
    _fields_ = [("shift", C.c_int64), ("status", C.c_int32), ("n_cand", C.c_int32), ("m1", C.c_int32),
                ("m2", C.c_int32), ("r1", C.c_double), ("r2", C.c_double), ("score", C.c_double),
                ("m3", C.c_int32), ("reserved", C.c_int32), ("r3", C.c_double)]


class tm_query(C.Structure):
    _fields_ = [("x", C.c_void_p), ("t", C.c_void_p), ("N", C.c_int64), ("K", C.c_int32),
                ("xdtype", C.c_int32), ("mode", C.c_int32), ("M1", C.c_int32), ("M2", C.c_int32),
                ("flags", C.c_uint32), ("M3", C.c_int32), ("reserved", C.c_int32)]


RESULT_BYTES = C.sizeof(tm_result)
assert RESULT_BYTES == 64

# name -> (restype, argtypes)
_SIGS = {
    "tm_version": (C.c_char_p, []),
    "tm_last_error": (C.c_char_p, []),
    "tm_plan_create": (C.c_int, [C.POINTER(tm_plan_desc), C.POINTER(C.c_void_p)]),
    "tm_plan_get_info": (C.c_int, [C.c_void_p, C.POINTER(tm_plan_info)]),
    "tm_plan_destroy": (C.c_int, [C.c_void_p]),
    "tm_match": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tm_batch_create": (C.c_int, [C.POINTER(tm_query), C.c_int32, C.c_uint32, C.POINTER(C.c_void_p)]),
    "tm_batch_set_inputs": (C.c_int, [C.c_void_p, C.POINTER(tm_query), C.c_int32]),
    "tm_batch_fold": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tm_batch_correlate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "tm_batch_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "tm_batch_run_host": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p,
                                    C.c_void_p]),
    "tm_batch_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.POINTER(C.c_int32)]),
    "tm_batch_set_grid": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "tm_batch_get_grid": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "tm_batch_run_pipelined": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tm_batch_pipeline_flush": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tm_batch_graph_capture": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tm_batch_graph_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tm_batch_folds": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_int32)]),
    "tm_batch_corr": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "tm_batch_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "tm_batch_device_error": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "tm_batch_destroy": (C.c_int, [C.c_void_p]),
    "tm_match_batch": (C.c_int, [C.POINTER(tm_query), C.c_int32, C.c_void_p, C.c_void_p]),
    "tm_crt_candidates": (C.c_int32, [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                      C.POINTER(C.c_int64), C.c_int32]),
    "tm_struct_size": (C.c_int64, [C.c_int32]),
    "tm_match_noalloc": (C.c_int, [C.POINTER(tm_plan_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tm_selftest_wait_timeout": (C.c_int, [C.c_int64, C.POINTER(C.c_int32)]),
    "tm_fold_slice": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]),
    "tm_correlate_folds": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tm_score_slice": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32,
                                 C.c_void_p, C.c_void_p]),
}


def selftest_wait_timeout(limit_ns: int = 1_000_000) -> bool:
    """True when a device-side bounded wait on a barrier nothing arrives at
    gave up at its limit (tm_selftest_wait_timeout)."""
    g = C.c_int32(-1)
    _check(lib().tm_selftest_wait_timeout(int(limit_ns), C.byref(g)), "tm_selftest_wait_timeout")
    return g.value == 1

TM_NOALLOC_SCRATCH_BYTES = 4 << 20


def tm_match_noalloc(x, t, out, N: int, K: int, xdtype: str = "i8", mode: str = "paper", M1: int = 0, M2: int = 0,
                     allow_ambig: bool = False, thm2: bool = False, stream=None):
    """One query through the entry point that allocates no device memory
    (its scratch is a fixed array inside the library; calls must not
    overlap on the GPU). x, t, out: CUDA tensors as for Plan.match."""
    import torch
    d = tm_plan_desc(N, K, DTYPE_CODES[xdtype], MODE_CODES[mode], M1, M2, _plan_flags(allow_ambig, thm2), 0, 0)
    sp = _stream_ptr(stream) if (stream is not None or torch.cuda.is_available()) else None
    _check(lib().tm_match_noalloc(C.byref(d), x.data_ptr(), t.data_ptr(), out.data_ptr(), sp), "tm_match_noalloc")

_lib: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    """The loaded libtm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libtm.so not built at {_LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class TMError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().tm_last_error().decode(errors="replace")
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def _check(st: int, where: str):
    if st != TM_OK:
        raise TMError(st, where)


def _stream_ptr(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def tm_version() -> str:
    return lib().tm_version().decode()


def tm_crt_candidates(N: int, M1: int, M2: int, m1: int, m2: int, cap: int = 4096) -> List[int]:
    """Host closed-form S1 ∩ S2 (Algorithm 1 steps 8-9), ascending."""
    buf = (C.c_int64 * cap)()
    n = lib().tm_crt_candidates(N, M1, M2, m1, m2, buf, cap)
    if n < 0:
        raise ValueError("invalid CRT arguments")
    return [buf[i] for i in range(min(n, cap))]


class Plan:
    """tm_plan_create / tm_plan_get_info / tm_match / tm_plan_destroy."""

    def __init__(self, N: int, K: int, xdtype: str = "i8", mode: str = "paper", M1: int = 0, M2: int = 0,
                 allow_ambig: bool = False, thm2: bool = False, three: bool = False, M3: int = 0):
        d = tm_plan_desc(N, K, DTYPE_CODES[xdtype], MODE_CODES[mode], M1, M2, _plan_flags(allow_ambig, thm2, three),
                         M3, 0)
        h = C.c_void_p()
        _check(lib().tm_plan_create(C.byref(d), C.byref(h)), "tm_plan_create")
        self._h = h
        info = tm_plan_info()
        _check(lib().tm_plan_get_info(h, C.byref(info)), "tm_plan_get_info")
        self.info = {f: getattr(info, f) for f, _ in tm_plan_info._fields_}

    def match(self, x, t, out, stream=None):
        """x, t, out: CUDA tensors (out: >= 64 bytes, e.g. result_buffer(1))."""
        _check(lib().tm_match(self._h, x.data_ptr(), t.data_ptr(), out.data_ptr(), _stream_ptr(stream)), "tm_match")

    # ---- slices of one signal (tm_fold_slice / tm_correlate_folds / tm_score_slice)
    def fold_slice(self, x_slice, n0: int, length: int, y, stream=None):
        """Folds of entries [n0, n0+length) into y (CUDA tensor of 2P int32 or float32)."""
        xp = x_slice.data_ptr() if length > 0 else None
        _check(lib().tm_fold_slice(self._h, xp, int(n0), int(length), y.data_ptr(), _stream_ptr(stream)),
               "tm_fold_slice")

    def correlate_folds(self, y, t, out, stream=None):
        """Steps 4-8 from complete folds y; out: one-result buffer (CUDA)."""
        _check(lib().tm_correlate_folds(self._h, y.data_ptr(), t.data_ptr(), out.data_ptr(), _stream_ptr(stream)),
               "tm_correlate_folds")

    def score_slice(self, x_slice, n0: int, length: int, t, m, out, stream=None):
        """Partial exact scores over the slice for the int64 CUDA tensor of
        positions m into the float64 CUDA tensor out."""
        xp = x_slice.data_ptr() if length > 0 else None
        _check(lib().tm_score_slice(self._h, xp, int(n0), int(length), t.data_ptr(), m.data_ptr(), int(m.numel()),
                                    out.data_ptr(), _stream_ptr(stream)), "tm_score_slice")

    def close(self):
        if self._h:
            lib().tm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tm_plan_create(N, K, xdtype="i8", mode="paper", M1=0, M2=0, allow_ambig=False) -> Plan:
    return Plan(N, K, xdtype, mode, M1, M2, allow_ambig)


def _plan_flags(allow_ambig=False, thm2=False, three=False, fine_pieces=False) -> int:
    return (TM_ALLOW_AMBIG if allow_ambig else 0) | (TM_THM2_SAMPLING if thm2 else 0) | \
        (TM_THREE_MODULI if three else 0) | (TM_FINE_PIECES if fine_pieces else 0)


def _query_struct(x_ptr, t_ptr, N, K, xdtype, mode, M1=0, M2=0, allow_ambig=False, thm2=False, three=False,
                  M3=0, fine_pieces=False) -> tm_query:
    return tm_query(x_ptr, t_ptr, int(N), int(K), DTYPE_CODES[xdtype], MODE_CODES[mode], int(M1), int(M2),
                    _plan_flags(allow_ambig, thm2, three, fine_pieces), int(M3), 0)


def _event_ptr(ev):
    """The cudaEvent_t of a torch.cuda.Event (created on first use)."""
    if ev.cuda_event == 0:   # torch creates the event lazily at its first record
        ev.record()
    return ev.cuda_event


class Batch:
    """tm_batch_create / tm_batch_run / tm_batch_fold / tm_batch_correlate / ...

    `specs` is a list of dicts with keys x (CUDA tensor or None for host-input
    batches), t (CUDA tensor or None), N, K, xdtype, mode, and optionally M1,
    M2, allow_ambig, thm2, three, M3, fine_pieces."""

    def __init__(self, specs: Sequence[dict], keep_corr: bool = False, host_inputs: bool = False,
                 pipelined: bool = False):
        self.n = len(specs)
        self.specs = list(specs)
        arr = (tm_query * self.n)()
        for i, s in enumerate(specs):
            xp = s["x"].data_ptr() if s.get("x") is not None else None
            tp = s["t"].data_ptr() if s.get("t") is not None else None
            arr[i] = _query_struct(xp, tp, s["N"], s["K"], s.get("xdtype", "i8"), s.get("mode", "paper"),
                                   s.get("M1", 0), s.get("M2", 0), s.get("allow_ambig", False), s.get("thm2", False),
                                   s.get("three", False), s.get("M3", 0), s.get("fine_pieces", False))
        self._arr = arr
        flags = (TM_BATCH_KEEP_CORR if keep_corr else 0) | (TM_BATCH_HOST_INPUTS if host_inputs else 0) | \
            (TM_BATCH_PIPELINED if pipelined else 0)
        h = C.c_void_p()
        _check(lib().tm_batch_create(arr, self.n, flags, C.byref(h)), "tm_batch_create")
        self._h = h
        # per-query plan information (host-only planner calls)
        self.infos = [Plan(s["N"], s["K"], s.get("xdtype", "i8"), s.get("mode", "paper"), s.get("M1", 0),
                           s.get("M2", 0), s.get("allow_ambig", False), s.get("thm2", False), s.get("three", False),
                           s.get("M3", 0)).info for s in specs]

    def set_inputs(self, xs, ts):
        for i in range(self.n):
            self._arr[i].x = xs[i].data_ptr()
            self._arr[i].t = ts[i].data_ptr()
        _check(lib().tm_batch_set_inputs(self._h, self._arr, self.n), "tm_batch_set_inputs")

    def run(self, out, stream=None):
        _check(lib().tm_batch_run(self._h, out.data_ptr(), _stream_ptr(stream)), "tm_batch_run")

    def set_grid(self, fold_ctas: int = 0, corr_ctas: int = 0):
        """tm_batch_set_grid: at most fold_ctas fold CTAs (0: one per SM) and
        corr_ctas correlation CTAs at a time (0: one per query)."""
        _check(lib().tm_batch_set_grid(self._h, int(fold_ctas), int(corr_ctas)), "tm_batch_set_grid")

    def get_grid(self):
        """(fold_ctas, corr_ctas) set by set_grid or the autotuner (0: default)."""
        f, c = C.c_int32(), C.c_int32()
        _check(lib().tm_batch_get_grid(self._h, C.byref(f), C.byref(c)), "tm_batch_get_grid")
        return f.value, c.value

    def run_pipelined(self, out, stream=None, fold_events=None):
        """tm_batch_run_pipelined: fold now, correlate the previous call's
        folds beside it (into the previous call's `out`). fold_events: an
        optional pair of torch.cuda.Event recorded around the fold."""
        e0 = e1 = None
        if fold_events is not None:
            e0, e1 = (_event_ptr(e) for e in fold_events)
        _check(lib().tm_batch_run_pipelined(self._h, out.data_ptr(), _stream_ptr(stream), e0, e1),
               "tm_batch_run_pipelined")

    def flush(self, stream=None):
        """tm_batch_pipeline_flush: the last pipelined call's correlation."""
        _check(lib().tm_batch_pipeline_flush(self._h, _stream_ptr(stream)), "tm_batch_pipeline_flush")

    def fold(self, stream=None):
        _check(lib().tm_batch_fold(self._h, _stream_ptr(stream)), "tm_batch_fold")

    def correlate(self, out, stream=None):
        _check(lib().tm_batch_correlate(self._h, out.data_ptr(), _stream_ptr(stream)), "tm_batch_correlate")

    def autotune(self, stream=None, force: bool = False, grid: bool = False) -> dict:
        """tm_batch_autotune: pick the fold's stage ring per storage type
        (and, with grid=True on a pipelined batch, the split of the SMs
        between fold and correlation); returns {dtype: stage bytes}."""
        tiles = (C.c_int32 * 4)()
        flags = (1 if force else 0) | (2 if grid else 0)
        _check(lib().tm_batch_autotune(self._h, _stream_ptr(stream), flags, tiles), "tm_batch_autotune")
        names = {v: k for k, v in DTYPE_CODES.items()}
        return {names[d]: tiles[d] for d in range(4) if tiles[d]}

    def capture_graph(self, out):
        """Record one run writing to `out` as a CUDA graph (tm_batch_graph_capture)."""
        _check(lib().tm_batch_graph_capture(self._h, out.data_ptr()), "tm_batch_graph_capture")

    def launch_graph(self, stream=None):
        _check(lib().tm_batch_graph_launch(self._h, _stream_ptr(stream)), "tm_batch_graph_launch")

    def run_host(self, x_host: Sequence, t_host: Sequence, out_host, stream=None):
        """x_host, t_host: CPU tensors (pinned for speed); out_host: CPU tensor of n*RESULT_BYTES bytes."""
        xs = (C.c_void_p * self.n)(*[x.data_ptr() for x in x_host])
        ts = (C.c_void_p * self.n)(*[t.data_ptr() for t in t_host])
        _check(lib().tm_batch_run_host(self._h, xs, ts, out_host.data_ptr(), _stream_ptr(stream)),
               "tm_batch_run_host")

    def folds_ptr(self, i: int):
        p = C.c_void_p()
        f = C.c_int32()
        _check(lib().tm_batch_folds(self._h, i, C.byref(p), C.byref(f)), "tm_batch_folds")
        return p.value, bool(f.value)

    def _nmod(self, i: int) -> int:
        return 3 if self.infos[i]["M3"] else 2

    def folds(self, i: int):
        """Query i's folds as a device tensor view: [0, P) for M1, [P, 2P) for M2 (and [2P, 3P) for M3)."""
        ptr, is_float = self.folds_ptr(i)
        return device_view(ptr, self._nmod(i) * self.infos[i]["P"], "<f4" if is_float else "<i4")

    def corr(self, i: int):
        """Query i's FFT correlations (float32 view): r1 at [0, M1), r2 at [P, P+M2) (r3 at [2P, 2P+M3))."""
        return device_view(self.corr_ptr(i), self._nmod(i) * self.infos[i]["P"], "<f4")

    def corr_ptr(self, i: int):
        p = C.c_void_p()
        _check(lib().tm_batch_corr(self._h, i, C.byref(p)), "tm_batch_corr")
        return p.value

    def stats(self):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int64()
        _check(lib().tm_batch_stats(self._h, C.byref(a), C.byref(b), C.byref(c)), "tm_batch_stats")
        return {"launches_per_run": a.value, "fold_ctas": b.value, "workspace_bytes": c.value}

    def device_error(self, stream=None) -> int:
        e = C.c_int32()
        _check(lib().tm_batch_device_error(self._h, _stream_ptr(stream), C.byref(e)), "tm_batch_device_error")
        return e.value

    def close(self):
        if self._h:
            lib().tm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tm_batch_create(specs, keep_corr=False, host_inputs=False, pipelined=False) -> Batch:
    return Batch(specs, keep_corr, host_inputs, pipelined)


def tm_match_batch(specs, out, stream=None):
    arr = (tm_query * len(specs))()
    for i, s in enumerate(specs):
        arr[i] = _query_struct(s["x"].data_ptr(), s["t"].data_ptr(), s["N"], s["K"], s.get("xdtype", "i8"),
                               s.get("mode", "paper"), s.get("M1", 0), s.get("M2", 0), s.get("allow_ambig", False))
    _check(lib().tm_match_batch(arr, len(specs), out.data_ptr(), _stream_ptr(stream)), "tm_match_batch")


def decode_results(buf) -> List[dict]:
    """tm_result records from a CPU tensor / bytes-like of n*RESULT_BYTES bytes."""
    import numpy as np
    raw = bytes(buf.cpu().numpy().tobytes()) if hasattr(buf, "cpu") else bytes(buf)
    n = len(raw) // RESULT_BYTES
    out = []
    for i in range(n):
        r = tm_result.from_buffer_copy(raw[i * RESULT_BYTES:(i + 1) * RESULT_BYTES])
        out.append({f: getattr(r, f) for f, _ in tm_result._fields_})
    return out


class _CudaArray:
    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 2}


def device_view(ptr: int, n: int, typestr: str):
    """Zero-copy torch view of n elements of library-owned device memory."""
    import torch
    return torch.as_tensor(_CudaArray(ptr, n, typestr), device="cuda")


def result_buffer(n: int, device="cuda"):
    import torch
    return torch.zeros(n * RESULT_BYTES // 8, dtype=torch.int64, device=device)


# ---------------------------------------------------------------- server (tm_serve_*)
class tm_serve_cfg(C.Structure):
    _fields_ = [("n_streams", C.c_int32), ("max_batch", C.c_int32), ("queue_capacity", C.c_int32),
                ("flags", C.c_uint32), ("arena_bytes", C.c_int64), ("hbm_reserve_bytes", C.c_int64),
                ("fold_cache_bytes", C.c_int64), ("idle_spin_us", C.c_int64)]


class tm_result_tagged(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("reserved", C.c_int32), ("latency_us", C.c_double),
                ("r", tm_result)]


class tm_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("iterations", C.c_int64), ("pending", C.c_int64), ("in_flight", C.c_int64),
                ("mean_batch", C.c_double), ("p50_us", C.c_double), ("p99_us", C.c_double), ("max_us", C.c_double),
                ("fold_cache_hits", C.c_int64), ("fold_cache_misses", C.c_int64),
                ("queue_us", C.c_double), ("host_us", C.c_double), ("device_us", C.c_double)]


TM_SERVE_SIGNAL_DEVICE = 0x1
_SIGS.update({
    "tm_serve_create": (C.c_int, [C.POINTER(tm_serve_cfg), C.POINTER(C.c_void_p)]),
    "tm_serve_register_signal": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_uint32,
                                           C.POINTER(C.c_int32)]),
    "tm_serve_submit_many": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                         C.c_uint32, C.c_void_p]),
    "tm_serve_submit": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                  C.c_uint32, C.c_uint64]),
    "tm_serve_poll": (C.c_int32, [C.c_void_p, C.POINTER(tm_result_tagged), C.c_int32, C.c_int64]),
    "tm_serve_stats_get": (C.c_int, [C.c_void_p, C.POINTER(tm_serve_stats)]),
    "tm_serve_destroy": (C.c_int, [C.c_void_p]),
})


class Server:
    """tm_serve_create / register_signal / submit / poll / stats / destroy."""

    def __init__(self, n_streams: int = 2, max_batch: int = 512, queue_capacity: int = 65536,
                 arena_bytes: int = 0, hbm_reserve_bytes: int = 0, fold_cache_bytes: int = 0,
                 idle_spin_us: int = 0, fine_pieces: bool = False):
        L = lib()
        cfg = tm_serve_cfg(n_streams, max_batch, queue_capacity, TM_SERVE_FINE_PIECES if fine_pieces else 0,
                           arena_bytes, hbm_reserve_bytes, fold_cache_bytes, idle_spin_us)
        h = C.c_void_p()
        _check(L.tm_serve_create(C.byref(cfg), C.byref(h)), "tm_serve_create")
        self._h = h
        self._keep = []

    def register_signal(self, x, N: int, xdtype: str = "i8") -> int:
        """x: numpy array / CPU tensor (copied to the device) or CUDA tensor (used in place)."""
        import numpy as np
        sid = C.c_int32()
        if hasattr(x, "is_cuda") and x.is_cuda:
            self._keep.append(x)
            st = lib().tm_serve_register_signal(self._h, x.data_ptr(), N, DTYPE_CODES[xdtype],
                                                TM_SERVE_SIGNAL_DEVICE, C.byref(sid))
        else:
            arr = np.ascontiguousarray(x.numpy() if hasattr(x, "numpy") else x)
            st = lib().tm_serve_register_signal(self._h, arr.ctypes.data, N, DTYPE_CODES[xdtype], 0, C.byref(sid))
        _check(st, "tm_serve_register_signal")
        return sid.value

    def submit(self, sig_id: int, t, tag: int, mode: str = "paper", M1: int = 0, M2: int = 0,
               allow_ambig: bool = False, thm2: bool = False, three: bool = False) -> int:
        """Queue one request; returns the status (TM_OK, TM_EAGAIN, ...) without raising for TM_EAGAIN."""
        import numpy as np
        tt = np.ascontiguousarray(t, dtype=np.float32)
        st = lib().tm_serve_submit(self._h, sig_id, tt.ctypes.data, int(tt.shape[0]), MODE_CODES[mode], M1, M2,
                                   _plan_flags(allow_ambig, thm2, three), tag)
        if st not in (TM_OK, TM_EAGAIN):
            raise TMError(st, "tm_serve_submit")
        return st

    def submit_many(self, sig_ids, ts, tags, mode: str = "paper", allow_ambig: bool = False) -> int:
        """tm_serve_submit_many: queue len(sig_ids) requests in one call
        (ts: float32 numpy arrays, kept alive by the caller until the call
        returns); returns how many were queued."""
        import numpy as np
        n = len(sig_ids)
        ids = (C.c_int32 * n)(*[int(v) for v in sig_ids])
        tps = (C.c_void_p * n)(*[t.ctypes.data for t in ts])
        ks = (C.c_int32 * n)(*[int(t.shape[0]) for t in ts])
        tg = (C.c_uint64 * n)(*[int(v) for v in tags])
        for t in ts:
            assert t.dtype == np.float32 and t.flags["C_CONTIGUOUS"]
        k = lib().tm_serve_submit_many(self._h, n, ids, tps, ks, MODE_CODES[mode], _plan_flags(allow_ambig), tg)
        if k < 0:
            raise TMError(-k, "tm_serve_submit_many")
        return k

    def submit_many_arrays(self, sig_ids, t_ptrs, ks, tags, mode: str = "paper", allow_ambig: bool = False) -> int:
        """tm_serve_submit_many with the request fields as contiguous numpy
        arrays (int32 sig_ids, uint64 template addresses of float32 data,
        int32 lengths, uint64 tags): no per-request Python work, for clients
        that submit at high rates. Returns how many were queued."""
        import numpy as np
        n = int(sig_ids.shape[0])
        for a, dt in ((sig_ids, np.int32), (t_ptrs, np.uint64), (ks, np.int32), (tags, np.uint64)):
            assert a.dtype == dt and a.flags["C_CONTIGUOUS"] and a.shape[0] == n
        k = lib().tm_serve_submit_many(self._h, n, sig_ids.ctypes.data, t_ptrs.ctypes.data, ks.ctypes.data,
                                       MODE_CODES[mode], _plan_flags(allow_ambig), tags.ctypes.data)
        if k < 0:
            raise TMError(-k, "tm_serve_submit_many")
        return k

    def poll_array(self, max_results: int = 4096, timeout_us: int = 0):
        """tm_serve_poll into a numpy structured array (fields tag, status,
        latency_us and r, the tm_result fields): no per-result Python work."""
        import numpy as np
        buf = (tm_result_tagged * max_results)()
        k = lib().tm_serve_poll(self._h, buf, max_results, timeout_us)
        if k < 0:
            raise TMError(-k, "tm_serve_poll")
        return np.ctypeslib.as_array(buf)[:k].copy()

    def poll(self, max_results: int = 1024, timeout_us: int = 0):
        buf = (tm_result_tagged * max_results)()
        k = lib().tm_serve_poll(self._h, buf, max_results, timeout_us)
        if k < 0:
            raise TMError(-k, "tm_serve_poll")
        out = []
        for i in range(k):
            r = buf[i]
            d = {f: getattr(r.r, f) for f, _ in tm_result._fields_}
            d.update(tag=r.tag, req_status=r.status, latency_us=r.latency_us)
            out.append(d)
        return out

    def stats(self) -> dict:
        s = tm_serve_stats()
        _check(lib().tm_serve_stats_get(self._h, C.byref(s)), "tm_serve_stats_get")
        return {f: getattr(s, f) for f, _ in tm_serve_stats._fields_}

    def close(self):
        if self._h:
            lib().tm_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
