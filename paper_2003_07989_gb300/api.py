"""Python API over librpp.so: the same entry points as include/rpp.h.

Argument marshalling only: every step of the barcode computation runs in the
library (CUDA kernels and its native host code). Inputs may be torch tensors
(CUDA or CPU) or numpy arrays; CUDA tensors are read in place on torch's
current stream.
"""
from __future__ import annotations

import ctypes as C
import math
import threading
from dataclasses import dataclass, field

import numpy as np

from . import _native as N

_ctx_lock = threading.Lock()
_contexts: dict = {}


def _torch():
    import torch
    return torch


class Context:
    """A library context on one CUDA device (rpp_context_create). ``record``
    selects intermediate arrays to keep in results (RPP_RECORD_* flags)."""

    def __init__(self, device: int = 0, mem_budget: int = 0, record: int = 0):
        L = N.lib()
        h = C.c_void_p()
        N.check(L.rpp_context_create(device, mem_budget, C.byref(h)), "rpp_context_create")
        self.handle = h
        self.device = device
        self.record = record
        if record:
            N.check(L.rpp_context_set_record(h, record), "rpp_context_set_record")

    def set_batch(self, fused: bool = True, autotune: bool = True):
        """rpp_context_set_batch: fused=False runs batched clouds one at a time."""
        N.check(N.lib().rpp_context_set_batch(self.handle, int(fused), int(autotune)),
                "rpp_context_set_batch")

    def set_device_reduce(self, mode=1):
        """rpp_context_set_device_reduce: batched clouds of <= 512 points also
        reduce their short column walks on the device, beside the host (1 or
        True); reduce every walk on the device, long ones as level sweeps, with
        the host waiting for the results (2 or "wait"); or reduce on the host
        only (0 or False, the context's default)."""
        m = 2 if mode == "wait" else int(mode)
        N.check(N.lib().rpp_context_set_device_reduce(self.handle, m),
                "rpp_context_set_device_reduce")

    def set_sparse(self, mode: int = 0):
        """rpp_context_set_sparse: 0 chooses the thresholded construction of
        dimensions >= 2 by edge density, 1 always takes it, 2 never."""
        N.check(N.lib().rpp_context_set_sparse(self.handle, int(mode)), "rpp_context_set_sparse")

    def batch_tuning(self, nmax: int):
        """(threads, lanes per column) the autotuner chose for a size bucket,
        (0, 0) if it has not run."""
        t, g = C.c_int32(), C.c_int32()
        N.check(N.lib().rpp_context_batch_tuning(self.handle, nmax, C.byref(t), C.byref(g)),
                "rpp_context_batch_tuning")
        return t.value, g.value

    def close(self):
        if self.handle:
            N.lib().rpp_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_context(device: int = 0) -> Context:
    with _ctx_lock:
        if device not in _contexts:
            _contexts[device] = Context(device)
        return _contexts[device]


@dataclass
class Barcodes:
    """Per dimension q: intervals[q] float32 [k, 2] (birth, death; death = inf
    for essential classes) sorted by (birth, death), and critical[q] int32 [k, 4]
    (bu, bv, du, dv): the youngest edge of the birth and of the death simplex.
    stats: the call's counters and stage times (a dict, built on first use)."""
    intervals: list = field(default_factory=list)
    critical: list = field(default_factory=list)
    columns: dict = field(default_factory=dict)   # p -> (diam, cidx) when recorded
    apparent: dict = field(default_factory=dict)  # p -> (sigma, tau) when recorded
    _raw_stats: object = None
    _stats: dict = None

    @property
    def stats(self) -> dict:
        if self._stats is None:
            self._stats = _stats_dict(self._raw_stats) if self._raw_stats is not None else {}
        return self._stats

    def __getitem__(self, q):
        return self.intervals[q]


def _stats_dict(s: N.Stats) -> dict:
    out = {}
    for name, _ in N.Stats._fields_:
        v = getattr(s, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


def _take_result(h, with_stats=True) -> Barcodes:
    """Copy a result out of the library (and free it)."""
    L = N.lib()
    try:
        b = Barcodes()
        st = N.Stats()
        N.check(L.rpp_result_stats(h, C.byref(st)), "rpp_result_stats")
        for q in range(st.max_dim + 1):
            k = L.rpp_result_count(h, q)
            if k > 0:
                iv = np.ctypeslib.as_array(C.cast(L.rpp_result_intervals(h, q),
                                                  C.POINTER(C.c_float)), shape=(k * 2,))
                cr = np.ctypeslib.as_array(C.cast(L.rpp_result_critical(h, q),
                                                  C.POINTER(C.c_int32)), shape=(k * 4,))
                b.intervals.append(iv.reshape(k, 2).copy())
                b.critical.append(cr.reshape(k, 4).copy())
            else:
                b.intervals.append(np.zeros((0, 2), np.float32))
                b.critical.append(np.zeros((0, 4), np.int32))
        if with_stats:
            b._raw_stats = st
        for p in range(1, st.max_dim + 1):
            dp, ip = C.POINTER(C.c_float)(), C.POINTER(C.c_uint64)()
            m = L.rpp_result_columns(h, p, C.byref(dp), C.byref(ip))
            if m >= 0:
                b.columns[p] = (np.ctypeslib.as_array(dp, shape=(m,)).copy() if m else
                                np.zeros(0, np.float32),
                                np.ctypeslib.as_array(ip, shape=(m,)).copy() if m else
                                np.zeros(0, np.uint64))
            sp, tp = C.POINTER(C.c_uint64)(), C.POINTER(C.c_uint64)()
            m = L.rpp_result_apparent(h, p, C.byref(sp), C.byref(tp))
            if m >= 0:
                b.apparent[p] = (np.ctypeslib.as_array(sp, shape=(m,)).copy() if m else
                                 np.zeros(0, np.uint64),
                                 np.ctypeslib.as_array(tp, shape=(m,)).copy() if m else
                                 np.zeros(0, np.uint64))
    finally:
        L.rpp_result_free(h)
    return b


def _take_results(handles) -> list:
    """Copy many results out of the library in a few calls (rpp_results_*) and
    free them; the per-result arrays are views of one array per dimension."""
    L = N.lib()
    B = len(handles)
    arr = (C.c_void_p * B)(*handles)
    try:
        stats = (N.Stats * B)()
        N.check(L.rpp_results_stats(arr, B, stats), "rpp_results_stats")
        top = max((s.max_dim for s in stats), default=-1)
        per_dim = []
        for q in range(top + 1):
            offs = np.zeros(B + 1, np.int64)
            N.check(L.rpp_results_gather(arr, B, q, offs.ctypes.data, None, None),
                    "rpp_results_gather")
            tot = int(offs[-1])
            iv = np.empty((tot, 2), np.float32)
            cr = np.empty((tot, 4), np.int32)
            N.check(L.rpp_results_gather(arr, B, q, offs.ctypes.data, iv.ctypes.data,
                                         cr.ctypes.data), "rpp_results_gather")
            o = offs.tolist()
            per_dim.append(([iv[o[i]:o[i + 1]] for i in range(B)],
                            [cr[o[i]:o[i + 1]] for i in range(B)]))
        out = []
        for i in range(B):
            b = Barcodes()
            b._raw_stats = stats[i]
            for q in range(stats[i].max_dim + 1):
                b.intervals.append(per_dim[q][0][i])
                b.critical.append(per_dim[q][1][i])
            out.append(b)
    finally:
        L.rpp_results_free(arr, B)
    return out


def _as_input(data):
    """(pointer, keepalive, is_cuda, device) for a tensor or array of float32."""
    try:
        torch = _torch()
        if isinstance(data, torch.Tensor):
            t = data.detach()
            if t.dtype != torch.float32:
                t = t.float()
            t = t.contiguous()
            return t.data_ptr(), t, t.is_cuda, (t.device.index if t.is_cuda else None)
    except ImportError:
        pass
    a = np.ascontiguousarray(data, dtype=np.float32)
    return a.ctypes.data, a, False, None


def _stream_ptr(stream, is_cuda):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    if is_cuda:
        return _torch().cuda.current_stream().cuda_stream
    return None


def rpp_barcodes(data, max_dim: int = 1, threshold: float = math.inf, kind: str = "points",
                 quantile: float | None = None, stream=None, context: Context | None = None
                 ) -> Barcodes:
    """Barcodes of dims 0..max_dim of the Vietoris-Rips filtration of a point
    cloud (n x dim) or of a distance matrix (n x n, kind="distances")."""
    ptr, keep, is_cuda, dev = _as_input(data)
    ctx = context or default_context(dev or 0)
    kd = N.RPP_INPUT_POINTS if kind == "points" else N.RPP_INPUT_DISTANCES
    n = int(keep.shape[0])
    dim = int(keep.shape[1]) if kd == N.RPP_INPUT_POINTS else 0
    s = _stream_ptr(stream, is_cuda)
    h = C.c_void_p()
    L = N.lib()
    if quantile is not None:
        rc = L.rpp_barcodes_quantile(ctx.handle, ptr, kd, n, dim, max_dim, quantile, s, C.byref(h))
    else:
        rc = L.rpp_barcodes(ctx.handle, ptr, kd, n, dim, max_dim, threshold, s, C.byref(h))
    N.check(rc, "rpp_barcodes")
    return _take_result(h.value)


def rpp_apparent_census(data, kind: str = "points", stream=None,
                        context: Context | None = None) -> dict:
    """Dimension-1 apparent-pair census of the full filtration (no threshold,
    no enclosing-radius cut): the apparent-pair pass without the reduction.
    Returns the call's counters; the apparent fraction is
    stats["apparent"][1] / stats["candidates"][1]."""
    ptr, keep, is_cuda, dev = _as_input(data)
    ctx = context or default_context(dev or 0)
    kd = N.RPP_INPUT_POINTS if kind == "points" else N.RPP_INPUT_DISTANCES
    n = int(keep.shape[0])
    dim = int(keep.shape[1]) if kd == N.RPP_INPUT_POINTS else 0
    st = N.Stats()
    N.check(N.lib().rpp_apparent_census(ctx.handle, ptr, kd, n, dim,
                                        _stream_ptr(stream, is_cuda), C.byref(st)),
            "rpp_apparent_census")
    return _stats_dict(st)


def rpp_filtration(data, p: int, threshold: float = math.inf, kind: str = "points",
                   out=None, stream=None, context: Context | None = None):
    """Dimension-p columns without clearing (rpp_filtration): every p-simplex
    with diameter <= min(threshold, enclosing radius), in coboundary order.

    out=None returns host arrays (diam float32[m], cidx uint64[m]) and the
    counters; out=False leaves the columns in the library's workspace and
    returns only (None, None, stats) (for timing); out=(diam, cidx) takes two
    caller tensors (device or host) of equal capacity."""
    ptr, keep, is_cuda, dev = _as_input(data)
    ctx = context or default_context(dev or 0)
    kd = N.RPP_INPUT_POINTS if kind == "points" else N.RPP_INPUT_DISTANCES
    n = int(keep.shape[0])
    dim = int(keep.shape[1]) if kd == N.RPP_INPUT_POINTS else 0
    s = _stream_ptr(stream, is_cuda)
    L = N.lib()
    count = C.c_int64(-1)
    st = N.Stats()
    if out is False:
        N.check(L.rpp_filtration(ctx.handle, ptr, kd, n, dim, p, threshold, s, None, None, 0,
                                 C.byref(count), C.byref(st)), "rpp_filtration")
        return None, None, _stats_dict(st)
    if out is None:
        cap = math.comb(n, p + 1)
        diam = np.empty(max(cap, 1), np.float32)
        cidx = np.empty(max(cap, 1), np.uint64)
        dptr, iptr = diam.ctypes.data, cidx.ctypes.data
    else:
        diam, cidx = out
        cap = int(diam.shape[0])
        dptr, iptr = diam.data_ptr(), cidx.data_ptr()
    N.check(L.rpp_filtration(ctx.handle, ptr, kd, n, dim, p, threshold, s, dptr, iptr, cap,
                             C.byref(count), C.byref(st)), "rpp_filtration")
    k = count.value
    return diam[:k], cidx[:k], _stats_dict(st)


def rpp_distance_matrix(points, stream=None, context: Context | None = None) -> np.ndarray:
    """The library's float32 distance matrix of a point cloud (host copy)."""
    ptr, keep, is_cuda, dev = _as_input(points)
    ctx = context or default_context(dev or 0)
    n, dim = int(keep.shape[0]), int(keep.shape[1])
    out = np.zeros((n, n), dtype=np.float32)
    N.check(N.lib().rpp_distance_matrix(ctx.handle, ptr, n, dim, out.ctypes.data,
                                        _stream_ptr(stream, is_cuda)), "rpp_distance_matrix")
    return out


def rpp_l2_read_probe(buf, reps: int, blocks: int, sink, stream=None) -> None:
    """Queue the L2 read-bandwidth probe (rpp_l2_read_probe): read the CUDA
    tensor `buf` (16-byte aligned, nbytes a multiple of 16) `reps` times with
    L2-only loads over `blocks` blocks of 512 threads, adding the sum of its
    32-bit words (mod 2^32) to the one-element int32/uint32 CUDA tensor
    `sink`. The caller times the launch on `stream`."""
    if not (getattr(buf, "is_cuda", False) and getattr(sink, "is_cuda", False)):
        raise ValueError("rpp_l2_read_probe: buf and sink must be CUDA tensors")
    N.check(N.lib().rpp_l2_read_probe(buf.data_ptr(), buf.numel() * buf.element_size(),
                                      int(reps), int(blocks), sink.data_ptr(),
                                      _stream_ptr(stream, True)),
            "rpp_l2_read_probe")


def rpp_barcodes_batched(clouds, max_dim: int = 1, thresholds=None, quantiles=None,
                         stream=None, context: Context | None = None) -> list:
    """Barcodes of many clouds in one call (rpp_barcodes_batched)."""
    items = [_as_input(c) for c in clouds]
    B = len(items)
    dev = next((d for _, _, cu, d in items if cu), 0)
    ctx = context or default_context(dev or 0)
    ptrs = (C.c_void_p * B)(*[p for p, _, _, _ in items])
    ns = (C.c_int64 * B)(*[int(k.shape[0]) for _, k, _, _ in items])
    dims = (C.c_int32 * B)(*[int(k.shape[1]) for _, k, _, _ in items])
    th = (C.c_float * B)(*thresholds) if thresholds is not None else None
    qs = (C.c_double * B)(*quantiles) if quantiles is not None else None
    outs = (C.c_void_p * B)()
    s = _stream_ptr(stream, any(cu for _, _, cu, _ in items))
    N.check(N.lib().rpp_barcodes_batched(ctx.handle, B, ptrs, ns, dims, max_dim, th, qs, s, outs),
            "rpp_barcodes_batched")
    if ctx.record & (N.RPP_RECORD_COLUMNS | N.RPP_RECORD_APPARENT):
        return [_take_result(outs[i]) for i in range(B)]
    return _take_results([outs[i] for i in range(B)])


class Server:
    """Continuous-batching server (rpp_server_*): submit clouds as they arrive,
    poll for results."""

    def __init__(self, max_slots: int = 8, device_bytes: int = 0, context: Context | None = None,
                 max_batch: int = 64):
        self.ctx = context or default_context(0)
        cfg = N.ServerConfig(max_slots, device_bytes, 0, max_batch)
        h = C.c_void_p()
        N.check(N.lib().rpp_server_create(self.ctx.handle, C.byref(cfg), C.byref(h)),
                "rpp_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, points, max_dim: int = 1, threshold: float = math.inf,
               quantile: float = 0.0) -> int:
        ptr, keep, _, _ = _as_input(points)
        t = C.c_uint64()
        N.check(N.lib().rpp_server_submit(self.handle, ptr, int(keep.shape[0]),
                                          int(keep.shape[1]), max_dim, threshold, quantile,
                                          C.byref(t)), "rpp_server_submit")
        return int(t.value)

    def poll(self, ticket: int, timeout_ms: int = -1):
        """Barcodes of a finished request; None if still running after timeout."""
        h = C.c_void_p()
        rc = N.lib().rpp_server_poll(self.handle, ticket, timeout_ms, C.byref(h))
        if rc == N.RPP_E_TIMEOUT:
            return None
        N.check(rc, "rpp_server_poll")
        return _take_result(h.value)

    def next(self, timeout_ms: int = -1):
        """(ticket, Barcodes) of the next finished request in completion order
        (rpp_server_next); None if none finished within timeout_ms."""
        t, h = C.c_uint64(), C.c_void_p()
        rc = N.lib().rpp_server_next(self.handle, timeout_ms, C.byref(t), C.byref(h))
        if rc == N.RPP_E_TIMEOUT:
            return None
        N.check(rc, "rpp_server_next")
        return int(t.value), _take_result(h.value)

    def close(self):
        if self.handle:
            N.lib().rpp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
