"""ctypes wrapper around the C oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this module; the GPU library never does. Every function here cites
the paper passage its C counterpart follows (see ``rpp_oracle.c``).
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

MODE_HOM, MODE_COHOM, MODE_COHOM_CLEAR = 0, 1, 2
MAXV = 8


class _Pair(C.Structure):
    _fields_ = [("dim", C.c_int32), ("birth", C.c_float), ("death", C.c_float),
                ("bv", C.c_int32 * MAXV), ("dv", C.c_int32 * MAXV)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        f32p, i32p = C.POINTER(C.c_float), C.POINTER(C.c_int32)
        L.oracle_distance_matrix.argtypes = [f32p, C.c_int64, C.c_int32, f32p]
        L.oracle_distance_matrix.restype = C.c_int
        L.oracle_enclosing_radius.argtypes = [f32p, C.c_int64]
        L.oracle_enclosing_radius.restype = C.c_float
        L.oracle_distance_quantile.argtypes = [f32p, C.c_int64, C.c_double]
        L.oracle_distance_quantile.restype = C.c_float
        L.oracle_barcodes.argtypes = [f32p, C.c_int64, C.c_int32, C.c_float, C.c_int32]
        L.oracle_barcodes.restype = C.c_void_p
        L.oracle_kruskal.argtypes = [f32p, C.c_int64, C.c_float]
        L.oracle_kruskal.restype = C.c_void_p
        L.oracle_result_count.argtypes = [C.c_void_p]
        L.oracle_result_count.restype = C.c_int64
        L.oracle_result_pairs.argtypes = [C.c_void_p]
        L.oracle_result_pairs.restype = C.POINTER(_Pair)
        L.oracle_result_additions.argtypes = [C.c_void_p]
        L.oracle_result_additions.restype = C.c_int64
        L.oracle_result_free.argtypes = [C.c_void_p]
        L.oracle_result_free.restype = None
        L.oracle_columns.argtypes = [f32p, C.c_int64, C.c_int32, C.c_float, f32p, i32p, C.c_int64]
        L.oracle_columns.restype = C.c_int64
        L.oracle_apparent_one.argtypes = [f32p, C.c_int64, C.c_int32, C.c_float, i32p, i32p]
        L.oracle_apparent_one.restype = C.c_int
        L.oracle_apparent_pairs.argtypes = [f32p, C.c_int64, C.c_int32, C.c_float, i32p, i32p,
                                            C.c_int64]
        L.oracle_apparent_pairs.restype = C.c_int64
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def distance_matrix(points: np.ndarray) -> np.ndarray:
    """Euclidean distance matrix in float32 with the fixed operation order
    (sum of squared differences left to right, no fused multiply-add, correctly
    rounded square root). The paper's input is the matrix itself (Sec. 2)."""
    X, xp = _f32(points)
    n, dim = X.shape
    D = np.zeros((n, n), dtype=np.float32)
    rc = lib().oracle_distance_matrix(xp, n, dim, D.ctypes.data_as(C.POINTER(C.c_float)))
    assert rc == 0
    return D


def enclosing_radius(D: np.ndarray) -> float:
    """min_x max_y d(x, y) (Sec. "Filtering Out Simplices by Diameter Equal to
    the Enclosing Radius")."""
    D, dp = _f32(D)
    return float(np.float32(lib().oracle_enclosing_radius(dp, D.shape[0])))


def distance_quantile(D: np.ndarray, q: float) -> float:
    """Nearest-rank q-quantile of the pairwise distances: the ceil(q m)-th
    smallest of the m = C(n,2) entries above the diagonal."""
    D, dp = _f32(D)
    return float(np.float32(lib().oracle_distance_quantile(dp, D.shape[0], q)))


@dataclass
class Pairs:
    """Every persistence pair (zero-length included) of a filtration."""
    dim: np.ndarray      # int32 [m]
    birth: np.ndarray    # float32 [m]
    death: np.ndarray    # float32 [m], +inf for essential classes
    bverts: np.ndarray   # int32 [m, 8] birth simplex, decreasing, -1 padded
    dverts: np.ndarray   # int32 [m, 8] death simplex, -1 padded
    additions: int       # column additions the reduction performed

    def barcode(self, q: int) -> np.ndarray:
        """Nonzero intervals of dimension q, sorted by (birth, death), float32 [k, 2]."""
        sel = (self.dim == q) & (self.death != self.birth)
        iv = np.stack([self.birth[sel], self.death[sel]], axis=1).astype(np.float32)
        if len(iv) == 0:
            return iv.reshape(0, 2)
        order = np.lexsort((iv[:, 1], iv[:, 0]))
        return iv[order]


def _collect(handle) -> Pairs:
    L = lib()
    if not handle:
        raise ValueError("oracle rejected the input")
    try:
        m = L.oracle_result_count(handle)
        P = L.oracle_result_pairs(handle)
        if m > 0:
            arr = np.ctypeslib.as_array(C.cast(P, C.POINTER(C.c_byte)),
                                        shape=(m * C.sizeof(_Pair),)).copy()
            rec = np.frombuffer(arr.tobytes(), dtype=np.dtype([
                ("dim", np.int32), ("birth", np.float32), ("death", np.float32),
                ("bv", np.int32, (MAXV,)), ("dv", np.int32, (MAXV,))]))
        else:
            rec = np.zeros(0, dtype=np.dtype([
                ("dim", np.int32), ("birth", np.float32), ("death", np.float32),
                ("bv", np.int32, (MAXV,)), ("dv", np.int32, (MAXV,))]))
        adds = int(L.oracle_result_additions(handle))
    finally:
        L.oracle_result_free(handle)
    return Pairs(rec["dim"].copy(), rec["birth"].copy(), rec["death"].copy(),
                 rec["bv"].copy(), rec["dv"].copy(), adds)


def barcodes(D: np.ndarray, max_dim: int, t: float = math.inf, mode: int = MODE_COHOM_CLEAR) -> Pairs:
    """All persistence pairs of dims 0..max_dim of Rips_t (Alg. 1; see the C
    header for the three modes)."""
    D, dp = _f32(D)
    return _collect(lib().oracle_barcodes(dp, D.shape[0], max_dim, C.c_float(t), mode))


def kruskal(D: np.ndarray, t: float = math.inf) -> Pairs:
    """H0 pairs by Kruskal's union-find in filtration order (Sec.
    "Zero-Dimensional Persistence Computation: Kruskal's Algorithm")."""
    D, dp = _f32(D)
    return _collect(lib().oracle_kruskal(dp, D.shape[0], C.c_float(t)))


def columns(D: np.ndarray, p: int, t: float = math.inf):
    """All p-simplices with diam <= t in coboundary order (decreasing diameter,
    then increasing combinatorial index). Returns (diam float32[m], verts int32[m, p+1])."""
    D, dp = _f32(D)
    L = lib()
    m = L.oracle_columns(dp, D.shape[0], p, C.c_float(t), None, None, 0)
    diam = np.zeros(m, dtype=np.float32)
    verts = np.zeros((m, p + 1), dtype=np.int32)
    m2 = L.oracle_columns(dp, D.shape[0], p, C.c_float(t),
                          diam.ctypes.data_as(C.POINTER(C.c_float)),
                          verts.ctypes.data_as(C.POINTER(C.c_int32)), m)
    assert m2 == m
    return diam, verts


def apparent_pairs(D: np.ndarray, p: int, t: float = math.inf):
    """Every apparent pair (sigma, tau), sigma a p-simplex with diam <= t, by the
    definition (sigma youngest facet of tau, tau oldest cofacet of sigma).
    Returns (sigma int32[k, p+1], tau int32[k, p+2]), sigma in coboundary order."""
    D, dp = _f32(D)
    L = lib()
    k = L.oracle_apparent_pairs(dp, D.shape[0], p, C.c_float(t), None, None, 0)
    s = np.zeros((k, p + 1), dtype=np.int32)
    tau = np.zeros((k, p + 2), dtype=np.int32)
    k2 = L.oracle_apparent_pairs(dp, D.shape[0], p, C.c_float(t),
                                 s.ctypes.data_as(C.POINTER(C.c_int32)),
                                 tau.ctypes.data_as(C.POINTER(C.c_int32)), k)
    assert k2 == k
    return s, tau


def apparent_one(D: np.ndarray, p: int, sigma, t: float = math.inf):
    """The definition applied to one simplex: tau (decreasing vertices) or None."""
    D, dp = _f32(D)
    s = np.ascontiguousarray(sorted(sigma, reverse=True), dtype=np.int32)
    tau = np.zeros(p + 2, dtype=np.int32)
    rc = lib().oracle_apparent_one(dp, D.shape[0], p, C.c_float(t),
                                   s.ctypes.data_as(C.POINTER(C.c_int32)),
                                   tau.ctypes.data_as(C.POINTER(C.c_int32)))
    assert rc >= 0
    return tuple(int(x) for x in tau) if rc == 1 else None
