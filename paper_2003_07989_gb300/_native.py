"""ctypes binding of librpp.so (include/rpp.h). Argument marshalling only.

The library is built in-tree by ``paper_2003_07989_gb300.build``. If it is
missing the import of this module fails loudly: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "librpp.so")

RPP_OK, RPP_E_INVALID, RPP_E_NOMEM, RPP_E_OVERFLOW, RPP_E_CUDA, RPP_E_TIMEOUT, RPP_E_BUSY = range(7)
RPP_INPUT_POINTS, RPP_INPUT_DISTANCES = 0, 1
RPP_MAX_DIM = 4

EXPORTED = [
    "rpp_context_create", "rpp_context_destroy", "rpp_barcodes", "rpp_barcodes_quantile",
    "rpp_result_count", "rpp_result_intervals", "rpp_result_critical", "rpp_result_stats",
    "rpp_result_free", "rpp_barcodes_batched", "rpp_barcodes_backward", "rpp_result_total",
    "rpp_server_create", "rpp_server_submit", "rpp_server_poll", "rpp_server_destroy",
    "rpp_status_string", "rpp_last_error", "rpp_distance_matrix", "rpp_context_set_record",
    "rpp_result_columns", "rpp_result_apparent", "rpp_filtration_edges_noalloc",
    "rpp_context_set_batch", "rpp_context_batch_tuning", "rpp_apparent_census",
    "rpp_results_gather", "rpp_results_stats", "rpp_results_free", "rpp_server_next",
    "rpp_filtration", "rpp_context_set_sparse", "rpp_context_set_device_reduce",
    "rpp_l2_read_probe",
]
RPP_RECORD_COLUMNS, RPP_RECORD_APPARENT, RPP_RECORD_TIMING = 1, 2, 4
STAGES = ["distance", "enclosing_radius", "build_columns", "sort_columns", "apparent",
          "partition", "sort_pairs", "other"]


class Interval(C.Structure):
    _fields_ = [("birth", C.c_float), ("death", C.c_float)]


class Critical(C.Structure):
    _fields_ = [("bu", C.c_int32), ("bv", C.c_int32), ("du", C.c_int32), ("dv", C.c_int32)]


_A = C.c_int64 * (RPP_MAX_DIM + 1)


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("max_dim", C.c_int32), ("threshold", C.c_float),
                ("enclosing_radius", C.c_float),
                ("candidates", _A), ("columns", _A), ("cleared", _A), ("apparent", _A),
                ("leftover", _A), ("free_pivot", _A), ("additions", _A), ("store_reads", _A),
                ("entries", _A),
                ("intervals", _A), ("scanned", _A), ("sweep_levels", _A),
                ("kernel_launches", C.c_int64),
                ("stage_ms", C.c_double * 8), ("stage_launches", C.c_int64 * 8),
                ("ms_device", C.c_double), ("ms_host_reduce", C.c_double),
                ("ms_host_h0", C.c_double), ("ms_total", C.c_double), ("sparse", _A),
                ("sweep_pivots", _A), ("sweep_idle", _A), ("ms_sweep_walks", C.c_double),
                ("device_columns", _A), ("sort_passes", _A)]


class ServerConfig(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("device_bytes", C.c_size_t),
                ("host_threads", C.c_int32), ("max_batch", C.c_int32)]


class RppError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status}: {detail}")
        self.status = status


_lib = None


def lib():
    """Load librpp.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, fp, i64, i32 = C.c_void_p, C.POINTER(C.c_float), C.c_int64, C.c_int32
    L.rpp_context_create.argtypes = [C.c_int, C.c_size_t, C.POINTER(vp)]
    L.rpp_context_destroy.argtypes = [vp]
    L.rpp_context_destroy.restype = None
    L.rpp_barcodes.argtypes = [vp, vp, C.c_int, i64, i32, i32, C.c_float, vp, C.POINTER(vp)]
    L.rpp_barcodes_quantile.argtypes = [vp, vp, C.c_int, i64, i32, i32, C.c_double, vp,
                                        C.POINTER(vp)]
    L.rpp_apparent_census.argtypes = [vp, vp, C.c_int, i64, i32, vp, C.POINTER(Stats)]
    L.rpp_result_count.argtypes = [vp, i32]
    L.rpp_result_count.restype = i64
    L.rpp_result_total.argtypes = [vp]
    L.rpp_result_total.restype = i64
    L.rpp_result_intervals.argtypes = [vp, i32]
    L.rpp_result_intervals.restype = C.POINTER(Interval)
    L.rpp_result_critical.argtypes = [vp, i32]
    L.rpp_result_critical.restype = C.POINTER(Critical)
    L.rpp_result_stats.argtypes = [vp, C.POINTER(Stats)]
    L.rpp_result_free.argtypes = [vp]
    L.rpp_result_free.restype = None
    L.rpp_barcodes_batched.argtypes = [vp, i32, C.POINTER(vp), C.POINTER(i64), C.POINTER(i32),
                                       i32, fp, C.POINTER(C.c_double), vp, C.POINTER(vp)]
    L.rpp_barcodes_backward.argtypes = [vp, i32, vp, C.POINTER(i64), i32, C.POINTER(vp),
                                        vp, vp, vp, vp]
    L.rpp_server_create.argtypes = [vp, C.POINTER(ServerConfig), C.POINTER(vp)]
    L.rpp_server_submit.argtypes = [vp, vp, i64, i32, i32, C.c_float, C.c_double,
                                    C.POINTER(C.c_uint64)]
    L.rpp_server_poll.argtypes = [vp, C.c_uint64, i32, C.POINTER(vp)]
    L.rpp_server_next.argtypes = [vp, i32, C.POINTER(C.c_uint64), C.POINTER(vp)]
    L.rpp_server_destroy.argtypes = [vp]
    L.rpp_server_destroy.restype = None
    L.rpp_status_string.argtypes = [C.c_int]
    L.rpp_status_string.restype = C.c_char_p
    L.rpp_last_error.argtypes = []
    L.rpp_last_error.restype = C.c_char_p
    L.rpp_distance_matrix.argtypes = [vp, vp, i64, i32, vp, vp]
    L.rpp_context_set_record.argtypes = [vp, i32]
    u64pp = C.POINTER(C.POINTER(C.c_uint64))
    L.rpp_result_columns.argtypes = [vp, i32, C.POINTER(C.POINTER(C.c_float)), u64pp]
    L.rpp_result_columns.restype = i64
    L.rpp_result_apparent.argtypes = [vp, i32, u64pp, u64pp]
    L.rpp_result_apparent.restype = i64
    L.rpp_filtration_edges_noalloc.argtypes = [vp, i64, C.c_float, vp, vp, i64,
                                               C.POINTER(i64), vp]
    L.rpp_context_set_batch.argtypes = [vp, i32, i32]
    L.rpp_results_gather.argtypes = [C.POINTER(vp), i32, i32, vp, vp, vp]
    L.rpp_results_stats.argtypes = [C.POINTER(vp), i32, C.POINTER(Stats)]
    L.rpp_results_free.argtypes = [C.POINTER(vp), i32]
    L.rpp_results_free.restype = None
    L.rpp_context_batch_tuning.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32)]
    L.rpp_context_set_sparse.argtypes = [vp, i32]
    L.rpp_context_set_device_reduce.argtypes = [vp, i32]
    L.rpp_filtration.argtypes = [vp, vp, C.c_int, i64, i32, i32, C.c_float, vp, vp, vp, i64,
                                 C.POINTER(i64), C.POINTER(Stats)]
    L.rpp_l2_read_probe.argtypes = [vp, C.c_size_t, i32, i32, vp, vp]
    for name in ("rpp_context_set_batch", "rpp_context_batch_tuning",
                 "rpp_context_create", "rpp_barcodes", "rpp_barcodes_quantile",
                 "rpp_distance_matrix", "rpp_context_set_record", "rpp_filtration_edges_noalloc",
                 "rpp_result_stats", "rpp_barcodes_batched", "rpp_barcodes_backward",
                 "rpp_server_create", "rpp_server_submit", "rpp_server_poll",
                 "rpp_results_gather", "rpp_results_stats", "rpp_server_next",
                 "rpp_filtration", "rpp_context_set_sparse", "rpp_context_set_device_reduce",
                 "rpp_l2_read_probe"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(status: int, where: str):
    if status != RPP_OK:
        L = lib()
        raise RppError(status, where, L.rpp_last_error().decode(errors="replace"))
