"""The C-ABI library builds, loads and exports every function include/rpp.h
declares; host-side argument checks work without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "rpp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(rpp_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2003_07989_gb300 import build
    build.build()
    from paper_2003_07989_gb300 import _native
    return _native.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rpp_barcodes", "rpp_barcodes_batched", "rpp_barcodes_backward",
                 "rpp_server_submit", "rpp_server_poll", "rpp_result_intervals"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2003_07989_gb300 import _native
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(_native.EXPORTED)


def test_status_strings(lib):
    for code in range(7):
        assert lib.rpp_status_string(code)
    assert lib.rpp_last_error() is not None


def test_argument_errors_without_gpu(lib):
    from paper_2003_07989_gb300 import _native as N
    # a NULL out pointer is rejected before any CUDA call
    assert lib.rpp_context_create(0, 0, None) == N.RPP_E_INVALID
    h = C.c_void_p()
    rc = lib.rpp_barcodes(None, None, 0, 10, 3, 1, float("inf"), None, C.byref(h))
    assert rc == N.RPP_E_INVALID
    assert b"NULL" in lib.rpp_last_error()
    assert lib.rpp_result_count(None, 0) == -1
    for set_mode in (lib.rpp_context_set_device_reduce, lib.rpp_context_set_sparse):
        assert set_mode(None, 1) == N.RPP_E_INVALID
    # C(n, 2) >= 2^32 from n = 92683 on: refused by the argument checks, which
    # need no context and read no input
    tiny = (C.c_float * 4)()
    for n_pts, want, msg in ((92683, N.RPP_E_OVERFLOW, b"92682"), (0, N.RPP_E_INVALID, b"n must")):
        rc = lib.rpp_barcodes(None, C.addressof(tiny), N.RPP_INPUT_DISTANCES, n_pts, 0, 0,
                              float("inf"), None, C.byref(h))
        assert rc == want and not h.value
        assert msg in lib.rpp_last_error()
    assert lib.rpp_result_total(None) == -1


def test_results_accessors_reject_bad_arguments(lib):
    from paper_2003_07989_gb300 import _native as N
    offs = (C.c_int64 * 3)()
    two = (C.c_void_p * 2)(None, None)
    # NULL entries, a NULL offsets array, a dimension out of range
    assert lib.rpp_results_gather(two, 2, 1, C.addressof(offs), None, None) == N.RPP_E_INVALID
    assert b"NULL" in lib.rpp_last_error()
    assert lib.rpp_results_gather(two, 0, 1, None, None, None) == N.RPP_E_INVALID
    assert lib.rpp_results_gather(two, 0, N.RPP_MAX_DIM + 1, C.addressof(offs), None,
                                  None) == N.RPP_E_INVALID
    assert lib.rpp_results_gather(two, -1, 0, C.addressof(offs), None, None) == N.RPP_E_INVALID
    stats = (N.Stats * 2)()
    assert lib.rpp_results_stats(two, 2, stats) == N.RPP_E_INVALID
    # an empty set is fine: offsets[0] = 0
    offs[0] = 7
    assert lib.rpp_results_gather(two, 0, 0, C.addressof(offs), None, None) == N.RPP_OK
    assert offs[0] == 0
    lib.rpp_results_free(two, 2)  # NULL entries are skipped


def test_l2_probe_rejects_bad_arguments_without_gpu(lib):
    from paper_2003_07989_gb300 import _native as N
    # every case below is refused by host checks before any CUDA call; the
    # addresses are never dereferenced
    buf, sink = 0x10000, 0x20000
    for args in ((None, 16, 1, 1, sink), (buf, 16, 1, 1, None),   # NULL pointers
                 (buf + 4, 16, 1, 1, sink), (buf, 24, 1, 1, sink),  # misaligned, ragged size
                 (buf, 0, 1, 1, sink), (buf, 16, 1, 1, sink + 2),   # empty, misaligned sink
                 (buf, 16, 0, 1, sink), (buf, 16, (1 << 20) + 1, 1, sink),  # reps
                 (buf, 16, 1, 0, sink), (buf, 16, 1, 65536, sink)):        # blocks
        assert lib.rpp_l2_read_probe(*args, None) == N.RPP_E_INVALID, args
        assert lib.rpp_last_error().startswith(b"rpp_l2_read_probe")
