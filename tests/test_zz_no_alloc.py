"""rpp_filtration_edges_noalloc: the edge filtration for callers that cannot
allocate device memory (inside another runtime's memory pool, or in loops
where cudaMalloc/cudaFree would synchronise the device).

Its output is checked two ways. Against the CPU oracle: every edge inside the
threshold in coboundary order (decreasing diameter, then increasing
combinatorial index), exactly oracle.columns(D, 1, t), entry for entry, at
the enclosing radius, with no threshold (+inf) and at n = 724, the largest
size the static scratch allows. Against the regular entry point:
rpp_barcodes records the dimension-1 columns after clearing, so the
allocation-free list with the minimum-spanning-tree edges (the H0 deaths)
removed must equal it. Consecutive calls share the static scratch array, so
each later call also checks that nothing of the one before leaks into it.
This file is collected last on purpose.
"""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _noalloc(L, N, D, n, t):
    import torch
    m = n * (n - 1) // 2
    diam = torch.full((max(m, 1),), float("nan"), device="cuda", dtype=torch.float32)
    cidx = torch.zeros(max(m, 1), device="cuda", dtype=torch.int64)
    count = C.c_int64(-1)
    rc = L.rpp_filtration_edges_noalloc(D.data_ptr(), n, t, diam.data_ptr(), cidx.data_ptr(),
                                        m, C.byref(count),
                                        torch.cuda.current_stream().cuda_stream)
    N.check(rc, "rpp_filtration_edges_noalloc")
    k = count.value
    return diam[:k].cpu().numpy(), cidx[:k].cpu().numpy().astype(np.uint64)


def _oracle_edges(D, t):
    diam, verts = O.columns(D, 1, t)
    a = verts.max(axis=1).astype(np.uint64)
    b = verts.min(axis=1).astype(np.uint64)
    return diam, a * (a - np.uint64(1)) // np.uint64(2) + b  # C(a, 2) + C(b, 1)


def test_noalloc_edges_match_oracle_and_recorded_columns():
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_2003_07989_gb300 as rpp
    from paper_2003_07989_gb300 import _native as N
    from paper_2003_07989_gb300 import inputs as I

    L = N.lib()
    ctx = rpp.Context(0, record=N.RPP_RECORD_COLUMNS)
    # (seed, n, threshold): None = the enclosing radius rpp_barcodes uses
    cases = ((1, 600, None), (2, 517, None), (3, 724, math.inf), (4, 724, None), (5, 2, math.inf))
    for seed, n, t in cases:
        X = I.noisy_torus(n, seed=seed)
        Dh = O.distance_matrix(X)
        D = torch.from_numpy(Dh).cuda()
        ref = None
        if t is None:
            ref = rpp.rpp_barcodes(torch.from_numpy(X).cuda(), max_dim=1, context=ctx)
            t = ref.stats["threshold"]
            assert t == O.enclosing_radius(Dh)
        got_d, got_i = _noalloc(L, N, D, n, t)
        # the oracle: every edge with diam <= t, in coboundary order
        od, oi = _oracle_edges(Dh, t)
        assert np.array_equal(got_d, od), (n, t)
        assert np.array_equal(got_i, oi), (n, t)
        if t == math.inf:
            assert len(got_i) == n * (n - 1) // 2
        if ref is None:
            continue
        # the regular entry point: its recorded columns are these edges minus
        # the spanning tree's, which clearing removed
        col_d, col_i = ref.columns[1]
        crit = ref.critical[0]
        fin = np.isfinite(ref.intervals[0][:, 1])
        mst = {int(u) * (int(u) - 1) // 2 + int(v) for u, v in crit[fin][:, 2:4]}
        assert len(mst) == n - 1
        keep = np.array([int(c) not in mst for c in got_i])
        assert int((~keep).sum()) == n - 1
        assert np.array_equal(got_d[keep], col_d)
        assert np.array_equal(got_i[keep], col_i)


def test_noalloc_rejects_sizes_beyond_the_bound():
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2003_07989_gb300 import _native as N
    L = N.lib()
    n = 725
    D = torch.zeros((n, n), device="cuda")
    out_d = torch.zeros(8, device="cuda")
    out_i = torch.zeros(8, device="cuda", dtype=torch.int64)
    count = C.c_int64(-1)
    rc = L.rpp_filtration_edges_noalloc(D.data_ptr(), n, math.inf, out_d.data_ptr(),
                                        out_i.data_ptr(), 8, C.byref(count), None)
    assert rc == N.RPP_E_INVALID
    assert b"724" in L.rpp_last_error()
    assert count.value == -1
    # outputs in host memory are refused before any GPU work
    host_d = np.zeros(8, np.float32)
    host_i = np.zeros(8, np.uint64)
    D2 = torch.zeros((4, 4), device="cuda")
    rc = L.rpp_filtration_edges_noalloc(D2.data_ptr(), 4, math.inf, host_d.ctypes.data,
                                        host_i.ctypes.data, 8, C.byref(count), None)
    assert rc == N.RPP_E_INVALID
    assert count.value == -1
