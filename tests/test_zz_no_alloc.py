"""rpp_filtration_edges_noalloc: the edge filtration for callers that cannot
allocate device memory (inside another runtime's memory pool, or in loops
where cudaMalloc/cudaFree would synchronise the device).

Its output is checked against the regular entry point: rpp_barcodes records
the dimension-1 columns after clearing, so the allocation-free edge list with
the minimum-spanning-tree edges (the H0 deaths) removed must equal it entry for
entry. Two calls in a row share the static scratch array, so the second call
also checks that nothing of the first one leaks into it. This file is collected
last on purpose.
"""
import ctypes as C
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_edges_match_recorded_columns_twice():
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_2003_07989_gb300 as rpp
    from paper_2003_07989_gb300 import _native as N
    from paper_2003_07989_gb300 import inputs as I

    L = N.lib()
    ctx = rpp.Context(0, record=N.RPP_RECORD_COLUMNS)
    for seed, n in ((1, 600), (2, 517)):
        X = I.noisy_torus(n, seed=seed)
        ref = rpp.rpp_barcodes(torch.from_numpy(X).cuda(), max_dim=1, context=ctx)
        t = ref.stats["threshold"]
        col_d, col_i = ref.columns[1]
        # the H0 deaths are the MST edges, which clearing removed from the columns
        crit = ref.critical[0]
        fin = np.isfinite(ref.intervals[0][:, 1])
        mst = {int(u) * (int(u) - 1) // 2 + int(v) for u, v in crit[fin][:, 2:4]}
        assert len(mst) == n - 1

        D = torch.from_numpy(rpp.rpp_distance_matrix(X)).cuda()
        m = n * (n - 1) // 2
        diam = torch.full((m,), float("nan"), device="cuda", dtype=torch.float32)
        cidx = torch.zeros(m, device="cuda", dtype=torch.int64)
        count = C.c_int64(-1)
        rc = L.rpp_filtration_edges_noalloc(D.data_ptr(), n, t, diam.data_ptr(), cidx.data_ptr(),
                                            m, C.byref(count),
                                            torch.cuda.current_stream().cuda_stream)
        N.check(rc, "rpp_filtration_edges_noalloc")
        k = count.value
        assert k == len(col_i) + (n - 1)
        got_d = diam[:k].cpu().numpy()
        got_i = cidx[:k].cpu().numpy().astype(np.uint64)
        keep = np.array([int(c) not in mst for c in got_i])
        assert int((~keep).sum()) == n - 1
        assert np.array_equal(got_d[keep], col_d)
        assert np.array_equal(got_i[keep], col_i)
        # every edge inside the threshold, in coboundary order
        assert np.all(got_d <= t)
        order = np.lexsort((got_i, -got_d.astype(np.float64)))
        assert np.array_equal(order, np.arange(k))


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
