"""Full-size parity: the 2000-point torus (H0-H1) and 192 points on S^3
(H0-H2), in the bench's configuration, against barcodes the oracle computed
offline (tests/golden/make_golden.py, which calls only oracle/), and a
300-point torus against the oracle's coboundary reduction with no clearing
and no Kruskal H0 (COHOM), so that a large comparison does not rest only on
the oracle mode that shares the GPU path's two shortcuts. The stored float32
points are the input, so the comparison does not depend on how a machine's
libm rounds the generators.

At full size the apparent-pair set is also checked on a sample of columns
against the oracle's definition, one column at a time.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cidx(verts):
    return sum(math.comb(int(v), i + 1) for i, v in enumerate(sorted(int(x) for x in verts)))


def _decode(c, k, n):
    """Vertices (decreasing) of the k-vertex simplex with index c."""
    out = []
    hi = n - 1
    for i in range(k, 0, -1):
        v = i - 1
        lo, h = v, hi
        while lo < h:
            mid = (lo + h + 1) // 2
            if math.comb(mid, i) <= c:
                lo = mid
            else:
                h = mid - 1
        out.append(lo)
        c -= math.comb(lo, i)
        hi = lo - 1
    return out


@pytest.fixture(scope="module")
def rpp():
    import __graft_entry__ as g
    g.build()
    import paper_2003_07989_gb300 as m
    return m


@pytest.mark.parametrize("name", ["torus2000", "sphere192", "torus300_cohom"])
def test_fullsize_barcodes_equal_oracle(rpp, name):
    import torch
    g = np.load(os.path.join(GOLDEN, f"{name}.npz"))
    X, max_dim = g["points"], int(g["max_dim"])
    got = rpp.rpp_barcodes(torch.from_numpy(X).cuda(), max_dim=max_dim)
    for q in range(max_dim + 1):
        assert np.array_equal(got.intervals[q], g[f"H{q}"]), (name, q)


def test_fullsize_apparent_sample(rpp):
    import torch
    from paper_2003_07989_gb300 import _native as N
    g = np.load(os.path.join(GOLDEN, "torus2000.npz"))
    X = g["points"]
    n = len(X)
    ctx = rpp.Context(0, record=N.RPP_RECORD_COLUMNS | N.RPP_RECORD_APPARENT)
    got = rpp.rpp_barcodes(torch.from_numpy(X).cuda(), max_dim=1, context=ctx)
    t = got.stats["threshold"]
    D = O.distance_matrix(X)
    _, cols = got.columns[1]
    sig, tau = got.apparent[1]
    app = dict(zip(sig.tolist(), tau.tolist()))
    rng = np.random.default_rng(0)
    for i in rng.choice(len(cols), size=3000, replace=False):
        c = int(cols[i])
        verts = _decode(c, 2, n)
        ref = O.apparent_one(D, 1, verts, t)
        if ref is None:
            assert c not in app
        else:
            assert app.get(c) == _cidx(ref)
    # every apparent pair is a zero-persistence pair, and the apparent count is
    # within the upper bound of the theorem on apparent pairs
    assert len(app) <= math.comb(n - 1, 2)
    assert got.stats["apparent"][1] + got.stats["leftover"][1] == got.stats["columns"][1]


def test_sphere192_served_beside_a_stream_of_small_requests(rpp):
    # The 192 points on S^3 (H0-H2) go in as one large request under a device
    # memory bound, among small requests of the serving mix that keep
    # arriving; the large one is admitted when memory allows, and every result
    # equals its stored or single-instance value.
    from paper_2003_07989_gb300 import inputs as I
    g = np.load(os.path.join(GOLDEN, "sphere192.npz"))
    X = np.ascontiguousarray(g["points"])
    small = I.serving_requests(48, seed=5, n_range=(32, 200))
    alone = [rpp.rpp_barcodes(r.points, max_dim=1, quantile=r.threshold_quantile)
             for r in small]
    srv = rpp.Server(max_slots=4, device_bytes=320 << 20, max_batch=8)
    try:
        first = [srv.submit(r.points, 1, quantile=r.threshold_quantile) for r in small[:24]]
        big = srv.submit(X, 2)
        rest = [srv.submit(r.points, 1, quantile=r.threshold_quantile) for r in small[24:]]
        got = srv.poll(big)
        for q in range(3):
            assert np.array_equal(got.intervals[q], g[f"H{q}"]), q
        for t, a in zip(first + rest, alone):
            r = srv.poll(t)
            for q in (0, 1):
                assert np.array_equal(r.intervals[q], a.intervals[q])
    finally:
        srv.close()
