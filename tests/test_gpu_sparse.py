"""The thresholded construction of dimensions p >= 2 (Sec. "Computation
Induced by Sparse 1-Skeletons"): simplices listed as cliques of the graph of
edges inside t, clearing by binary search, apparent tests over neighbour
lists.

* Thresholds far below the enclosing radius, against the oracle (the
  explicit boundary-matrix reduction where it finishes, else the coboundary
  reduction), with the thresholded construction forced on.
* The thresholded and the dense construction give the same column arrays,
  apparent pairs, barcodes and realising edges, on random, tie-heavy and
  permutation inputs.
* The O(3) workload on 2,000 points, with the long walk of its long-lived
  H2 class, against the oracle.
* A cloud whose C(n, 3) exceeds 2^32, which the dense construction cannot
  enumerate, against the oracle run on each connected component of the
  threshold graph on its own (the Rips complex of a disjoint union is the
  disjoint union of the components' complexes, so the barcodes add up).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_07989_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rpp():
    import __graft_entry__ as g
    g.build()
    import paper_2003_07989_gb300 as m
    return m


def _ctx(rpp, mode, record=0):
    c = rpp.Context(0, record=record)
    c.set_sparse(mode)
    return c


CASES = [  # name, points or D, kind, max_dim, quantile of the distances as t, oracle mode
    ("cube60_h3", lambda: I.uniform_cube(60, 3, seed=1), "points", 3, 0.3, O.MODE_HOM),
    ("sphere120_h2", lambda: I.sphere_s3(120, seed=2), "points", 2, 0.2, O.MODE_HOM),
    ("o3_300_h2", lambda: I.orthogonal3(300, seed=3), "points", 2, 0.05, O.MODE_COHOM_CLEAR),
    ("ties50_h2", lambda: I.integer_distances(50, 5, 4), "distances", 2, 0.4, O.MODE_HOM),
    ("torus250_h2", lambda: I.noisy_torus(250, seed=5), "points", 2, 0.08, O.MODE_COHOM_CLEAR),
    ("perm40_h3", lambda: I.permutation_distances(40, 6), "distances", 3, 0.5, O.MODE_HOM),
]


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_thresholded_construction_matches_oracle(rpp, idx):
    name, gen, kind, max_dim, q, mode = CASES[idx]
    X = gen()
    D = O.distance_matrix(X) if kind == "points" else X
    t = O.distance_quantile(D, q)
    assert t < O.enclosing_radius(D)
    got = rpp.rpp_barcodes(X, max_dim=max_dim, threshold=t, kind=kind,
                           context=_ctx(rpp, 1))
    for p in range(2, max_dim + 1):
        assert got.stats["sparse"][p] == 1, (name, p)
    ref = O.barcodes(D, max_dim, t, mode)
    for k in range(max_dim + 1):
        assert np.array_equal(got.intervals[k], ref.barcode(k)), (name, k)


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_thresholded_equals_dense(rpp, idx):
    from paper_2003_07989_gb300 import _native as N
    name, gen, kind, max_dim, q, _ = CASES[idx]
    X = gen()
    D = O.distance_matrix(X) if kind == "points" else X
    t = O.distance_quantile(D, q)
    rec = N.RPP_RECORD_COLUMNS | N.RPP_RECORD_APPARENT
    a = rpp.rpp_barcodes(X, max_dim=max_dim, threshold=t, kind=kind, context=_ctx(rpp, 1, rec))
    b = rpp.rpp_barcodes(X, max_dim=max_dim, threshold=t, kind=kind, context=_ctx(rpp, 2, rec))
    assert b.stats["sparse"][2] == 0
    for k in range(max_dim + 1):
        assert np.array_equal(a.intervals[k], b.intervals[k]), (name, k)
        assert np.array_equal(a.critical[k], b.critical[k]), (name, k)
    for p in range(1, max_dim + 1):
        for x, y in zip(a.columns[p], b.columns[p]):
            assert np.array_equal(x, y), (name, p)
        for x, y in zip(a.apparent[p], b.apparent[p]):
            assert np.array_equal(x, y), (name, p)
        for key in ("columns", "cleared", "apparent", "leftover", "additions"):
            assert a.stats[key][p] == b.stats[key][p], (name, p, key)


def _components(D, t):
    n = len(D)
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    ii, jj = np.nonzero(np.triu(D <= t, 1))
    for i, j in zip(ii.tolist(), jj.tolist()):
        a, b = find(i), find(j)
        if a != b:
            parent[a] = b
    comp = {}
    for v in range(n):
        comp.setdefault(find(v), []).append(v)
    return list(comp.values())


def test_beyond_the_dense_index_range(rpp):
    """2960 points: C(2960, 3) > 2^32 candidate triangles. Auto mode takes the
    thresholded construction; the barcode equals the union of the oracle's
    barcodes of the threshold graph's components."""
    n = 2960
    assert math.comb(n, 3) >= 2 ** 32
    X = I.uniform_cube(n, 2, seed=7)
    D = O.distance_matrix(X)
    t = O.distance_quantile(D, 0.0006)
    got = rpp.rpp_barcodes(X, max_dim=2, threshold=t, context=_ctx(rpp, 0))
    assert got.stats["sparse"][2] == 1
    want = {k: [] for k in range(3)}
    comps = _components(D, t)
    assert max(len(c) for c in comps) <= 400  # the oracle runs on each one
    for comp in comps:
        sub = np.ascontiguousarray(D[np.ix_(comp, comp)])
        ref = O.barcodes(sub, 2, t, O.MODE_COHOM_CLEAR)
        for k in range(3):
            want[k].append(ref.barcode(k))
    for k in range(3):
        w = np.concatenate(want[k]) if want[k] else np.zeros((0, 2), np.float32)
        w = w[np.lexsort((w[:, 1], w[:, 0]))]
        assert np.array_equal(got.intervals[k], w), k
    # and the dense construction refuses it
    from paper_2003_07989_gb300 import _native as N
    with pytest.raises(N.RppError) as e:
        rpp.rpp_barcodes(X, max_dim=2, threshold=t, context=_ctx(rpp, 2))
    assert e.value.status == N.RPP_E_NOMEM


def test_o3_long_h2_walks_match_the_oracle(rpp):
    """2,000 random O(3) matrices at threshold 1.4, H0-H2 (the thresholded
    workload of the bench on its first 2,000 points), against the coboundary
    reduction with clearing: SO(3) = RP^3 carries a long-lived H2 class over
    Z/2, whose column makes a long walk (13,130 additions in dimension 2 in
    all), the case that the reduction's cofacet bitsets and column heap are
    for."""
    X = I.orthogonal3(4096)[:2000]
    ref = O.barcodes(O.distance_matrix(X), 2, 1.4, O.MODE_COHOM_CLEAR)
    got = rpp.rpp_barcodes(X, max_dim=2, threshold=1.4)
    for q in range(3):
        assert np.array_equal(got.intervals[q], ref.barcode(q)), q
    assert got.stats["sparse"][2] == 1
