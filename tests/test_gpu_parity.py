"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: the distance matrix, the column arrays of every dimension (after
threshold and clearing, in coboundary order), the apparent-pair set, and the
barcodes (multisets of float32 intervals). Inputs cover several tiles and
ragged tails, ties, duplicate points, thresholds and the degenerate sizes.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_07989_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def cidx_of(verts) -> int:
    """Combinatorial index sum_i C(v_i, i+1) of vertices sorted ascending
    (Sec. 'The Combinatorial Number System')."""
    return sum(math.comb(int(v), i + 1) for i, v in enumerate(sorted(int(x) for x in verts)))


@pytest.fixture(scope="module")
def rpp():
    import __graft_entry__ as g
    g.build()
    import paper_2003_07989_gb300 as m
    return m


@pytest.fixture(scope="module")
def rec_ctx(rpp):
    from paper_2003_07989_gb300 import _native as N
    return rpp.Context(0, record=N.RPP_RECORD_COLUMNS | N.RPP_RECORD_APPARENT)


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _check_barcodes(got, ref, max_dim, where=""):
    for q in range(max_dim + 1):
        a, b = got.intervals[q], ref.barcode(q)
        assert a.shape == b.shape, (where, q, a.shape, b.shape)
        assert np.array_equal(a, b), (where, q)


# ---------------------------------------------------------------------------
# distances


@pytest.mark.parametrize("n,dim", [(1, 3), (2, 2), (31, 3), (33, 8), (97, 5), (300, 3), (257, 64),
                                   (40, 300)])
def test_distance_matrix_bitwise(rpp, n, dim):
    X = I.noisy_torus(n, seed=n) if dim == 3 else I.blob_cloud(n, dim, seed=n)
    ref = O.distance_matrix(X)
    assert np.array_equal(rpp.rpp_distance_matrix(X), ref)          # host input
    assert np.array_equal(rpp.rpp_distance_matrix(_cuda(X)), ref)   # device input


# ---------------------------------------------------------------------------
# columns and apparent pairs, dimension by dimension


def _oracle_dim_arrays(D, p, t):
    """Oracle columns of dim p after clearing, and the apparent pairs, as cidx."""
    diam, verts = O.columns(D, p, t)
    if p == 1:
        K = O.kruskal(D, t)
        dead = {cidx_of(v[:2]) for v in K.dverts[np.isfinite(K.death)]}
    else:
        P = O.barcodes(D, p - 1, t, O.MODE_COHOM_CLEAR)
        sel = (P.dim == p - 1) & np.isfinite(P.death)
        dead = {cidx_of(v[:p + 1]) for v in P.dverts[sel]}
    keep = [i for i in range(len(diam)) if cidx_of(verts[i]) not in dead]
    cols = (diam[keep], np.array([cidx_of(verts[i]) for i in keep], dtype=np.uint64))
    s, tau = O.apparent_pairs(D, p, t)
    pairs = sorted((cidx_of(b), cidx_of(a)) for a, b in zip(s, tau))
    return cols, pairs


def _cases_small():
    out = [("cube50", O.distance_matrix(I.uniform_cube(50, 3, 0)), 2)]
    out.append(("torus120", O.distance_matrix(I.noisy_torus(120, seed=1)), 2))
    out.append(("sphere70", O.distance_matrix(I.sphere_s3(70, seed=2)), 3))
    out.append(("ties40", I.integer_distances(40, 5, 3), 2))
    out.append(("ties2_33", I.integer_distances(33, 2, 4), 3))
    out.append(("perm45", I.permutation_distances(45, 5), 2))
    return out


@pytest.mark.parametrize("idx", range(6))
def test_columns_and_apparent_pairs_bit_exact(rpp, rec_ctx, idx):
    name, D, max_dim = _cases_small()[idx]
    got = rpp.rpp_barcodes(_cuda(D), max_dim=max_dim, kind="distances", context=rec_ctx)
    t = got.stats["threshold"]
    assert t == O.enclosing_radius(D)
    for p in range(1, max_dim + 1):
        (cd, ci), pairs = _oracle_dim_arrays(D, p, t)
        gd, gi = got.columns[p]
        assert np.array_equal(gd, cd), (name, p)
        assert np.array_equal(gi, ci), (name, p)
        gs, gt = got.apparent[p]
        assert list(zip(gt.tolist(), gs.tolist())) == pairs, (name, p)


# ---------------------------------------------------------------------------
# barcodes


# Oracle mode per case: the literal form with none of the shortcuts, HOM
# (Alg. 1 on the explicit boundary matrix, no clearing, no cohomology),
# wherever it finishes in seconds; COHOM (the coboundary reduction without clearing) for
# the 150-point 2-sphere; COHOM_CLEAR only for the 200-point torus, whose
# 300-point sibling is compared with COHOM in test_gpu_fullsize.py.
HOM, COHOM, CLEAR = O.MODE_HOM, O.MODE_COHOM, O.MODE_COHOM_CLEAR


def _barcode_cases():
    cases = [("cfg1_cube50_seed0", I.uniform_cube(50, 3, 0), "points", 1, math.inf, None, HOM)]
    for i, (n, dim) in enumerate([(33, 2), (64, 3), (65, 4), (97, 8), (130, 3)]):
        cases.append((f"blob{n}", I.blob_cloud(n, dim, 10 + i), "points", 1, math.inf, None, HOM))
    cases.append(("torus200", I.noisy_torus(200, seed=7), "points", 1, math.inf, None, CLEAR))
    cases.append(("sphere60_h2", I.sphere_s3(60, seed=8), "points", 2, math.inf, None, HOM))
    cases.append(("cube40_h3", I.uniform_cube(40, 3, 9), "points", 3, math.inf, None, HOM))
    cases.append(("ties50", I.integer_distances(50, 5, 11), "distances", 2, math.inf, None, HOM))
    cases.append(("ties2_40", I.integer_distances(40, 2, 12), "distances", 1, math.inf, None, HOM))
    cases.append(("circle80_t", I.circle_cloud(80, 1.0, 0.05, 2, 13), "points", 1, 0.4, None, HOM))
    cases.append(("cube70_t0", I.uniform_cube(70, 3, 14), "points", 1, 0.0, None, HOM))
    cases.append(("cube90_q", I.uniform_cube(90, 3, 15), "points", 1, math.inf, 0.6, HOM))
    cases.append(("sphere2_q", I.sphere2_cloud(150, 1.0, 0.05, 5, 16), "points", 2, math.inf, 0.3,
                  COHOM))
    cases.append(("blob_q1", I.blob_cloud(60, 2, 17), "points", 1, math.inf, 1.0, HOM))
    return cases


@pytest.mark.parametrize("idx", range(16))
def test_barcodes_bit_exact(rpp, idx):
    name, X, kind, max_dim, t, q, mode = _barcode_cases()[idx]
    D = O.distance_matrix(X) if kind == "points" else X
    t_ref = O.distance_quantile(D, q) if q is not None else t
    ref = O.barcodes(D, max_dim, t_ref, mode)
    for data in (X, _cuda(X)):
        got = rpp.rpp_barcodes(data, max_dim=max_dim, threshold=t, kind=kind, quantile=q)
        _check_barcodes(got, ref, max_dim, name)


def test_cfg4_clouds_against_the_boundary_matrix_oracle(rpp):
    """Four clouds of the differentiation workload (128 points on noisy
    planar circles, full filtration, H0-H1) against Alg. 1 on the explicit
    boundary matrix of all 341,376 triangles, with no clearing, no
    cohomology and no apparent pairs: through the single-instance path and
    through the fused batched launch of the 128-point bucket."""
    clouds = I.noisy_circles(4, 128, seed=0)
    batched = rpp.rpp_barcodes_batched([c for c in clouds], max_dim=1)
    for i, X in enumerate(clouds):
        ref = O.barcodes(O.distance_matrix(X), 1, math.inf, O.MODE_HOM)
        _check_barcodes(rpp.rpp_barcodes(_cuda(X), max_dim=1), ref, 1, f"cloud{i}")
        _check_barcodes(batched[i], ref, 1, f"batched cloud{i}")


def test_degenerate_sizes(rpp):
    for n in (1, 2, 3):
        X = I.uniform_cube(n, 2, 20 + n)
        got = rpp.rpp_barcodes(X, max_dim=2)
        ref = O.barcodes(O.distance_matrix(X), 2, math.inf, O.MODE_HOM)
        _check_barcodes(got, ref, 2, f"n={n}")
    # duplicate points: zero distances, zero-length H0 bars dropped
    X = np.repeat(I.uniform_cube(20, 3, 30), 2, axis=0)
    got = rpp.rpp_barcodes(X, max_dim=1)
    _check_barcodes(got, O.barcodes(O.distance_matrix(X), 1, math.inf, O.MODE_HOM), 1)
    # every distance equal
    D = np.ones((30, 30), np.float32)
    np.fill_diagonal(D, 0)
    got = rpp.rpp_barcodes(D, max_dim=2, kind="distances")
    _check_barcodes(got, O.barcodes(D, 2, math.inf, O.MODE_HOM), 2)
    assert got.stats["apparent"][1] == math.comb(29, 2)


def test_invalid_inputs(rpp):
    from paper_2003_07989_gb300 import _native as N
    X = I.uniform_cube(20, 3, 1)
    bad = X.copy()
    bad[3, 1] = np.nan
    for data in (bad, _cuda(bad)):
        with pytest.raises(N.RppError) as e:
            rpp.rpp_barcodes(data, max_dim=1)
        assert e.value.status == N.RPP_E_INVALID
    D = O.distance_matrix(X)
    D[2, 5] += 1.0  # asymmetric
    with pytest.raises(N.RppError) as e:
        rpp.rpp_barcodes(_cuda(D), max_dim=1, kind="distances")
    assert e.value.status == N.RPP_E_INVALID
    for kw in ({"threshold": -1.0}, {"max_dim": 9}, {"quantile": 1.5}):
        with pytest.raises(N.RppError):
            rpp.rpp_barcodes(X, **{"max_dim": 1, **kw})
    # the context stays usable after errors
    got = rpp.rpp_barcodes(X, max_dim=1)
    _check_barcodes(got, O.barcodes(O.distance_matrix(X), 1, math.inf, O.MODE_HOM), 1)


def test_deterministic(rpp):
    X = I.noisy_torus(400, seed=3)
    a = rpp.rpp_barcodes(_cuda(X), max_dim=1)
    b = rpp.rpp_barcodes(_cuda(X), max_dim=1)
    for q in (0, 1):
        assert np.array_equal(a.intervals[q], b.intervals[q])
        assert np.array_equal(a.critical[q], b.critical[q])


def test_critical_edges_realise_endpoints(rpp):
    X = I.noisy_torus(300, seed=4)
    D = O.distance_matrix(X)
    got = rpp.rpp_barcodes(X, max_dim=1)
    for q in (0, 1):
        iv, cr = got.intervals[q], got.critical[q]
        for (b, d), (bu, bv, du, dv) in zip(iv, cr):
            if bu >= 0:
                assert D[bu, bv] == b
            if math.isfinite(d):
                assert D[du, dv] == d


def test_apparent_shape_tuning_changes_nothing(rpp):
    """The apparent pass's launch shape, tuned per size bucket on the first
    instance or left at its default, gives the same barcodes, realising edges
    and counters (the tuning launches count into a scratch state)."""
    tuned, fixed = rpp.Context(0), rpp.Context(0)
    fixed.set_batch(fused=True, autotune=False)
    for X, md in ((I.noisy_torus(400, seed=3), 1), (I.sphere_s3(60, seed=2), 2)):
        a = rpp.rpp_barcodes(_cuda(X), max_dim=md, context=tuned)
        b = rpp.rpp_barcodes(_cuda(X), max_dim=md, context=fixed)
        c = rpp.rpp_barcodes(_cuda(X), max_dim=md, context=tuned)  # the tuned shape
        for q in range(md + 1):
            assert np.array_equal(a.intervals[q], b.intervals[q])
            assert np.array_equal(a.critical[q], b.critical[q])
            assert np.array_equal(c.intervals[q], b.intervals[q])
        for k in ("columns", "apparent", "leftover", "scanned", "additions"):
            assert a.stats[k] == b.stats[k] == c.stats[k], k


def test_unread_apparent_taus_change_nothing(rpp):
    """With H0-H1 only, each edge's apparent vertex kept and no pairs
    recorded, the apparent pass computes no cofacet index for apparent
    columns and the partition only counts them. Recording the pairs (or a
    second dimension, which clears with them) makes both write the taus. The
    barcodes, realising edges and counters must not depend on which, and
    the recorded pairs must be the oracle's."""
    from paper_2003_07989_gb300 import _native as N
    X = I.noisy_torus(400, seed=3)
    D = O.distance_matrix(X)
    plain = rpp.Context(0)
    rec = rpp.Context(0, record=N.RPP_RECORD_APPARENT)
    a = rpp.rpp_barcodes(_cuda(X), max_dim=1, context=plain)
    b = rpp.rpp_barcodes(_cuda(X), max_dim=1, context=rec)
    for q in (0, 1):
        assert np.array_equal(a.intervals[q], b.intervals[q])
        assert np.array_equal(a.critical[q], b.critical[q])
    for k in ("columns", "apparent", "leftover", "free_pivot", "additions", "scanned"):
        assert a.stats[k] == b.stats[k], k
    _check_barcodes(a, O.barcodes(D, 1, O.enclosing_radius(D), O.MODE_COHOM_CLEAR), 1)
    gs, gt = b.apparent[1]
    assert len(gs) == a.stats["apparent"][1]
    _, pairs = _oracle_dim_arrays(D, 1, a.stats["threshold"])
    assert list(zip(gt.tolist(), gs.tolist())) == pairs
