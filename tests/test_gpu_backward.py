"""Gradients of the barcode endpoints (rpp_barcodes_backward, RipsPersistence).

The loss is the total H1 persistence, sum over finite H1 intervals of
(death - birth), over a batch of noisy planar circles. It is checked against
  * a float64 reference gradient built from the oracle's pairing: each endpoint
    is the length of the youngest edge of the birth or death simplex;
  * float64 central finite differences (h = 1e-3) on tie-free clouds, where the
    oracle's pairing is the same at x - h and x + h.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_07989_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _youngest_edge(D, verts):
    """Largest distance among the simplex's edges; ties: smallest edge index."""
    vs = [int(v) for v in verts if v >= 0]
    best = None
    for a, b in itertools.combinations(vs, 2):
        u, w = max(a, b), min(a, b)
        key = (float(D[u, w]), -(u * (u - 1) // 2 + w))
        if best is None or key > best[0]:
            best = (key, (u, w))
    return best[1]


def _h1_edges(X):
    """(birth edge, death edge) of every finite nonzero H1 interval, from the oracle."""
    D = O.distance_matrix(X)
    P = O.barcodes(D, 1, math.inf, O.MODE_COHOM_CLEAR)
    sel = (P.dim == 1) & np.isfinite(P.death) & (P.death > P.birth)
    return sorted((_youngest_edge(D, b), _youngest_edge(D, d))
                  for b, d in zip(P.bverts[sel], P.dverts[sel]))


def _loss64(X, edges):
    X = X.astype(np.float64)
    L = 0.0
    for (bu, bv), (du, dv) in edges:
        L += np.linalg.norm(X[du] - X[dv]) - np.linalg.norm(X[bu] - X[bv])
    return L


def _ref_grad64(X, edges):
    X64 = X.astype(np.float64)
    g = np.zeros_like(X64)
    for (bu, bv), (du, dv) in edges:
        for (u, v), s in (((du, dv), 1.0), ((bu, bv), -1.0)):
            d = X64[u] - X64[v]
            nrm = np.linalg.norm(d)
            g[u] += s * d / nrm
            g[v] -= s * d / nrm
    return g


def _tie_free(X):
    """Every birth and death simplex of a finite H1 interval has a unique
    longest edge (so each endpoint has one realising edge)."""
    D = O.distance_matrix(X)
    P = O.barcodes(D, 1, math.inf, O.MODE_COHOM_CLEAR)
    sel = (P.dim == 1) & np.isfinite(P.death) & (P.death > P.birth)
    for verts in list(P.bverts[sel]) + list(P.dverts[sel]):
        vs = [int(v) for v in verts if v >= 0]
        lengths = sorted((float(D[a, b]) for a, b in itertools.combinations(vs, 2)), reverse=True)
        if len(lengths) > 1 and lengths[0] == lengths[1]:
            return False
    return True


@pytest.fixture(scope="module")
def rpp():
    import __graft_entry__ as g
    g.build()
    import paper_2003_07989_gb300 as m
    return m


def test_backward_matches_oracle_pairing_gradient_batch(rpp):
    import torch
    Xb = I.noisy_circles(256, 128, seed=0)
    pts = torch.from_numpy(Xb).cuda().requires_grad_(True)
    loss = rpp.total_persistence(pts, 1)
    loss.backward()
    g = pts.grad.detach().cpu().numpy()
    ref_loss = 0.0
    for i in range(256):
        edges = _h1_edges(Xb[i])
        ref_loss += _loss64(Xb[i], edges)
        ref = _ref_grad64(Xb[i], edges)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(g[i] - ref).max() <= 1e-5 * scale, i
    assert abs(float(loss.detach()) - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss))


def test_backward_against_finite_differences(rpp):
    import torch
    rng = np.random.default_rng(0)
    checked = skipped = 0
    for seed in range(12):
        X = I.noisy_circles(1, 128, seed=100 + seed)[0]
        if not _tie_free(X):
            skipped += 1
            continue
        edges = _h1_edges(X)
        pts = torch.from_numpy(X).cuda().requires_grad_(True)
        rpp.total_persistence(pts, 1).backward()
        g = pts.grad.detach().cpu().numpy()
        h = 1e-3
        for k in rng.choice(X.size, size=12, replace=False):
            i, j = divmod(int(k), 2)
            Xp, Xm = X.astype(np.float64).copy(), X.astype(np.float64).copy()
            Xp[i, j] += h
            Xm[i, j] -= h
            ep, em = _h1_edges(Xp.astype(np.float32)), _h1_edges(Xm.astype(np.float32))
            if ep != edges or em != edges:  # the pairing moved: not a smooth point
                skipped += 1
                continue
            fd = (_loss64(Xp, edges) - _loss64(Xm, edges)) / (2 * h)
            assert abs(fd - g[i, j]) <= 1e-3 + 1e-2 * abs(g[i, j]), (seed, i, j, fd, g[i, j])
            checked += 1
    assert checked >= 60, (checked, skipped)


def test_backward_is_deterministic(rpp):
    import torch
    Xb = I.noisy_circles(16, 128, seed=5)
    grads = []
    for _ in range(2):
        pts = torch.from_numpy(Xb).cuda().requires_grad_(True)
        rpp.total_persistence(pts, 1).backward()
        grads.append(pts.grad.detach().cpu().numpy())
    assert np.array_equal(grads[0], grads[1])
