"""Long dimension-1 walks of the submatrix reduction, bit-exact against the
oracle.

Clouds with long-lived H1 classes make the reduction of a few leftover
columns add thousands of apparent columns (Alg. 1 in the coboundary matrix,
Sec. "Core System Optimizations"); past a few hundred edges such a walk
sweeps the triangles level by level in diameter instead of listing
coboundaries. These cases make sure the sweep runs (its level counter is
nonzero) and that the barcodes are the oracle's, also with a threshold below
the enclosing radius and with many equal distances (diameter levels holding
several edges, triangles with two or three edges of the same length).
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


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _check(got, ref, max_dim=1):
    for q in range(max_dim + 1):
        a, b = got.intervals[q], ref.barcode(q)
        assert a.shape == b.shape, (q, a.shape, b.shape)
        assert np.array_equal(a, b), q


@pytest.mark.parametrize("n,seed,t", [(500, 1, math.inf), (520, 2, math.inf), (600, 3, 0.8)])
def test_torus_long_walks(rpp, n, seed, t):
    X = I.noisy_torus(n, seed=seed)
    got = rpp.rpp_barcodes(_cuda(X), max_dim=1, threshold=t)
    ref = O.barcodes(O.distance_matrix(X), 1, t, O.MODE_COHOM_CLEAR)
    _check(got, ref)
    assert got.stats["sweep_levels"][1] > 0, "no walk was long enough to sweep"


@pytest.mark.parametrize("scale", [16.0, 64.0])
def test_tie_heavy_long_walks(rpp, scale):
    # torus distances rounded to multiples of 1/scale: most diameter levels
    # hold several edges
    X = I.noisy_torus(480, seed=5)
    D = O.distance_matrix(X).astype(np.float64)
    Dq = (np.round(D * scale) / scale).astype(np.float32)
    np.fill_diagonal(Dq, 0.0)
    got = rpp.rpp_barcodes(_cuda(Dq), max_dim=1, kind="distances")
    ref = O.barcodes(Dq, 1, math.inf, O.MODE_COHOM_CLEAR)
    _check(got, ref)
    assert got.stats["sweep_levels"][1] > 0, "no walk was long enough to sweep"
