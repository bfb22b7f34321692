"""rpp_filtration: the filtration construction of one dimension (Alg. 6 and
Alg. 7 without clearing) against the oracle's column list, bit for bit.

The oracle lists every p-simplex with diam <= t as a vertex tuple, sorted by
decreasing diameter then increasing combinatorial index by plain comparison
sorting; the library builds the same list by enumerating indices in runs that
share all but the lowest vertex, compacting with warp ballots and sorting with
its onesweep radix sort. Sizes cover one tile and several tiles of the sort,
ragged tails, ties (integer distances), thresholds below the enclosing radius
and a threshold of zero.
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


def _cidx(verts: np.ndarray) -> np.ndarray:
    """sum_i C(v_i, i+1) over the ascending vertices of every row (exact)."""
    v = np.sort(verts.astype(np.int64), axis=1)
    out = np.zeros(len(v), dtype=np.uint64)
    for i in range(v.shape[1]):
        out += np.array([math.comb(int(x), i + 1) for x in v[:, i]], dtype=np.uint64)
    return out


CASES = [
    ("torus120", lambda: I.noisy_torus(120, seed=1), "points", 1, math.inf),
    ("torus120_p2", lambda: I.noisy_torus(120, seed=1), "points", 2, math.inf),
    ("sphere40_p3", lambda: I.sphere_s3(40, seed=2), "points", 3, math.inf),
    ("cube70_p2_t", lambda: I.uniform_cube(70, 3, seed=3), "points", 2, 0.35),
    ("ties45_p2", lambda: I.integer_distances(45, 5, 4), "distances", 2, math.inf),
    ("blob33_p1_t0", lambda: I.blob_cloud(33, 4, seed=5), "points", 1, 0.0),
    ("circle200_p2_t", lambda: I.circle_cloud(200, 1.0, 0.05, 3, 6), "points", 2, 0.5),
    ("tiny3_p2", lambda: I.uniform_cube(3, 2, seed=7), "points", 2, math.inf),
]


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_filtration_equals_oracle_columns(rpp, idx):
    name, gen, kind, p, t = CASES[idx]
    X = gen()
    D = O.distance_matrix(X) if kind == "points" else X
    diam, cidx, st = rpp.rpp_filtration(X, p, threshold=t, kind=kind)
    t_used = float(np.float32(min(t, O.enclosing_radius(D))))  # the library's float32 t
    assert st["threshold"] == t_used
    od, ov = O.columns(D, p, t_used)
    assert np.array_equal(diam, od), name
    assert np.array_equal(cidx, _cidx(ov)), name
    assert st["candidates"][p] == math.comb(len(D), p + 1)
    assert st["sort_passes"][p] == _passes_needed(od), name


def _passes_needed(diam: np.ndarray) -> int:
    """Radix passes a stable LSD sort of the columns needs when they arrive in
    index order: the key is the diameter's float bits minus their smallest
    value (ascending key = descending diameter after complementing the bits),
    sorted in 9-bit digits, and a digit position where every key has the same
    digit needs no pass."""
    if len(diam) < 2:
        return 0
    key = (~diam.astype(np.float32).view(np.uint32)).astype(np.uint64)
    key -= key.min()
    return sum(1 for k in range(4) if len(np.unique((key >> np.uint64(9 * k)) & np.uint64(511))) > 1)


def test_filtration_into_device_buffers_and_workspace(rpp):
    import torch
    X = I.noisy_torus(300, seed=8)
    D = O.distance_matrix(X)
    ref_d, ref_i, _ = rpp.rpp_filtration(X, 2)
    cap = len(ref_d) + 5
    dd = torch.full((cap,), float("nan"), device="cuda")
    di = torch.zeros(cap, dtype=torch.int64, device="cuda")
    got_d, got_i, st = rpp.rpp_filtration(torch.from_numpy(X).cuda(), 2, out=(dd, di))
    assert np.array_equal(got_d.cpu().numpy(), ref_d)
    assert np.array_equal(got_i.cpu().numpy().astype(np.uint64), ref_i)
    # columns left in the workspace: only the count comes back
    _, _, st2 = rpp.rpp_filtration(X, 2, out=False)
    assert st2["columns"][2] == len(ref_d)
    # a short output is refused and the count still reported
    from paper_2003_07989_gb300 import _native as N
    with pytest.raises(N.RppError):
        rpp.rpp_filtration(X, 2, out=(dd[:10], di[:10]))
    # the edges of the same cloud agree with the oracle at the enclosing radius
    e_d, e_i, _ = rpp.rpp_filtration(X, 1)
    od, ov = O.columns(D, 1, O.enclosing_radius(D))
    assert np.array_equal(e_d, od) and np.array_equal(e_i, _cidx(ov))
