"""The apparent-pair census (rpp_apparent_census): the dimension-1 apparent-pair
pass on the full filtration without the reduction (Sec. "Experiments on the
Apparent Pairs Rate").

Small inputs: the census counts equal the oracle's apparent pairs by their
definition on the full filtration, and the counts partition the C(n,2) edges.
Random total orders of the edges (the paper's random permutations of
1..C(n,2)): the apparent fraction obeys the theorem's upper bound
(n-2)/n, and at 10,000 points it is the paper's 0.991127743 (the average of
ten samples, whose spread the paper calls very low) within 0.002.
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


@pytest.mark.parametrize("case", ["torus60", "rank45", "cube50", "ties40", "sphere192"])
def test_census_equals_oracle(rpp, case):
    if case == "sphere192":  # the stand-in for the paper's sphere_3_192 (its Table of
        # apparent percentages per dimension counts pairs of the full filtration)
        D = O.distance_matrix(I.sphere_s3(192, seed=0))
    elif case == "torus60":
        D = O.distance_matrix(I.noisy_torus(60, seed=3))
    elif case == "rank45":
        D = I.rank_distances(45, seed=1)
    elif case == "cube50":
        D = O.distance_matrix(I.uniform_cube(50, 3, seed=0))
    else:
        D = I.integer_distances(40, levels=4, seed=2)
    n = len(D)
    st = rpp.rpp_apparent_census(D, kind="distances")
    sigma, _ = O.apparent_pairs(D, 1, math.inf)
    m = n * (n - 1) // 2
    assert st["candidates"][1] == m
    assert st["apparent"][1] == len(sigma)
    assert st["cleared"][1] == n - 1  # every case is connected
    assert st["cleared"][1] + st["apparent"][1] + st["leftover"][1] == m


def test_census_points_and_distances_agree(rpp):
    X = I.noisy_torus(300, seed=4)
    a = rpp.rpp_apparent_census(X)
    b = rpp.rpp_apparent_census(O.distance_matrix(X), kind="distances")
    for k in ("candidates", "cleared", "apparent", "leftover"):
        assert a[k][1] == b[k][1], k


@pytest.mark.parametrize("n", [200, 1000])
def test_census_upper_bound_on_random_orders(rpp, n):
    st = rpp.rpp_apparent_census(I.rank_distances(n, seed=n), kind="distances")
    assert st["apparent"][1] <= math.comb(n - 1, 2)  # fraction <= (n - 2) / n


def test_census_random_orders_10000_points(rpp):
    import torch
    n = 10000
    D = torch.from_numpy(I.rank_distances(n, seed=0)).cuda()
    st = rpp.rpp_apparent_census(D, kind="distances")
    frac = st["apparent"][1] / st["candidates"][1]
    assert abs(frac - 0.991127743) < 0.002, frac
