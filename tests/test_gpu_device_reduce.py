"""The device reduction of batched clouds' leftover columns (reduce_small.cu).

Clouds of up to 512 points in a fused launch reduce their dimension-1 leftover
columns on the device, one warp per cloud in column order (Alg. 1), and hand a
cloud back to the host when a column's walk outgrows the device's budget. The
barcodes and realising edges must be the host reduction's, bit for bit, and
the oracle's; the serving mix exercises both outcomes (short walks stay on the
device with cursors, circles whose H1 class outlives the threshold sweep by
diameter level in a second phase, and a cloud whose sweep meets a level of
more than 32 equal edges goes back to the host). Mode "wait"
fixes which clouds finish on the device; the default mode lets the host take
a cloud whose device result is not back yet, with the same barcodes.
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


def _ctx(rpp, device):
    c = rpp.Context(0)
    c.set_device_reduce(device)
    return c


def _same(a, b):
    for q in (0, 1):
        assert np.array_equal(a.intervals[q], b.intervals[q]), q
        assert np.array_equal(a.critical[q], b.critical[q]), q


def test_serving_mix_device_equals_host(rpp):
    reqs = I.serving_requests(200, seed=13, n_range=(32, 512))
    clouds = [r.points for r in reqs]
    qs = [r.threshold_quantile for r in reqs]
    dev = rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs, context=_ctx(rpp, "wait"))
    host = rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs, context=_ctx(rpp, False))
    both = rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs, context=_ctx(rpp, True))
    on_device = with_left = 0
    for a, b, c in zip(dev, host, both):
        _same(a, b)
        _same(c, b)
        on_device += a.stats["device_columns"][1] > 0
        with_left += a.stats["leftover"][1] > 0
        assert b.stats["device_columns"][1] == 0
        # the default mode takes a device result or the host's, whole
        assert c.stats["device_columns"][1] in (0, c.stats["leftover"][1])
    assert on_device > with_left * 9 // 10, (on_device, with_left)  # short walks and sweeps alike


def test_device_reduction_matches_oracle(rpp):
    reqs = I.serving_requests(24, seed=17, n_range=(40, 300))
    got = rpp.rpp_barcodes_batched([r.points for r in reqs], max_dim=1,
                                   quantiles=[r.threshold_quantile for r in reqs],
                                   context=_ctx(rpp, "wait"))
    n_dev = 0
    for r, a in zip(reqs, got):
        D = O.distance_matrix(r.points)
        ref = O.barcodes(D, 1, O.distance_quantile(D, r.threshold_quantile))
        n_dev += a.stats["device_columns"][1] > 0
        for q in (0, 1):
            assert np.array_equal(a.intervals[q], ref.barcode(q)), (r.index, r.kind, q)
    assert n_dev > 0


def test_ties_thresholds_and_full_filtrations(rpp):
    grid = np.stack(np.meshgrid(np.arange(12.0), np.arange(11.0)), -1).reshape(-1, 2)
    clouds = [grid.astype(np.float32),                       # many equal distances
              I.uniform_cube(150, 3, seed=3), I.blob_cloud(260, 4, seed=4),
              I.sphere2_cloud(200, 1.0, 0.05, 3, 5), I.uniform_cube(500, 2, seed=6),
              I.circle_cloud(120, 1.0, 0.05, 2, 7)]
    for th in (None, [1.5, 0.25, 1.0, 0.6, 0.08, 0.9]):
        dev = rpp.rpp_barcodes_batched(clouds, max_dim=1, thresholds=th,
                                       context=_ctx(rpp, "wait"))
        host = rpp.rpp_barcodes_batched(clouds, max_dim=1, thresholds=th,
                                        context=_ctx(rpp, False))
        for X, a, b in zip(clouds, dev, host):
            _same(a, b)
        # and the oracle on the small ones
        for i in (0, 1, 5):
            D = O.distance_matrix(clouds[i])
            t = math.inf if th is None else th[i]
            ref = O.barcodes(D, 1, t)
            for q in (0, 1):
                assert np.array_equal(dev[i].intervals[q], ref.barcode(q)), (i, q)


def _lattice_annulus(r_in, r_out):
    g = np.arange(-r_out, r_out + 1, dtype=np.float32)
    P = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)
    r = np.hypot(P[:, 0], P[:, 1])
    return P[(r >= r_in) & (r <= r_out)]


def test_level_ties_go_back_to_the_host(rpp):
    # integer lattice points of an annulus: a long-lived H1 class, so columns
    # sweep, through levels of many equal edges (lengths 1, sqrt 2, 2, ...)
    X = _lattice_annulus(6.0, 9.0)
    assert len(X) <= 512
    clouds = [X, I.circle_cloud(300, 1.0, 0.02, 2, 3)]
    dev = rpp.rpp_barcodes_batched(clouds, max_dim=1, context=_ctx(rpp, "wait"))
    host = rpp.rpp_barcodes_batched(clouds, max_dim=1, context=_ctx(rpp, False))
    for a, b in zip(dev, host):
        _same(a, b)
    assert dev[0].stats["device_columns"][1] == 0          # handed back
    assert dev[1].stats["device_columns"][1] == dev[1].stats["leftover"][1]  # swept on the device
    D = O.distance_matrix(X)
    ref = O.barcodes(D, 1, math.inf)
    for q in (0, 1):
        assert np.array_equal(dev[0].intervals[q], ref.barcode(q)), q
