"""The fused batch pass: every cloud's result equals the one-at-a-time pipeline.

rpp_barcodes_batched runs clouds of up to 1024 points (H0-H1) as fused launches
per size bucket (distances, threshold, spanning forest and apparent-pair test
in one block per cloud, a captured CUDA graph per bucket, autotuned launch
shapes). A context with fused=False runs the same clouds one at a time through
the per-instance pipeline; both must agree bit for bit on intervals, realising
edges, thresholds and column counts. Clouds of every bucket (up to 90 points,
and 129-256, 257-512 and 513-1024 points) must also equal the CPU oracle.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_07989_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STAT_KEYS = ("threshold", "enclosing_radius")
# "scanned" counts the candidates a sequential apparent test examines up to its
# exit, whatever launch shape ran it, so both paths must agree on it too
STAT_LISTS = ("candidates", "columns", "cleared", "apparent", "leftover", "intervals",
              "scanned")


@pytest.fixture(scope="module")
def rpp():
    import __graft_entry__ as g
    g.build()
    import paper_2003_07989_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx_fused(rpp):
    return rpp.Context(0)


@pytest.fixture(scope="module")
def ctx_alone(rpp):
    c = rpp.Context(0)
    c.set_batch(fused=False)
    return c


def _same(a, b, stats=True):
    assert len(a.intervals) == len(b.intervals)
    for q in range(len(a.intervals)):
        assert np.array_equal(a.intervals[q], b.intervals[q]), q
        assert np.array_equal(a.critical[q], b.critical[q]), q
    if stats:
        for k in STAT_KEYS:
            assert a.stats[k] == b.stats[k], k
        for k in STAT_LISTS:
            assert a.stats[k][:2] == b.stats[k][:2], k


def _both(rpp, ctx_fused, ctx_alone, clouds, **kw):
    got = rpp.rpp_barcodes_batched(clouds, context=ctx_fused, **kw)
    ref = rpp.rpp_barcodes_batched(clouds, context=ctx_alone, **kw)
    return got, ref


def test_serving_mix_every_bucket(rpp, ctx_fused, ctx_alone):
    reqs = I.serving_requests(160, seed=11, n_range=(2, 1024))
    clouds = [r.points for r in reqs]
    qs = [r.threshold_quantile for r in reqs]
    got, ref = _both(rpp, ctx_fused, ctx_alone, clouds, max_dim=1, quantiles=qs)
    for a, b in zip(got, ref):
        _same(a, b)
    sizes = {r.points.shape[0] for r in reqs}
    assert min(sizes) <= 64 and max(sizes) > 512  # all five buckets ran


def test_full_filtration_and_explicit_thresholds(rpp, ctx_fused, ctx_alone):
    clouds = [I.circle_cloud(n, 1.0, 0.05, d, seed=n) for n, d in
              [(40, 2), (90, 3), (150, 2), (300, 5), (700, 3)]]
    got, ref = _both(rpp, ctx_fused, ctx_alone, clouds, max_dim=1)
    for a, b in zip(got, ref):
        _same(a, b)
    th = [0.3, 0.8, math.inf, 0.05, 1.2]
    got, ref = _both(rpp, ctx_fused, ctx_alone, clouds, max_dim=1, thresholds=th)
    for a, b in zip(got, ref):
        _same(a, b)


def test_h0_only(rpp, ctx_fused, ctx_alone):
    clouds = [I.blob_cloud(n, 4, seed=n) for n in (3, 77, 200, 513)]
    got, ref = _both(rpp, ctx_fused, ctx_alone, clouds, max_dim=0)
    for a, b in zip(got, ref):
        _same(a, b)
        assert len(a.intervals) == 1


def test_degenerate_clouds(rpp, ctx_fused, ctx_alone):
    dup = np.repeat(I.uniform_cube(5, 3, seed=1), 3, axis=0)  # duplicate points: zero H0 deaths
    grid = np.stack(np.meshgrid(np.arange(6.0), np.arange(5.0)), -1).reshape(-1, 2)  # ties
    clouds = [np.zeros((1, 3), np.float32), I.uniform_cube(2, 3, seed=2),
              I.uniform_cube(3, 2, seed=3), dup.astype(np.float32), grid.astype(np.float32),
              np.zeros((9, 2), np.float32)]
    got, ref = _both(rpp, ctx_fused, ctx_alone, clouds, max_dim=1)
    for a, b in zip(got, ref):
        _same(a, b)
    for X, a in zip(clouds, got):  # and the oracle
        D = O.distance_matrix(X)
        res = O.barcodes(D, 1, O.enclosing_radius(D))
        for q in (0, 1):
            assert np.array_equal(a.intervals[q], res.barcode(q)), q


def test_matches_oracle(rpp, ctx_fused):
    reqs = I.serving_requests(12, seed=5, n_range=(20, 90))
    got = rpp.rpp_barcodes_batched([r.points for r in reqs], max_dim=1,
                                   quantiles=[r.threshold_quantile for r in reqs],
                                   context=ctx_fused)
    for r, a in zip(reqs, got):
        D = O.distance_matrix(r.points)
        res = O.barcodes(D, 1, O.distance_quantile(D, r.threshold_quantile))
        for q in (0, 1):
            assert np.array_equal(a.intervals[q], res.barcode(q)), (r.index, q)


@pytest.mark.parametrize("lo,hi,nmax", [(129, 256, 256), (257, 512, 512), (513, 1024, 1024)])
def test_large_buckets_match_oracle(rpp, lo, hi, nmax):
    """The fused kernel's larger buckets against the oracle itself: the
    257-512 bucket keeps the spanning forest as a shared-memory bitmap and
    the 513-1024 bucket finds forest edges by binary search, so each bucket's
    own code path is compared with the CPU oracle, interval by interval, on
    serving-mix clouds at the 0.6 quantile (a fresh context, so the bucket's
    tuning record shows that the fused launch ran)."""
    reqs = I.serving_requests(4, seed=31 + lo, n_range=(lo, hi))
    ctx = rpp.Context(0)
    got = rpp.rpp_barcodes_batched([r.points for r in reqs], max_dim=1,
                                   quantiles=[r.threshold_quantile for r in reqs], context=ctx)
    assert ctx.batch_tuning(nmax) != (0, 0)
    for r, a in zip(reqs, got):
        assert lo <= r.points.shape[0] <= hi
        D = O.distance_matrix(r.points)
        t = O.distance_quantile(D, r.threshold_quantile)
        # the library cuts at min(t, enclosing radius), which leaves every
        # nonzero interval unchanged; the oracle takes t itself
        assert a.stats["threshold"] == min(t, O.enclosing_radius(D))
        res = O.barcodes(D, 1, t)
        for q in (0, 1):
            assert np.array_equal(a.intervals[q], res.barcode(q)), (r.index, r.kind, q)


def test_launches_split_at_bucket_capacity(rpp, ctx_fused, ctx_alone):
    # the 1024-point bucket holds 64 clouds per launch: 70 clouds take two launches
    clouds = [I.uniform_cube(520 + (i % 7), 2, seed=100 + i) for i in range(70)]
    got, ref = _both(rpp, ctx_fused, ctx_alone, clouds, max_dim=1, quantiles=[0.3] * 70)
    for a, b in zip(got, ref):
        _same(a, b)


def test_tuned_and_default_shapes_agree(rpp, ctx_fused):
    reqs = I.serving_requests(48, seed=8, n_range=(100, 250))
    clouds = [r.points for r in reqs]
    qs = [r.threshold_quantile for r in reqs]
    tuned = rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs, context=ctx_fused)
    threads, group = ctx_fused.batch_tuning(256)
    # group: lanes per column, or 10 x lanes + candidate blocks per step
    assert threads in (128, 256, 512, 1024) and group in (4, 8, 16, 42, 44)
    plain = rpp.Context(0)
    plain.set_batch(fused=True, autotune=False)
    default = rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs, context=plain)
    assert plain.batch_tuning(256) == (0, 0)
    for a, b in zip(tuned, default):
        _same(a, b)
    again = rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs, context=ctx_fused)  # graph replay
    for a, b in zip(tuned, again):
        _same(a, b)


def test_mixed_host_and_device_inputs(rpp, ctx_fused, ctx_alone):
    import torch
    reqs = I.serving_requests(10, seed=21, n_range=(30, 300))
    clouds = [torch.from_numpy(r.points).cuda() if i % 2 else r.points
              for i, r in enumerate(reqs)]
    qs = [r.threshold_quantile for r in reqs]
    got = rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs, context=ctx_fused)
    ref = rpp.rpp_barcodes_batched([r.points for r in reqs], max_dim=1, quantiles=qs,
                                   context=ctx_alone)
    for a, b in zip(got, ref):
        _same(a, b)


def test_non_finite_points_are_rejected(rpp, ctx_fused):
    bad = I.uniform_cube(30, 3, seed=4)
    bad[7, 1] = np.nan
    with pytest.raises(rpp.RppError):
        rpp.rpp_barcodes_batched([I.uniform_cube(20, 3, seed=5), bad], max_dim=1,
                                 context=ctx_fused)
    # the context stays usable
    ok = rpp.rpp_barcodes_batched([I.uniform_cube(20, 3, seed=5)], max_dim=1, context=ctx_fused)
    assert len(ok) == 1
