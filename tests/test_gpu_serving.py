"""Batched and served barcodes: every result is the same alone and in the mix.

Requests are clouds of uneven size (the serving workload's mixture of noisy
circles, 2-spheres and blobs) with the threshold at the 0.6 nearest-rank
quantile of their distances. Each batched or served result must equal the
single-instance result bit for bit, and a sample equals the CPU oracle.
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


@pytest.fixture(scope="module")
def requests():
    return I.serving_requests(40, seed=3, n_range=(32, 220))


@pytest.fixture(scope="module")
def alone(rpp, requests):
    return [rpp.rpp_barcodes(r.points, max_dim=1, quantile=r.threshold_quantile)
            for r in requests]


def _same(a, b):
    for q in range(len(a.intervals)):
        if not (np.array_equal(a.intervals[q], b.intervals[q])
                and np.array_equal(a.critical[q], b.critical[q])):
            return False
    return True


def test_alone_matches_oracle(requests, alone):
    for r, got in list(zip(requests, alone))[:10]:
        D = O.distance_matrix(r.points)
        t = O.distance_quantile(D, r.threshold_quantile)
        ref = O.barcodes(D, 1, t, O.MODE_COHOM_CLEAR)
        for q in (0, 1):
            assert np.array_equal(got.intervals[q], ref.barcode(q)), (r.index, q)


def test_batched_equals_alone(rpp, requests, alone):
    got = rpp.rpp_barcodes_batched([r.points for r in requests], max_dim=1,
                                   quantiles=[r.threshold_quantile for r in requests])
    assert all(_same(a, b) for a, b in zip(got, alone))


def test_batched_device_inputs(rpp, requests, alone):
    import torch
    clouds = [torch.from_numpy(r.points).cuda() for r in requests[:12]]
    got = rpp.rpp_barcodes_batched(clouds, max_dim=1,
                                   quantiles=[r.threshold_quantile for r in requests[:12]])
    assert all(_same(a, b) for a, b in zip(got, alone[:12]))


@pytest.mark.parametrize("slots,budget_mb", [(4, 0), (8, 64), (2, 24)])
def test_served_equals_alone(rpp, requests, alone, slots, budget_mb):
    srv = rpp.Server(max_slots=slots, device_bytes=budget_mb << 20)
    try:
        tickets = [srv.submit(r.points, 1, quantile=r.threshold_quantile) for r in requests]
        for t, a in zip(tickets, alone):
            assert _same(srv.poll(t), a)
    finally:
        srv.close()


def test_server_rejects_a_request_that_can_never_fit(rpp):
    from paper_2003_07989_gb300 import _native as N
    srv = rpp.Server(max_slots=2, device_bytes=1 << 20)
    try:
        with pytest.raises(N.RppError) as e:
            srv.submit(I.uniform_cube(400, 3, 1), 1)
        assert e.value.status == N.RPP_E_BUSY
        small = I.uniform_cube(20, 3, 2)
        got = srv.poll(srv.submit(small, 1))
        ref = rpp.rpp_barcodes(small, max_dim=1)
        assert _same(got, ref)
    finally:
        srv.close()


def test_server_poll_unknown_ticket(rpp):
    from paper_2003_07989_gb300 import _native as N
    srv = rpp.Server(max_slots=1)
    try:
        with pytest.raises(N.RppError) as e:
            srv.poll(12345, 0)
        assert e.value.status == N.RPP_E_INVALID
    finally:
        srv.close()


def test_served_mixed_buckets_under_load(rpp):
    # many slots launching clouds of every size bucket (32 .. 1024 points, up
    # to 12 dimensions) at once: per-kernel launch limits are shared by all
    # slots, and each result must still equal its single-instance result
    reqs = I.serving_requests(160, seed=11, n_range=(32, 1024), dim_range=(2, 12))
    alone = [rpp.rpp_barcodes(r.points, max_dim=1, quantile=r.threshold_quantile)
             for r in reqs]
    srv = rpp.Server(max_slots=8, max_batch=16)
    try:
        tickets = [srv.submit(r.points, 1, quantile=r.threshold_quantile) for r in reqs]
        for t, a in zip(tickets, alone):
            assert _same(srv.poll(t), a)
    finally:
        srv.close()


def test_server_completion_queue(rpp, requests, alone):
    """rpp_server_next hands every finished request back once, in completion
    order, with the same result as alone; one taken by rpp_server_poll first is
    skipped, and an empty queue times out."""
    from paper_2003_07989_gb300 import _native as N
    srv = rpp.Server(max_slots=4, max_batch=16)
    try:
        assert srv.next(0) is None
        tickets = [srv.submit(r.points, 1, quantile=r.threshold_quantile) for r in requests]
        first = srv.poll(tickets[0])  # taken here, so next() must skip it
        assert _same(first, alone[0])
        seen = {}
        while len(seen) < len(tickets) - 1:
            got = srv.next(60000)
            assert got is not None
            t, res = got
            assert t not in seen and t != tickets[0]
            seen[t] = res
        assert srv.next(0) is None
        for i, t in enumerate(tickets[1:], start=1):
            assert _same(seen[t], alone[i]), i
        with pytest.raises(N.RppError):
            srv.poll(tickets[1], 0)  # already handed out by next()
    finally:
        srv.close()
