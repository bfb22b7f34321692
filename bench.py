#!/usr/bin/env python
"""Benchmark of the barcode hot path on the 2000-point noisy torus (H0-H1).

One step = one full barcode computation of one synthetic cloud already
resident in device memory: distance matrix, enclosing radius, filtration with
clearing, radix sort, Kruskal H0, apparent-pair pass, partition, submatrix
reduction, barcode assembly. The metric is simplices/s through the
apparent-pair pass: columns tested (the dimension-1 simplices inside the
threshold that clearing kept) per second of whole-step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank computes its own cloud (seed = rank); the value is the
columns of all ranks divided by the slowest rank's time (weak scaling).
`--impl reference` times the CPU oracle in its COHOM_CLEAR mode (Kruskal H0,
then Alg. 1 on the coboundary matrix with the clearing lemma; no apparent
pairs) on a bounded sample of the same workload on the host cores: the first
500 of the torus's points per step, which its config states.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_POINTS, DIM, MAX_DIM = 2000, 3, 1
WORKLOAD = "torus2000_h1"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB of L2


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=4096,
                    help="requests of the serving section (0 skips it)")
    ap.add_argument("--serving-slots", type=int, default=8)
    ap.add_argument("--no-census", action="store_true",
                    help="skip the apparent-pair census of random edge orders")
    ap.add_argument("--profile-batched", action="store_true",
                    help="profiling aid: one batched call over the serving mix's clouds of "
                         "257-512 points inside an NVTX range 'batched' (after an untimed "
                         "call), then exit")
    ap.add_argument("--profile-filtration", action="store_true",
                    help="profiling aid: the dimension-2 filtration (build and sort, no "
                         "clearing) of the first 1000 torus points, three times, then exit")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the torus steps: no serving, census, differentiation or S^3 section")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2003_07989_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


STAGE_FILES = {
    "apparent": ["apparent.cu", "device_common.cuh"],
    "sort_columns": ["radix_sort.cu"],
    "sort_pairs": ["radix_sort.cu"],
    "build_columns": ["filtration.cu", "device_common.cuh"],
    "partition": ["apparent.cu"],
}


def traffic_for(stage, key="dram_bytes_per_launch"):
    """Bytes per launch (DRAM by default; `key` names another counter) from a
    committed ncu summary, if it was taken on the current source of the
    kernel; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p) or stage not in STAGE_FILES:
        return None
    d = json.load(open(p)).get(stage)
    if not d or d.get("source_hash") != kernel_source_hash(STAGE_FILES[stage]):
        return None
    return d.get(key)


def algorithmic_bytes(stage, st):
    """Bytes a stage must move per launch by its definition: the per-unit
    figures (distance reads per examined candidate, key and output bytes per
    column, key bytes per sort pass) times the units of one launch."""
    p = 1
    cols = st["columns"][p] + st["cleared"][p]
    if stage == "apparent":
        # the measurement plan's per-unit figure: (p+1) distance reads of 4 B
        # per candidate a sequential scan examines, (p+1) p / 2 more for the
        # facet test (one for p = 1), 12 B of column key in and 9 B out
        # (status and pivot) per column
        return (st["scanned"][p] * (p + 1) * 4 + cols * (p + 1) * p // 2 * 4
                + cols * (12 + 9))
    if stage == "build_columns":
        return st["candidates"][p] * 4 + cols * 12
    if stage in ("sort_columns", "sort_pairs"):
        # the column sort reports the passes that ran (digits that were not
        # constant); the pair sort's launches are (histogram, offsets, one per
        # digit position, finish)
        if stage == "sort_columns":
            passes = st["sort_passes"][p]
        else:
            passes = max(0, st["stage_launches"][6] - 3)
        n = cols if stage == "sort_columns" else st["apparent"][p]
        w = 12 if stage == "sort_columns" else 16
        return n * w + passes * n * 2 * w  # histogram read + per pass one read and one write
    if stage == "partition":
        return cols * (1 + 12 + 12) + st["apparent"][p] * 16 + st["leftover"][p] * 32
    return None


# ---------------------------------------------------------------------------
# serving: plain one-at-a-time path vs the continuous-batching server


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]


def serving_bench(rpp, count: int, slots: int):
    """Barcodes/s at saturation and p50/p99 latency under Poisson arrivals at
    0.8 x the plain path's sustained rate, for the plain path (the same
    library, one request at a time, synchronous) and for the server (one
    long-running server, measured after an untimed pass over the requests)."""
    import threading
    from paper_2003_07989_gb300 import inputs as I
    reqs = I.serving_requests(count, seed=0)
    for r in reqs[:8]:
        rpp.rpp_barcodes(r.points, max_dim=1, quantile=r.threshold_quantile)
    # warm-up of the fused batch path: the autotuner picks each size bucket's
    # launch shape on first use, outside every timed run below
    clouds = [r.points for r in reqs]
    qs = [r.threshold_quantile for r in reqs]
    rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs)
    # batched: all requests in one call (fused launches per size bucket)
    t0 = time.perf_counter()
    rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs)
    batched_s = time.perf_counter() - t0
    # plain, saturation
    t0 = time.perf_counter()
    for r in reqs:
        rpp.rpp_barcodes(r.points, max_dim=1, quantile=r.threshold_quantile)
    plain_s = time.perf_counter() - t0
    plain_rps = count / plain_s
    lam = 0.8 * plain_rps
    arrivals = [r.arrival_s for r in I.serving_requests(count, rate_per_s=lam, seed=0)]

    def plain_poisson():
        lat, start = [], time.perf_counter()
        for r, a in zip(reqs, arrivals):
            now = time.perf_counter() - start
            if now < a:
                time.sleep(a - now)
            rpp.rpp_barcodes(r.points, max_dim=1, quantile=r.threshold_quantile)
            lat.append(time.perf_counter() - start - a)
        return lat

    # one long-running server: its slots' workspaces are allocated by an
    # untimed pass, as a serving process would have them after start-up
    srv = rpp.Server(max_slots=slots, max_batch=64)

    def served(arr):
        done = {}
        tickets = []
        lock = threading.Lock()
        finished = threading.Event()

        def poller():  # results in completion order (rpp_server_next), timed on return
            while True:
                with lock:
                    all_in = finished.is_set() and len(done) == len(tickets)
                if all_in:
                    return
                got = srv.next(20)
                if got is not None:
                    done[got[0]] = time.perf_counter()

        th = threading.Thread(target=poller)
        start = time.perf_counter()
        th.start()
        for r, a in zip(reqs, arr):
            now = time.perf_counter() - start
            if now < a:
                time.sleep(a - now)
            t = srv.submit(r.points, 1, quantile=r.threshold_quantile)
            with lock:
                tickets.append(t)
        finished.set()
        th.join()
        end = max(done.values())
        lat = [done[tickets[i]] - start - arr[i] for i in range(count)]
        return lat, end - start

    plain_lat = plain_poisson()
    served([0.0] * count)  # warm-up pass
    _, sat_s = served([0.0] * count)
    srv_lat, _ = served(arrivals)
    srv.close()
    return {
        "requests": count, "slots": slots, "poisson_rate_per_s": lam,
        "plain": {"barcodes_per_s": plain_rps, "p50_ms": 1e3 * _pct(plain_lat, 0.5),
                  "p99_ms": 1e3 * _pct(plain_lat, 0.99)},
        "served": {"barcodes_per_s": count / sat_s, "p50_ms": 1e3 * _pct(srv_lat, 0.5),
                   "p99_ms": 1e3 * _pct(srv_lat, 0.99), "max_batch": 64},
        "batched": {"barcodes_per_s": count / batched_s,
                    "note": "one rpp_barcodes_batched call over every request (fused launches)"},
        "workload": "serving mix: n uniform in [32, 512], dim uniform in [2, 8], circle/2-sphere/"
                    "blob, threshold = 0.6 nearest-rank distance quantile, H0-H1, seed 0",
    }


# ---------------------------------------------------------------------------
# differentiation: total H1 persistence of a batch of noisy circles, backward


def backward_bench(rpp, torch, dev, reps: int = 10):
    """Forward (batched barcodes) + backward (gradients to the points) of the
    total H1 persistence of 256 noisy planar circles of 128 points."""
    import numpy as np
    from paper_2003_07989_gb300 import inputs as I
    X = torch.from_numpy(np.ascontiguousarray(I.noisy_circles(256, 128, seed=0))).to(dev)
    for _ in range(2):
        pts = X.clone().requires_grad_(True)
        rpp.total_persistence(pts, 1).backward()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(reps):
        pts = X.clone().requires_grad_(True)
        loss = rpp.total_persistence(pts, 1)
        loss.backward()
    torch.cuda.synchronize(dev)
    dt = (time.perf_counter() - t0) / reps
    return {"clouds": 256, "points": 128, "ms_per_batch": 1e3 * dt,
            "clouds_per_s": 256 / dt, "loss": float(loss.detach()),
            "workload": "256 noisy planar circles of 128 points (radius U[0.5,2], sigma 0.05), "
                        "loss = total H1 persistence, forward + backward to the points"}


# ---------------------------------------------------------------------------
# 192 points on S^3, H0-H2 (the stand-in for the paper's sphere_3_192)


def sphere_bench(rpp, torch, dev, reps: int = 10, stream_count: int = 512):
    """Time per barcode of 192 points on S^3 with H0-H2 (full filtration)
    alone; its apparent fraction per dimension beside the paper's for its
    sphere_3_192 dataset (another sample of the same distribution); and its
    latency as one large request submitted to the server amid a Poisson
    stream of small serving-mix requests, with that stream's p99."""
    import threading
    from paper_2003_07989_gb300 import inputs as I
    X = I.sphere_s3(192, seed=0)
    pts = torch.from_numpy(X).to(dev)
    for _ in range(2):
        rpp.rpp_barcodes(pts, max_dim=2)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(reps):
        b = rpp.rpp_barcodes(pts, max_dim=2)
    torch.cuda.synchronize(dev)
    alone_ms = 1e3 * (time.perf_counter() - t0) / reps
    st = b.stats
    frac = {str(q): st["apparent"][q] / st["columns"][q] for q in (1, 2) if st["columns"][q]}
    # the paper's table counts pairs of the full filtration (no enclosing-radius
    # cut): dimension 1 has C(n-1, 2) of them; the census runs that filtration
    cs = rpp.rpp_apparent_census(pts)
    full1 = cs["apparent"][1] / math.comb(191, 2)
    # the same request amid a stream of small ones; one untimed pass first
    # (the fused buckets' autotuning, the slots' first allocations)
    reqs = I.serving_requests(stream_count, rate_per_s=2000.0, seed=1)
    rpp.rpp_barcodes_batched([r.points for r in reqs], max_dim=1,
                             quantiles=[r.threshold_quantile for r in reqs])
    at = reqs[len(reqs) // 2].arrival_s  # the large request arrives mid-stream
    srv = rpp.Server(max_slots=8, max_batch=64)

    def one_pass():
        done, sub = {}, {}
        lock = threading.Lock()
        finished = threading.Event()

        def poller():
            while True:
                with lock:
                    if finished.is_set() and len(done) == len(sub):
                        return
                got = srv.next(20)
                if got is not None:
                    done[got[0]] = time.perf_counter()

        th = threading.Thread(target=poller)
        start = time.perf_counter()
        th.start()
        big = None
        for r in reqs:
            if big is None and r.arrival_s >= at:
                now = time.perf_counter() - start
                if now < at:
                    time.sleep(at - now)
                big = srv.submit(X, 2)
                with lock:
                    sub[big] = at
            now = time.perf_counter() - start
            if now < r.arrival_s:
                time.sleep(r.arrival_s - now)
            t = srv.submit(r.points, 1, quantile=r.threshold_quantile)
            with lock:
                sub[t] = r.arrival_s
        finished.set()
        th.join()
        return {t: 1e3 * (done[t] - start - a) for t, a in sub.items()}, big

    one_pass()
    lat, big = one_pass()
    srv.close()
    small = sorted(v for t, v in lat.items() if t != big)
    return {"n": 192, "max_dim": 2, "ms_alone": alone_ms,
            "columns": {str(q): st["columns"][q] for q in (1, 2)},
            "apparent_fraction": frac,
            "apparent_of_all_pairs_dim1_full_filtration": full1,
            "paper_apparent_of_all_pairs_sphere_3_192": {"1": 0.99707909, "2": 0.99734764},
            "served_ms": lat[big], "stream_requests": len(small),
            "stream_p50_ms": small[len(small) // 2],
            "stream_p99_ms": small[min(len(small) - 1, int(0.99 * len(small)))],
            "workload": "192 points uniform on S^3 (normalised Gaussian 4-vectors, seed 0), "
                        "full filtration, H0-H2; served amid 512 serving-mix requests "
                        "(Poisson, 2000/s, seed 1)"}


# ---------------------------------------------------------------------------
# apparent-pair census of random edge orders (the paper's apparent-rate experiment)


def l2_read_peak(rpp, torch, dev, reps: int = 64, trials: int = 5):
    """The L2 read bandwidth of this GPU, measured by the library's probe
    (rpp_l2_read_probe): a 16 MB buffer, the size of the 2000-point distance
    matrix the apparent-pair pass reads, brought into L2 by one launch, then
    read `reps` times per launch with L2-only loads; best of `trials` launches
    per grid shape, CUDA events on the launching stream."""
    nbytes = 16 << 20
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    buf = torch.ones(nbytes // 4, dtype=torch.int32, device=dev)
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    shapes = {}
    for per_sm in (2, 4, 8):
        blocks = per_sm * sms
        rpp.rpp_l2_read_probe(buf, 1, blocks, sink, stream)
        best = None
        for _ in range(trials):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rpp.rpp_l2_read_probe(buf, reps, blocks, sink, stream)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        shapes[f"{per_sm}x{sms}x512"] = nbytes * reps / (best / 1e3) / 1e9
    # every word is 1: the counter holds the number of words read (mod 2^32)
    words = (nbytes // 4) * (1 + trials * reps) * len(shapes)
    ok = int(sink.item()) % (1 << 32) == words % (1 << 32)
    top = max(shapes, key=shapes.get)
    return {"gbs": shapes[top], "grid": top, "per_grid_gbs": shapes, "buffer_bytes": nbytes,
            "reps_per_launch": reps, "words_checked": ok,
            "method": "rpp_l2_read_probe: ld.global.cg (L2 only) reads of an L2-resident "
                      "buffer, best of %d launches per grid" % trials}


def filtration_bench(rpp, torch, dev, reps: int = 5):
    """The HBM-bound stage: the dimension-2 filtration (every triangle inside
    the enclosing radius, no clearing) of the 2000-point torus, built and
    radix-sorted on the device through rpp_filtration, the columns left in the
    workspace. Build: 1.33e9 candidates decoded, 12 B written per kept
    triangle. Sort: per pass one read and one write of the 12-byte keys, plus
    the histogram sweep (12 B) and the minimum sweep (4 B)."""
    from paper_2003_07989_gb300 import _native as N
    from paper_2003_07989_gb300 import inputs as I
    X = torch.from_numpy(I.noisy_torus(N_POINTS, seed=0)).to(dev)
    ctx = rpp.Context(dev.index or 0, record=N.RPP_RECORD_TIMING)
    try:
        rpp.rpp_filtration(X, 2, out=False, context=ctx)  # allocation, first launch
        torch.cuda.synchronize(dev)
        builds, sorts, st = [], [], None
        for _ in range(reps):
            _, _, st = rpp.rpp_filtration(X, 2, out=False, context=ctx)
            builds.append(st["stage_ms"][2])
            sorts.append(st["stage_ms"][3])
        m = st["columns"][2]
        cand = st["candidates"][2]
        passes = st["sort_passes"][2]  # digit positions that were not constant
        build_ms, sort_ms = statistics.median(builds), statistics.median(sorts)
        build_bytes = 12 * m + 4 * N_POINTS * N_POINTS  # columns written, D read once
        sort_bytes = m * (4 + 12 + passes * 24)
        peak, kind = measured_peaks()
        return {
            "workload": "2000-point noisy torus (seed 0), dimension-2 columns inside the "
                        "enclosing radius, no clearing; build + radix sort on the device",
            "candidates": cand, "columns": m, "sort_passes": passes,
            "build_ms": build_ms, "sort_ms": sort_ms,
            "build_gbs": build_bytes / (build_ms / 1e3) / 1e9,
            "sort_gbs": sort_bytes / (sort_ms / 1e3) / 1e9,
            "build_frac_of_hbm": build_bytes / (build_ms / 1e3) / 1e9 / peak,
            "sort_frac_of_hbm": sort_bytes / (sort_ms / 1e3) / 1e9 / peak,
            "peak_gbs": peak, "peak_source": kind,
            "candidates_per_s": cand / (build_ms / 1e3),
            "keys_sorted_per_s": m / (sort_ms / 1e3),
        }
    finally:
        ctx.close()
        del X
        torch.cuda.empty_cache()


def sparse_bench(rpp, torch, dev, reps: int = 3, t: float = 1.4, max_dim: int = 2):
    """The thresholded workload (the paper's sparse o3 row): 4096 random
    matrices of O(3) as points of R^9, threshold 1.4 (about 2.8% of the
    edges), H0-H2. C(4096, 3) > 2^32, so only the thresholded construction of
    dimension 2 (cliques of the threshold graph) can run it. Times the whole
    call from device-resident points (CUDA events), its stages, and the
    dimension-2 columns per second through the apparent-pair pass."""
    from paper_2003_07989_gb300 import _native as N
    from paper_2003_07989_gb300 import inputs as I
    X = torch.from_numpy(I.orthogonal3(4096, seed=0)).to(dev)
    ctx = rpp.Context(dev.index or 0, record=N.RPP_RECORD_TIMING)
    try:
        rpp.rpp_barcodes(X, max_dim=max_dim, threshold=t, context=ctx)  # allocation, tuning
        stream = torch.cuda.current_stream(dev)
        times, res = [], None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = rpp.rpp_barcodes(X, max_dim=max_dim, threshold=t, context=ctx)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        st = res.stats
        ms = statistics.median(times)
        return {
            "workload": f"4096 random O(3) matrices in R^9 (seed 0), threshold {t}, "
                        f"H0-H{max_dim}, thresholded construction of dimensions >= 2",
            "ms": ms, "sparse": st["sparse"][:max_dim + 1],
            "edges_inside_t": st["columns"][1] + st["cleared"][1],
            "columns": st["columns"][:max_dim + 1], "apparent": st["apparent"][:max_dim + 1],
            "leftover": st["leftover"][:max_dim + 1],
            "intervals": [len(iv) for iv in res.intervals],
            "stage_ms": dict(zip(N.STAGES, [round(x, 4) for x in st["stage_ms"]])),
            "host_reduce_ms": st["ms_host_reduce"],
            "simplices_per_s": sum(st["columns"][1:max_dim + 1]) / (ms / 1e3),
        }
    finally:
        ctx.close()
        del X
        torch.cuda.empty_cache()


def census_bench(rpp, torch, dev, ctx):
    """Dimension-1 apparent fraction of uniformly random total orders of the
    C(n,2) edges (the paper's random permutations of 1..C(n,2)), full
    filtration, one sample per n; beside the paper's value at 10,000 points
    (the average of ten samples) and the theorem's upper bound (n-2)/n."""
    from paper_2003_07989_gb300 import inputs as I
    out = []
    for n in (1000, 4000, 10000):
        D = torch.from_numpy(I.rank_distances(n, seed=0)).to(dev)
        rpp.rpp_apparent_census(D, kind="distances", context=ctx)  # warm-up (allocations)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st = rpp.rpp_apparent_census(D, kind="distances", context=ctx)
        wall = time.perf_counter() - t0
        frac = st["apparent"][1] / st["candidates"][1]
        out.append({"n": n, "edges": st["candidates"][1], "apparent": st["apparent"][1],
                    "fraction": frac, "upper_bound": (n - 2) / n,
                    "apparent_pass_ms": st["stage_ms"][4], "wall_ms": 1e3 * wall,
                    "edges_per_s": st["candidates"][1] / wall})
        del D
    return {"samples": out, "paper_fraction_at_10000": 0.991127743,
            "workload": "random total order of the edges (distinct float32 values), seed 0, "
                        "dimension 1, full filtration, no reduction"}


# ---------------------------------------------------------------------------
# the oracle as the CPU baseline / reference arm


def oracle_rate(n_sample: int, seed: int):
    """The oracle in its COHOM_CLEAR mode (Kruskal H0, then the standard
    reduction of the coboundary matrix with the clearing lemma) on the first
    n_sample points of the same torus cloud: dimension-1 columns processed per
    second, and the threads it used."""
    from oracle import oracle as O
    from paper_2003_07989_gb300 import inputs as I
    X = I.noisy_torus(N_POINTS, seed=seed)[:n_sample]
    D = O.distance_matrix(X)
    t0 = time.perf_counter()
    O.barcodes(D, MAX_DIM, math.inf, O.MODE_COHOM_CLEAR)
    dt = time.perf_counter() - t0
    cols = n_sample * (n_sample - 1) // 2 - (n_sample - 1)  # every edge but the cleared MST
    return cols / dt, dt, cols, O.num_threads()


def over_ranks(dist, slowest, summed, device):
    """The job's figures from every rank's: the maximum of `slowest` (times:
    the slowest rank bounds the job) and the sum of `summed` (work done)."""
    import torch
    mx = torch.tensor(slowest, dtype=torch.float64, device=device)
    sm = torch.tensor(summed, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx.tolist(), sm.tolist()


def bench_config(world: int) -> dict:
    """The workload both arms report (the oracle computes the same barcodes of
    the full filtration; the library cuts it at the enclosing radius, which
    leaves every nonzero interval unchanged)."""
    return {"workload": WORKLOAD, "n": N_POINTS, "dim": DIM, "max_dim": MAX_DIM,
            "threshold": "none (full filtration)", "seed": "rank",
            "l2": "flushed between steps (512 MB write, outside the timed events)",
            "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    n_sample = 500
    for _ in range(args.warmup):
        oracle_rate(n_sample, 0)
    rates, secs, cols = [], 0.0, 0
    cores = 1
    for _ in range(args.steps):
        r, dt, c, cores = oracle_rate(n_sample, 0)
        rates.append(r)
        secs += dt
        cols += c
    value = cols / secs
    line = {
        "impl": "reference", "metric": "simplices/s in apparent-pair pass", "value": value,
        "unit": "simplices/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(bench_config(world), sample_points=n_sample,
                       sample=f"each step computes the first {n_sample} of the {N_POINTS} "
                              f"torus points"),
        "cpu_baseline": {"value": value, "unit": "simplices/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {n_sample} of the 2000 torus points per step"},
        "e2e": {"value": value, "unit": "simplices/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_2003_07989_gb300 as rpp
    from paper_2003_07989_gb300 import _native as N
    from paper_2003_07989_gb300 import inputs as I

    torch.cuda.set_device(local)
    if args.profile_filtration:
        X = torch.from_numpy(I.noisy_torus(N_POINTS, seed=0)[:1000]).cuda()
        c = rpp.Context(local)
        for _ in range(3):
            _, _, st = rpp.rpp_filtration(X, 2, out=False, context=c)
        torch.cuda.synchronize()
        print(json.dumps({"profile_filtration": 1000, "columns": st["columns"][2],
                          "candidates": st["candidates"][2]}))
        return
    if args.profile_batched:
        reqs = [r for r in I.serving_requests(4096, seed=0) if r.points.shape[0] > 256]
        clouds = [r.points for r in reqs]
        qs = [r.threshold_quantile for r in reqs]
        rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs)  # autotuning, allocations
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("batched")
        t0 = time.perf_counter()
        out = rpp.rpp_barcodes_batched(clouds, max_dim=1, quantiles=qs)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_batched": len(clouds), "ms": 1e3 * dt,
                          "h1_intervals": sum(len(b.intervals[1]) for b in out)}))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    ctx = rpp.Context(local, record=N.RPP_RECORD_TIMING)
    X = I.noisy_torus(N_POINTS, seed=rank)
    pts = torch.from_numpy(X).to(dev)
    pts_host = torch.from_numpy(X).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(data):
        """K steps, each bracketed by events on the launching stream; L2 is
        flushed between steps, outside the events."""
        total_ms, stats = 0.0, []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = rpp.rpp_barcodes(data, max_dim=MAX_DIM, context=ctx)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            stats.append(res)
        return total_ms, stats

    for _ in range(args.warmup):
        rpp.rpp_barcodes(pts, max_dim=MAX_DIM, context=ctx)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    total_ms, results = timed(pts)
    barrier()
    clk = clocks.stop()

    # end to end through the public API from pinned host memory
    for _ in range(max(1, args.warmup // 2)):
        rpp.rpp_barcodes(pts_host, max_dim=MAX_DIM, context=ctx)
    barrier()
    e2e_ms, e2e_results = timed(pts_host)
    barrier()

    st = [r.stats for r in results]
    cols_rank = sum(s["columns"][1] for s in st)
    e2e_cols_rank = sum(r.stats["columns"][1] for r in e2e_results)
    launches_rank = sum(s["kernel_launches"] for s in st)
    (total_ms, e2e_ms), (cols_all, e2e_cols_all, launches_all) = over_ranks(
        dist, [total_ms, e2e_ms], [cols_rank, e2e_cols_rank, launches_rank], dev)
    if rank != 0:
        dist.destroy_process_group()
        return

    value = cols_all / (total_ms / 1000.0)
    e2e_value = e2e_cols_all / (e2e_ms / 1000.0)
    # per-stage breakdown (rank 0)
    stage_ms = [sum(s["stage_ms"][i] for s in st) / len(st) for i in range(8)]
    stage_launch = [st[0]["stage_launches"][i] for i in range(8)]
    names = N.STAGES
    kernels = {names[i]: {"ms_per_step": round(stage_ms[i], 4), "launches_per_step": stage_launch[i]}
               for i in range(8)}
    # dominant single kernel (stages launched as one kernel per step); the sort
    # stages are several kernels each and are reported in the breakdown
    cand = ["build_columns", "apparent", "partition", "distance"]
    dom = max(cand, key=lambda k: stage_ms[names.index(k)] / max(1, stage_launch[names.index(k)]))
    i = names.index(dom)
    launches = max(1, stage_launch[i])
    dur_s = stage_ms[i] / 1000.0 / launches
    alg = algorithmic_bytes(dom, st[0])
    peak, peak_kind = measured_peaks()
    achieved = (alg / launches) / dur_s / 1e9 if (alg and dur_s > 0) else None
    s0 = st[0]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": traffic_for(dom), "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": (alg / launches) if alg else None,
                "avg_launch_ms": dur_s * 1000.0}
    # the apparent pass's rows stay in L2: its L2 read bytes (ncu, same
    # kernel source) over its live launch time, against the probe's L2 peak
    l2 = l2_read_peak(rpp, torch, dev)
    l2_read = traffic_for(dom, "l2_read_bytes_per_launch")
    roofline["l2"] = {"achieved": (l2_read / dur_s / 1e9) if (l2_read and dur_s > 0) else None,
                      "peak": l2["gbs"], "unit": "GB/s", "peak_source": "measured (probe)",
                      "frac": (l2_read / dur_s / 1e9 / l2["gbs"]) if (l2_read and dur_s > 0)
                      else None,
                      "l2_read_bytes_per_launch": l2_read, "probe": l2}

    cpu = None
    if not args.no_cpu_baseline:
        r, dt, c, cores = oracle_rate(1000, 0)
        cpu = {"value": r, "unit": "simplices/s", "cores": cores, "kind": "oracle",
               "sample": f"first 1000 of the 2000 torus points ({c} dimension-1 columns, "
                         f"{dt:.1f} s)"}
    serving = None
    if args.serving_requests > 0 and not args.no_extras:
        serving = serving_bench(rpp, args.serving_requests, args.serving_slots)
    census = None if (args.no_census or args.no_extras) else census_bench(rpp, torch, dev, ctx)
    backward = None if args.no_extras else backward_bench(rpp, torch, dev)
    sphere = None if args.no_extras else sphere_bench(rpp, torch, dev)
    filtration = None if args.no_extras else filtration_bench(rpp, torch, dev)
    sparse = None if args.no_extras else sparse_bench(rpp, torch, dev)
    h2d = X.nbytes
    d2h = sum(len(iv) * (8 + 16) for iv in e2e_results[0].intervals)
    line = {
        "metric": "simplices/s in apparent-pair pass", "value": value, "unit": "simplices/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(world),
        "e2e": {"value": e2e_value, "unit": "simplices/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps},
        "gpu_launches": int(launches_all),
        "clocks": clk,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "serving": serving,
        "apparent_census": census,
        "differentiation": backward,
        "sphere_h2": sphere,
        "filtration_dim2": filtration,
        "thresholded_o3": sparse,
        "breakdown": {
            "kernels": kernels,
            "host_reduce_ms": statistics.mean(s["ms_host_reduce"] for s in st),
            "host_kruskal_ms": statistics.mean(s["ms_host_h0"] for s in st),
            "columns": s0["columns"][1], "cleared": s0["cleared"][1],
            "apparent": s0["apparent"][1], "leftover": s0["leftover"][1],
            "free_pivot": s0["free_pivot"][1], "additions": s0["additions"][1],
            "scanned": s0["scanned"][1], "intervals_h1": s0["intervals"][1],
            "sweep_levels": s0["sweep_levels"][1], "sweep_pivots": s0["sweep_pivots"][1],
            "sweep_idle_tests": s0["sweep_idle"][1],
            "sweep_walks_ms": statistics.mean(s["ms_sweep_walks"] for s in st),
            "apparent_pass_simplices_per_s": s0["columns"][1] / (stage_ms[4] / 1000.0)
            if stage_ms[4] > 0 else None,
        },
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
