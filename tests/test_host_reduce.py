"""The library's host reduction (csrc/host.cpp) on the CPU, against the oracle.

tests/host_reduce_harness.cpp prepares what the GPU stages would hand over
(sorted edges, Kruskal clearing, apparent pairs by definition, leftovers with
their unreduced pivots, neighbour rows) and runs the dimension-1 submatrix
reduction; its H1 intervals must be the oracle's, bit for bit. The cases make
the reduction walk long enough to sweep diameter levels (the long-lived H1
classes of tori), with and without a threshold below the enclosing radius,
with many equal distances, with the levels taken from the sorted edges handed
over or from the reduction's own sort of the edges, and with apparent pivots
looked up or tested again.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_07989_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2003_07989_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def _build(tmp_path_factory, name, extra):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("hr") / name)
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", *extra, "-I", CSRC, "-I", inc,
           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "host_reduce_harness.cpp"),
           os.path.join(CSRC, "host.cpp"), "-o", exe, "-lpthread"]
    subprocess.run(cmd, check=True)
    return exe


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    return _build(tmp_path_factory, "host_reduce_harness", [])


@pytest.fixture(scope="module")
def harness_wide(tmp_path_factory):
    # the 128-bit heap keys that inputs of more than 2953 points take
    return _build(tmp_path_factory, "host_reduce_harness_wide", ["-DRPP_WIDE_KEYS_ONLY"])


def _run_full(exe, D, t, threads, flags, tmp):
    """(sorted H1 intervals, levels swept, additions) of one harness run."""
    D = np.ascontiguousarray(D, dtype=np.float32)
    dpath, opath = str(tmp / "D.f32"), str(tmp / "out.f32")
    D.tofile(dpath)
    r = subprocess.run([exe, dpath, str(len(D)), repr(float(t)), str(threads), str(flags), opath],
                       capture_output=True, text=True, check=True)
    iv = np.fromfile(opath, dtype=np.float32).reshape(-1, 2)
    iv = iv[np.lexsort((iv[:, 1], iv[:, 0]))]
    levels = int(r.stdout.split("levels ")[1].split()[0])
    additions = int(r.stdout.split("additions ")[1].split()[0])
    return iv, levels, additions


def _run(exe, D, t, threads, flags, tmp):
    D = np.ascontiguousarray(D, dtype=np.float32)
    dpath, opath = str(tmp / "D.f32"), str(tmp / "out.f32")
    D.tofile(dpath)
    r = subprocess.run([exe, dpath, str(len(D)), repr(float(t)), str(threads), str(flags), opath],
                       capture_output=True, text=True, check=True)
    iv = np.fromfile(opath, dtype=np.float32).reshape(-1, 2)
    iv = iv[np.lexsort((iv[:, 1], iv[:, 0]))]
    levels = int(r.stdout.split("levels ")[1].split()[0])
    return iv, levels


def _quantized(D, scale):
    Dq = (np.round(D.astype(np.float64) * scale) / scale).astype(np.float32)
    np.fill_diagonal(Dq, 0.0)
    return Dq


CASES = {
    "torus500": lambda: (O.distance_matrix(I.noisy_torus(500, seed=1)), math.inf),
    "torus420_t": lambda: (O.distance_matrix(I.noisy_torus(420, seed=2)), 0.8),
    "torus450_ties": lambda: (_quantized(O.distance_matrix(I.noisy_torus(450, seed=5)), 16.0),
                              math.inf),
    "cube300": lambda: (O.distance_matrix(I.uniform_cube(300, 3, seed=3)), math.inf),
    "circle400_q": lambda: (O.distance_matrix(I.circle_cloud(400, 1.0, 0.05, 3, 7)), None),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("flags", [0, 3])
def test_host_reduction_equals_oracle(harness, tmp_path, name, flags):
    D, t = CASES[name]()
    if t is None:  # the serving workload's 0.6 nearest-rank quantile threshold
        t = O.distance_quantile(D, 0.6)
    got, levels = _run(harness, D, t, 4, flags, tmp_path)
    ref = O.barcodes(D, 1, t, O.MODE_COHOM_CLEAR).barcode(1)
    assert got.shape == ref.shape and np.array_equal(got, ref), name
    if name in ("torus500", "torus450_ties"):
        assert levels > 0, "the long walks should sweep"


@pytest.mark.parametrize("name", ["torus500", "torus450_ties", "circle400_q"])
def test_host_reduction_wide_keys_equal_oracle(harness_wide, tmp_path, name):
    D, t = CASES[name]()
    if t is None:
        t = O.distance_quantile(D, 0.6)
    for flags in (0, 3):
        got, _ = _run(harness_wide, D, t, 4, flags, tmp_path)
        ref = O.barcodes(D, 1, t, O.MODE_COHOM_CLEAR).barcode(1)
        assert got.shape == ref.shape and np.array_equal(got, ref), (name, flags)


def test_host_reduction_threads_agree(harness, tmp_path):
    D = O.distance_matrix(I.noisy_torus(360, seed=9))
    a, _ = _run(harness, D, math.inf, 1, 0, tmp_path)
    b, _ = _run(harness, D, math.inf, 8, 1, tmp_path)
    assert np.array_equal(a, b)


PARALLEL_CASES = {
    # random edge orders and integer ties: many leftover columns whose walks
    # meet one another's pivots
    "perm160": lambda: (I.permutation_distances(160, seed=4), math.inf),
    "int140": lambda: (I.integer_distances(140, levels=6, seed=2), math.inf),
    "torus450_ties": CASES["torus450_ties"],
}


@pytest.mark.parametrize("name", sorted(PARALLEL_CASES))
def test_host_reduction_parallel_columns_equal_oracle(harness, harness_wide, tmp_path, name):
    """Leftover columns reduced concurrently (each waiting only for earlier
    columns that may still end at its pivot) give the oracle's barcode on
    every run, with 64- and 128-bit keys."""
    D, t = PARALLEL_CASES[name]()
    ref = O.barcodes(D, 1, t, O.MODE_COHOM_CLEAR).barcode(1)
    # flags 1: the edges are sorted by the reduction itself, a bucket at a
    # time, by whichever walk reaches it first
    for exe, threads, flags in ((harness, 8, 0), (harness, 3, 1), (harness_wide, 8, 1),
                                (harness, 8, 1)):
        got, _ = _run(exe, D, t, threads, flags, tmp_path)
        assert got.shape == ref.shape and np.array_equal(got, ref), (name, threads, flags)


@pytest.mark.parametrize("index", [29, 136, 3, 52])
def test_host_sorted_levels_add_what_the_sorted_array_adds(harness, tmp_path, index):
    """Serving clouds (circles whose H1 class outlives the 0.6-quantile
    threshold sweep long walks): with the reduction sorting the edges itself,
    a bucket at a time as its sweeps reach them, it makes exactly the
    additions it makes over a sorted edge array handed over, and the barcode
    is the oracle's. Clouds 29 and 136 have buckets of one or two edges that
    the sweep's look-ahead crosses."""
    r = I.serving_requests(4096, seed=0)[index]
    D = O.distance_matrix(r.points)
    t = O.distance_quantile(D, r.threshold_quantile)
    ref = O.barcodes(D, 1, t, O.MODE_COHOM_CLEAR).barcode(1)
    given, lv0, add0 = _run_full(harness, D, t, 1, 0, tmp_path)
    own, lv1, add1 = _run_full(harness, D, t, 1, 1, tmp_path)
    assert np.array_equal(given, ref) and np.array_equal(own, ref)
    assert (lv1, add1) == (lv0, add0)


@pytest.fixture(scope="module")
def harness_sanitized(tmp_path_factory):
    # AddressSanitizer and UndefinedBehaviorSanitizer, every report fatal
    flags = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined"]
    try:
        return _build(tmp_path_factory, "host_reduce_harness_asan", flags)
    except subprocess.CalledProcessError:
        pytest.skip("the compiler cannot build with the sanitizers here")


@pytest.mark.parametrize("name,flags,threads", [("perm160", 1, 4), ("circle400_q", 3, 4),
                                                ("torus450_ties", 1, 1)])
def test_host_reduction_under_sanitizers(harness_sanitized, tmp_path, name, flags, threads):
    """No out-of-bounds access, use after free or undefined behaviour in the
    host reduction (concurrent columns, host-sorted level buckets, apparent
    pivots tested again), and still the oracle's barcode."""
    D, t = {**CASES, **PARALLEL_CASES}[name]()
    if t is None:
        t = O.distance_quantile(D, 0.6)
    got, _ = _run(harness_sanitized, D, t, threads, flags, tmp_path)
    ref = O.barcodes(D, 1, t, O.MODE_COHOM_CLEAR).barcode(1)
    assert np.array_equal(got, ref), name
