"""Seeded synthetic inputs shared by the CUDA path's harness and the oracle's tests.

This module draws random numbers and shapes point clouds. It holds none of the
barcode method's arithmetic: no distances, no diameters, no filtration order.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014; the
finaliser constants are Stafford's "Mix13"). Output ``k`` (k = 0, 1, ...) of
stream ``s`` is ``mix(s + (k + 1) * 0x9E3779B97F4A7C15)``. A double in [0, 1)
takes the top 53 bits. Gaussians use the Box-Muller transform. Everything is
computed in float64 and rounded to float32 once at the end, so the same seed
gives the same bytes on every machine.

Workloads (sizes and shapes of the paper's experiments, Sec. "Experiments"):
  * ``uniform_cube``     : n points uniform in [0,1]^dim
  * ``noisy_torus``      : points on a 2-torus in R^3 plus Gaussian noise
  * ``sphere_s3``        : points uniform on S^3 in R^4 (stand-in for the paper's
                           sphere_3_192 dataset, which is not shipped here)
  * ``orthogonal3``      : random matrices of O(3) as points of R^9 (stand-in for
                           the paper's sparse o3 dataset)
  * ``noisy_circles``    : batches of noisy planar circles of random radius
  * ``serving_requests`` : a Poisson stream of clouds of uneven size drawn from a
                           mixture of noisy circles, noisy 2-spheres and blobs
  * ``integer_distances``: symmetric matrices with few distinct integer values
                           (tie-heavy inputs)
  * ``permutation_distances``: a uniformly random permutation of 1..C(n,2) on the
                           upper triangle (the random-distance experiment,
                           Sec. "Experiments on the Apparent Pairs Rate")
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, tag: int) -> int:
    """Derive an independent stream id from a user seed and a purpose tag."""
    with np.errstate(over="ignore"):
        z = np.array([(seed * 0x2545F4914F6CDD1D + tag * 0x9E3779B97F4A7C15) & _MASK64],
                     dtype=np.uint64)
        return int(_mix(z)[0])


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of SplitMix64 stream ``seed`` (uint64)."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + k * _GOLDEN
        return _mix(z)


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """float64 uniform in [0, 1) from the top 53 bits of each output."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """float64 standard normals by Box-Muller on consecutive output pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]              # (0, 1]: log is finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m, dtype=np.float64)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


def uniform_int(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), by scaling the 53-bit double."""
    u = uniform01(seed, count)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


# ---------------------------------------------------------------------------
# point clouds


def uniform_cube(n: int, dim: int = 3, seed: int = 0) -> np.ndarray:
    """n points uniform in [0,1]^dim, float32, shape (n, dim)."""
    u = uniform01(stream_seed(seed, 1), n * dim).reshape(n, dim)
    return u.astype(np.float32)


def noisy_torus(n: int = 2000, R: float = 1.0, r: float = 0.4, sigma: float = 0.02,
                seed: int = 0) -> np.ndarray:
    """n points on the torus ((R + r cos v) cos u, (R + r cos v) sin u, r sin v)
    with u, v uniform in [0, 2 pi), plus N(0, sigma^2) noise per coordinate."""
    uv = uniform01(stream_seed(seed, 2), 2 * n).reshape(n, 2) * (2.0 * math.pi)
    u, v = uv[:, 0], uv[:, 1]
    x = np.stack([(R + r * np.cos(v)) * np.cos(u),
                  (R + r * np.cos(v)) * np.sin(u),
                  r * np.sin(v)], axis=1)
    x = x + sigma * normal(stream_seed(seed, 3), 3 * n).reshape(n, 3)
    return x.astype(np.float32)


def sphere_s3(n: int = 192, seed: int = 0) -> np.ndarray:
    """n points uniform on the unit sphere S^3 in R^4: normalised Gaussian 4-vectors."""
    g = normal(stream_seed(seed, 4), 4 * n).reshape(n, 4)
    g = g / np.linalg.norm(g, axis=1, keepdims=True)
    return g.astype(np.float32)


def orthogonal3(n: int = 4096, seed: int = 0) -> np.ndarray:
    """n random 3 x 3 rotation-or-reflection matrices as points of R^9 (row-major
    entries), Haar-distributed on O(3): Gram-Schmidt of a Gaussian 3 x 3 matrix
    (the QR factor with a positive diagonal). A synthetic stand-in for the
    paper's sparse o3 workload (4096 points, evaluated below a threshold)."""
    g = normal(stream_seed(seed, 11), 9 * n).reshape(n, 3, 3)
    q = np.empty_like(g)
    for i in range(3):  # columns, classical Gram-Schmidt in float64
        c = g[:, :, i].copy()
        for j in range(i):
            c -= np.sum(q[:, :, j] * g[:, :, i], axis=1, keepdims=True) * q[:, :, j]
        q[:, :, i] = c / np.linalg.norm(c, axis=1, keepdims=True)
    return q.reshape(n, 9).astype(np.float32)


def circle_cloud(n: int, radius: float, sigma: float, dim: int, seed: int) -> np.ndarray:
    """A noisy circle of the given radius in the first two coordinates of R^dim."""
    ang = uniform01(stream_seed(seed, 5), n) * (2.0 * math.pi)
    x = np.zeros((n, dim), dtype=np.float64)
    x[:, 0] = radius * np.cos(ang)
    x[:, 1] = radius * np.sin(ang)
    x = x + sigma * normal(stream_seed(seed, 6), n * dim).reshape(n, dim)
    return x.astype(np.float32)


def sphere2_cloud(n: int, radius: float, sigma: float, dim: int, seed: int) -> np.ndarray:
    """A noisy 2-sphere of the given radius in the first three coordinates of R^dim."""
    assert dim >= 3
    g = normal(stream_seed(seed, 7), 3 * n).reshape(n, 3)
    g = g / np.linalg.norm(g, axis=1, keepdims=True)
    x = np.zeros((n, dim), dtype=np.float64)
    x[:, :3] = radius * g
    x = x + sigma * normal(stream_seed(seed, 8), n * dim).reshape(n, dim)
    return x.astype(np.float32)


def blob_cloud(n: int, dim: int, seed: int) -> np.ndarray:
    """A standard Gaussian blob N(0, I) in R^dim."""
    return normal(stream_seed(seed, 9), n * dim).reshape(n, dim).astype(np.float32)


def noisy_circles(batch: int = 256, n: int = 128, sigma: float = 0.05,
                  seed: int = 0) -> np.ndarray:
    """``batch`` planar clouds of ``n`` points each, shape (batch, n, 2): radius
    uniform in [0.5, 2], angle uniform in [0, 2 pi), N(0, sigma^2) noise."""
    radii = 0.5 + 1.5 * uniform01(stream_seed(seed, 10), batch)
    out = np.empty((batch, n, 2), dtype=np.float32)
    for b in range(batch):
        out[b] = circle_cloud(n, float(radii[b]), sigma, 2, stream_seed(seed, 1000 + b))
    return out


@dataclass
class Request:
    """One serving request: a point cloud plus its arrival time (seconds)."""
    index: int
    points: np.ndarray         # (n, dim) float32
    kind: str                  # "circle" | "sphere" | "blob"
    arrival_s: float
    threshold_quantile: float  # threshold = this nearest-rank quantile of distances


def serving_requests(count: int = 4096, rate_per_s: float | None = None, seed: int = 0,
                     n_range=(32, 512), dim_range=(2, 8),
                     quantile: float = 0.6) -> list[Request]:
    """A seeded stream of clouds of uneven size.

    n uniform in ``n_range``, ambient dim uniform in ``dim_range``; the shape is a
    noisy circle, a noisy 2-sphere (redrawn when dim == 2) or a Gaussian blob with
    probability 1/3 each. Circle/sphere radius uniform in [0.5, 2], noise
    N(0, 0.05^2) on every coordinate. Arrivals form a Poisson process of the given
    rate (exponential gaps); ``rate_per_s=None`` puts every arrival at t = 0.
    """
    reqs = []
    ns = uniform_int(stream_seed(seed, 20), count, n_range[0], n_range[1])
    dims = uniform_int(stream_seed(seed, 21), count, dim_range[0], dim_range[1])
    kinds_u = uniform01(stream_seed(seed, 22), 4 * count)
    radii = 0.5 + 1.5 * uniform01(stream_seed(seed, 23), count)
    gaps = -np.log(1.0 - uniform01(stream_seed(seed, 24), count))
    t = 0.0
    for i in range(count):
        n, dim = int(ns[i]), int(dims[i])
        # draw the shape; a 2-sphere needs three coordinates, so redraw if dim == 2
        kind = None
        for j in range(4):
            k = int(kinds_u[4 * i + j] * 3.0)
            kind = ("circle", "sphere", "blob")[min(k, 2)]
            if not (kind == "sphere" and dim == 2):
                break
        if kind == "sphere" and dim == 2:
            kind = "circle"
        s = stream_seed(seed, 100000 + i)
        if kind == "circle":
            pts = circle_cloud(n, float(radii[i]), 0.05, dim, s)
        elif kind == "sphere":
            pts = sphere2_cloud(n, float(radii[i]), 0.05, dim, s)
        else:
            pts = blob_cloud(n, dim, s)
        if rate_per_s is not None:
            t += float(gaps[i]) / rate_per_s
        reqs.append(Request(i, pts, kind, t if rate_per_s is not None else 0.0, quantile))
    return reqs


# ---------------------------------------------------------------------------
# distance matrices given directly


def integer_distances(n: int, levels: int = 5, seed: int = 0) -> np.ndarray:
    """Symmetric float32 n x n matrix, zero diagonal, off-diagonal entries drawn
    uniformly from {1, ..., levels}: many exact ties."""
    m = n * (n - 1) // 2
    vals = uniform_int(stream_seed(seed, 30), m, 1, levels).astype(np.float32)
    D = np.zeros((n, n), dtype=np.float32)
    iu = np.triu_indices(n, 1)
    D[iu] = vals
    D.T[iu] = vals
    return D


def permutation_distances(n: int, seed: int = 0) -> np.ndarray:
    """Upper triangle filled with a uniformly random permutation of 1..C(n,2)
    (the ranks of one uniform draw per entry), as float32; symmetric, zero
    diagonal. Exact in float32 while C(n,2) <= 2^24."""
    m = n * (n - 1) // 2
    u = uniform01(stream_seed(seed, 31), m)
    perm = np.empty(m, dtype=np.int64)
    perm[np.argsort(u, kind="stable")] = np.arange(1, m + 1, dtype=np.int64)
    D = np.zeros((n, n), dtype=np.float32)
    iu = np.triu_indices(n, 1)
    D[iu] = perm.astype(np.float32)
    D.T[iu] = perm.astype(np.float32)
    return D


def rank_distances(n: int, seed: int = 0) -> np.ndarray:
    """A uniformly random total order of the C(n,2) edges, as distinct float32
    values at any n: the edge of rank r (1-based) gets the float whose bit
    pattern is that of 1.0 plus r, so values increase with rank and no two are
    equal (integers would tie in float32 beyond 2^24). Symmetric, zero
    diagonal. The ranks are those of permutation_distances."""
    m = n * (n - 1) // 2
    u = uniform01(stream_seed(seed, 31), m)
    rank = np.empty(m, dtype=np.int64)
    rank[np.argsort(u, kind="stable")] = np.arange(1, m + 1, dtype=np.int64)
    vals = (np.int64(0x3F800000) + rank).astype(np.uint32).view(np.float32)
    D = np.zeros((n, n), dtype=np.float32)
    iu = np.triu_indices(n, 1)
    D[iu] = vals
    D.T[iu] = vals
    return D


def decreasing_lex_distances(n: int) -> np.ndarray:
    """Edge (a, b), a > b, gets C(n,2) - (its rank in lexicographic order of the
    decreasing vertex pair); the construction of Sec. "The Upper Bound Under
    Differing Diameters". The rank here is counted by enumeration."""
    m = n * (n - 1) // 2
    D = np.zeros((n, n), dtype=np.float32)
    rank = 0
    for a in range(1, n):          # decreasing pairs (a, b) in lexicographic order
        for b in range(a):
            D[a, b] = D[b, a] = float(m - rank)
            rank += 1
    return D
