"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formulas. Each pin comes from outside
the oracle: printed values of the paper (tests/golden/), closed forms, ranks
computed by independent Gaussian elimination, a library minimum spanning tree,
the duality between the homology and cohomology reductions, and the paper's
lemmas and theorems about apparent pairs.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_07989_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODES = (O.MODE_HOM, O.MODE_COHOM, O.MODE_COHOM_CLEAR)


def _small_inputs():
    """Tiny seeded inputs: random points in several dimensions and tie-heavy
    integer matrices (values in {1..5})."""
    out = []
    for seed in range(6):
        out.append(("cube", O.distance_matrix(I.uniform_cube(9, 3, seed))))
    for seed in range(6):
        out.append(("ties", I.integer_distances(9, 5, seed)))
    out.append(("ties2", I.integer_distances(10, 2, 7)))
    return out


# ---------------------------------------------------------------------------
# independent helpers (rank over Z/2 by Gaussian elimination)


def _rank_gf2(M: np.ndarray) -> int:
    M = M.copy().astype(bool)
    rows, cols = M.shape
    r = 0
    for c in range(cols):
        piv = None
        for i in range(r, rows):
            if M[i, c]:
                piv = i
                break
        if piv is None:
            continue
        M[[r, piv]] = M[[piv, r]]
        for i in range(rows):
            if i != r and M[i, c]:
                M[i] ^= M[r]
        r += 1
        if r == rows:
            break
    return r


def _complex(D, s, top):
    """Simplices (as sorted tuples) of dims 0..top with diam <= s."""
    n = D.shape[0]
    cx = []
    for q in range(top + 1):
        cq = []
        for t in itertools.combinations(range(n), q + 1):
            d = 0.0
            for a, b in itertools.combinations(t, 2):
                d = max(d, float(D[a, b]))
            if d <= s:
                cq.append(t)
        cx.append(cq)
    return cx


def _boundary_rank(cx, q):
    """rank of the boundary map from dim q to dim q-1."""
    if q == 0 or not cx[q] or not cx[q - 1]:
        return 0
    index = {t: i for i, t in enumerate(cx[q - 1])}
    M = np.zeros((len(cx[q - 1]), len(cx[q])), dtype=bool)
    for j, t in enumerate(cx[q]):
        for r in range(len(t)):
            M[index[t[:r] + t[r + 1:]], j] = True
    return _rank_gf2(M)


def _bars_alive(P, q, s):
    return int(np.sum((P.dim == q) & (P.birth <= s) & (s < P.death)))


def _pairing(P):
    return sorted((int(d), tuple(bv), tuple(dv)) for d, bv, dv in zip(P.dim, P.bverts, P.dverts))


# ---------------------------------------------------------------------------
# distances


def test_distance_matrix_within_float32_rounding_of_exact():
    """The float32 distance is within a few ulps of the exact Euclidean distance
    of the float32 coordinates (computed in float64), symmetric, zero diagonal."""
    X = I.noisy_torus(300, seed=3)
    D = O.distance_matrix(X)
    X64 = X.astype(np.float64)
    E = np.sqrt(((X64[:, None, :] - X64[None, :, :]) ** 2).sum(-1))
    assert np.array_equal(D, D.T)
    assert np.all(np.diag(D) == 0)
    off = ~np.eye(300, dtype=bool)
    rel = np.abs(D[off].astype(np.float64) - E[off]) / E[off]
    assert rel.max() < 4 * 2.0 ** -24 * 3  # 3 adds + square root, each half an ulp


def _f32_round(x):
    """x (an exact Fraction) rounded to the nearest float32, ties to even,
    as an exact Fraction (normal range only; zero stays zero)."""
    from fractions import Fraction
    if x == 0:
        return Fraction(0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    assert -126 <= e <= 127, "outside the float32 normal range"
    ulp = Fraction(2) ** (e - 23)
    q, r = divmod(a, ulp)  # q integer, 0 <= r < ulp
    if r * 2 > ulp or (r * 2 == ulp and q % 2 == 1):
        q += 1
    return sign * q * ulp


def _f32_sqrt(s):
    """The float32 nearest to sqrt(s) for an exact Fraction s >= 0, chosen by
    comparing squares exactly (no floating-point square root decides it)."""
    from fractions import Fraction
    import math
    if s == 0:
        return Fraction(0)
    guess = _f32_round(Fraction(math.sqrt(float(s))))
    e = guess.numerator.bit_length() - guess.denominator.bit_length()
    if Fraction(2) ** e > guess:
        e -= 1
    ulp = Fraction(2) ** (e - 23)
    best = None
    for c in (guess - 2 * ulp, guess - ulp, guess, guess + ulp, guess + 2 * ulp):
        c = _f32_round(c)
        if best is None or abs(c * c - s) < abs(best * best - s):
            best = c
    return best


def _emulated_distance(xi, xj, order, fused=False):
    """The float32 distance with one rounding after every operation: per
    coordinate in `order`, d = x_i - x_j, sq = d * d, s = s + sq; then sqrt.
    fused: s + d * d rounded once (a fused multiply-add)."""
    from fractions import Fraction
    s = Fraction(0)
    for k in order:
        d = _f32_round(Fraction(float(xi[k])) - Fraction(float(xj[k])))
        if fused:
            s = _f32_round(s + d * d)
        else:
            s = _f32_round(s + _f32_round(d * d))
    return _f32_sqrt(s)


def test_distance_matrix_operation_order_exact():
    """The oracle's float32 distances equal, bit for bit, an exact-arithmetic
    emulation of the stated operation order (coordinates in increasing
    index, a rounding after each subtraction, square and addition, no fused
    multiply-add, then a correctly rounded square root). The fixture is
    chosen so that summing the coordinates in reverse order, or fusing each
    square into its addition, changes some distances: the pin tells the
    stated order from other equally accurate ones."""
    from fractions import Fraction
    rng = np.random.default_rng(17)
    n, dim = 10, 16
    X = (rng.standard_normal((n, dim)) * np.float32(3.0)).astype(np.float32)
    D = O.distance_matrix(X)
    fwd, rev = list(range(dim)), list(range(dim - 1, -1, -1))
    reordered = fused = 0
    for i in range(n):
        for j in range(i + 1, n):
            want = _emulated_distance(X[i], X[j], fwd)
            assert Fraction(float(D[i, j])) == want, (i, j)
            assert D[j, i] == D[i, j]
            reordered += _emulated_distance(X[i], X[j], rev) != want
            fused += _emulated_distance(X[i], X[j], fwd, fused=True) != want
    assert reordered > 0, "the fixture does not discriminate the summation order"
    assert fused > 0, "the fixture does not discriminate a fused multiply-add"


def test_enclosing_radius_closed_forms():
    """Closed forms, independent of any row max/min code: n collinear points
    at 0, 1, ..., n-1 have R = ceil((n-1)/2) (every point's farthest point is
    an end of the line; the middle points minimise that); a regular 2k-gon on
    the unit circle has R = its diameter 2 (each vertex's antipode); a star
    of unit spokes has R = 1 (its centre's row) although every other row's
    maximum is 2. A max taken for a min, or a row skipped, gives another
    value in each case."""
    for n in (2, 3, 7, 10, 31):
        X = np.zeros((n, 2), np.float32)
        X[:, 0] = np.arange(n, dtype=np.float32)
        assert O.enclosing_radius(O.distance_matrix(X)) == float((n - 1 + 1) // 2)
    k = 8
    ang = np.arange(2 * k) * (np.pi / k)
    X = np.stack([np.cos(ang), np.sin(ang)], 1).astype(np.float32)
    D = O.distance_matrix(X)
    R = O.enclosing_radius(D)
    assert abs(R - 2.0) < 1e-6
    assert R == float(min(D[i, (i + k) % (2 * k)] for i in range(2 * k)))
    # a star: the centre is within 1 of every other point, and every other
    # point has a point 2 away, so R = 1 exactly (the centre's row)
    X = np.zeros((9, 2), np.float32)
    X[1:, 0] = [1, -1, 0, 0, 1, -1, 0, 0]
    X[1:, 1] = [0, 0, 1, -1, 0, 0, 1, -1]
    X[5:] *= -1
    assert O.enclosing_radius(O.distance_matrix(X)) == 1.0


def test_distance_quantile_closed_form():
    """On a matrix whose C(n,2) edge values are 1.0 + r for the ranks r =
    1..m (distinct floats in rank order), the nearest-rank q-quantile is the
    edge of rank ceil(q m), whose value is known without sorting."""
    n = 23
    D = I.rank_distances(n, seed=4)
    m = n * (n - 1) // 2
    for q in (0.01, 0.25, 0.5, 0.6, 0.999, 1.0):
        r = math.ceil(q * m)
        want = np.array([0x3F800000 + r], dtype=np.uint32).view(np.float32)[0]
        assert O.distance_quantile(D, q) == float(want), q


def test_enclosing_radius_and_quantile_definitions():
    X = I.uniform_cube(40, 3, 5)
    D = O.distance_matrix(X)
    R = O.enclosing_radius(D)
    assert R == float(np.min(np.max(D, axis=1)))
    tri = np.sort(D[np.triu_indices(40, 1)])
    m = len(tri)
    for q in (0.1, 0.6, 1.0):
        assert O.distance_quantile(D, q) == float(tri[math.ceil(q * m) - 1])


# ---------------------------------------------------------------------------
# printed values of the paper


def test_square_barcode_from_figure():
    g = json.load(open(os.path.join(GOLDEN, "square.json")))
    X = np.array(g["points"], dtype=np.float32)
    D = O.distance_matrix(X)
    assert D[1, 0] == np.float32(g["edge_10_diameter"])
    sqrt2 = float(np.sqrt(np.float32(2.0)))
    for mode in MODES:
        P = O.barcodes(D, 1, math.inf, mode)
        h1 = P.barcode(1)
        assert h1.tolist() == [[1.0, sqrt2]]
        h0 = P.barcode(0)
        assert sorted(h0[np.isfinite(h0[:, 1]), 1].tolist()) == g["H0_finite_deaths"]
        assert int(np.sum(np.isinf(h0[:, 1]))) == g["H0_essential"]


def test_all_pairs_column_matches_rank_identity():
    """The paper's 'all pairs' column equals sum_q C(n-1, q+1); the oracle's pair
    count on small full filtrations follows the same identity."""
    g = json.load(open(os.path.join(GOLDEN, "all_pairs_table.json")))
    for row in g["rows"]:
        n, p = row["n"], row["p"]
        assert sum(math.comb(n - 1, q + 1) for q in range(1, p + 1)) == row["all_pairs"]
    for name, D in _small_inputs():
        n = D.shape[0]
        for mode in MODES:
            P = O.barcodes(D, 2, math.inf, mode)
            for q in (0, 1, 2):
                finite = int(np.sum((P.dim == q) & np.isfinite(P.death)))
                assert finite == math.comb(n - 1, q + 1), (name, mode, q)
            assert int(np.sum(np.isinf(P.death))) == 1  # one component, nothing else


# ---------------------------------------------------------------------------
# closed forms


@pytest.mark.parametrize("n", [8, 10, 11, 13, 16, 20, 25])
def test_circle_closed_form(n):
    """Evenly spaced points on the unit circle: VR is a circle while the scale
    spans fewer than n/3 steps (Adamaszek-Adams), so one H1 bar
    [2 sin(pi/n), 2 sin(pi ceil(n/3)/n)) and every other H1 bar has length ~0."""
    if n % 3 == 0:
        pytest.skip("n divisible by 3 gives a wedge of 2-spheres at the death scale")
    ang = 2.0 * np.pi * np.arange(n) / n
    X = np.stack([np.cos(ang), np.sin(ang)], 1).astype(np.float32)
    D = O.distance_matrix(X)
    P = O.barcodes(D, 1, math.inf, O.MODE_COHOM_CLEAR)
    h1 = P.barcode(1)
    long = h1[(h1[:, 1] - h1[:, 0]) > 1e-5]
    assert len(long) == 1
    b, d = 2 * math.sin(math.pi / n), 2 * math.sin(math.pi * math.ceil(n / 3) / n)
    assert abs(long[0, 0] - b) <= 1e-5 * b and abs(long[0, 1] - d) <= 1e-5 * d


# ---------------------------------------------------------------------------
# Betti numbers and the Euler identity at every scale


@pytest.mark.parametrize("idx", range(13))
def test_betti_numbers_at_every_scale(idx):
    name, D = _small_inputs()[idx]
    n = D.shape[0]
    vals = sorted(set(D[np.triu_indices(n, 1)].tolist()))
    scales = [0.0] + vals + [vals[-1] + 1.0]
    P = O.barcodes(D, 2, math.inf, O.MODE_HOM)
    for s in scales:
        cx = _complex(D, s, 3)
        ranks = [_boundary_rank(cx, q) for q in range(4)]
        for q in range(3):
            beta = len(cx[q]) - ranks[q] - ranks[q + 1]
            assert _bars_alive(P, q, s) == beta, (name, s, q)
        # Euler identity with the pair counts (zero-length pairs included)
        for k in range(3):
            lhs = sum((-1) ** q * _bars_alive(P, q, s) for q in range(k + 1))
            r_k = int(np.sum((P.dim == k) & (P.death <= s)))
            rhs = sum((-1) ** q * len(cx[q]) for q in range(k + 1)) - (-1) ** k * r_k
            assert lhs == rhs, (name, s, k)


def test_betti_with_threshold_below_enclosing_radius():
    """Essential classes above dimension 0 appear when t is small."""
    for seed in range(4):
        D = O.distance_matrix(I.uniform_cube(10, 2, 100 + seed))
        t = float(np.quantile(D[np.triu_indices(10, 1)], 0.3))
        t = float(D[np.triu_indices(10, 1)][np.argmin(np.abs(D[np.triu_indices(10, 1)] - t))])
        for mode in MODES:
            P = O.barcodes(D, 1, t, mode)
            cx = _complex(D, t, 2)
            ranks = [_boundary_rank(cx, q) for q in range(3)]
            for q in range(2):
                beta = len(cx[q]) - ranks[q] - ranks[q + 1]
                assert int(np.sum((P.dim == q) & np.isinf(P.death))) == beta


# ---------------------------------------------------------------------------
# the three reductions agree pair by pair; H0 equals Kruskal and a library MST


@pytest.mark.parametrize("idx", range(13))
def test_modes_give_identical_pairings(idx):
    name, D = _small_inputs()[idx]
    ref = _pairing(O.barcodes(D, 2, math.inf, O.MODE_HOM))
    for mode in (O.MODE_COHOM, O.MODE_COHOM_CLEAR):
        assert _pairing(O.barcodes(D, 2, math.inf, mode)) == ref, (name, mode)
    vals = np.unique(D[np.triu_indices(D.shape[0], 1)])
    t = float(vals[len(vals) // 2])
    ref_t = _pairing(O.barcodes(D, 2, t, O.MODE_HOM))
    for mode in (O.MODE_COHOM, O.MODE_COHOM_CLEAR):
        assert _pairing(O.barcodes(D, 2, t, mode)) == ref_t, (name, mode, t)


def test_h0_equals_kruskal_and_library_mst():
    from scipy.sparse.csgraph import minimum_spanning_tree
    for seed in range(5):
        D = O.distance_matrix(I.uniform_cube(30, 3, seed))
        K = O.kruskal(D)
        H = O.barcodes(D, 1, math.inf, O.MODE_HOM)
        h0 = H.dim == 0
        assert sorted(zip(H.bverts[h0, 0].tolist(), H.death[h0].tolist())) == \
            sorted(zip(K.bverts[:, 0].tolist(), K.death.tolist()))
        mst = minimum_spanning_tree(D.astype(np.float64)).toarray()
        lengths = np.sort(mst[mst > 0]).astype(np.float32)
        fin = np.sort(K.death[np.isfinite(K.death)])
        assert np.array_equal(fin, lengths)


def test_enclosing_radius_keeps_nonzero_intervals():
    """Proposition: thresholding at the enclosing radius does not change the
    nonzero persistence intervals of the full filtration."""
    for seed in range(4):
        D = O.distance_matrix(I.uniform_cube(14, 3, 50 + seed))
        R = O.enclosing_radius(D)
        a = O.barcodes(D, 2, math.inf, O.MODE_COHOM_CLEAR)
        b = O.barcodes(D, 2, R, O.MODE_COHOM_CLEAR)
        for q in range(3):
            assert np.array_equal(a.barcode(q), b.barcode(q))


# ---------------------------------------------------------------------------
# combinatorial number system and column order


def test_colex_rank_is_the_binomial_sum():
    """Brute-force colexicographic ranking of all (p+1)-subsets equals
    sum_i C(v_i, i+1) (the bijection of Sec. 'The Combinatorial Number System')."""
    for n in (6, 12, 20):
        for k in (1, 2, 3, 4):
            subs = [tuple(sorted(c, reverse=True)) for c in itertools.combinations(range(n), k)]
            subs.sort()  # lexicographic on the decreasing tuple
            for rank, s in enumerate(subs):
                asc = s[::-1]
                assert sum(math.comb(v, i + 1) for i, v in enumerate(asc)) == rank


def test_columns_in_coboundary_order():
    D = I.integer_distances(11, 3, 4)
    for p in (1, 2):
        diam, verts = O.columns(D, p)
        ref = []
        for c in itertools.combinations(range(11), p + 1):
            d = max(float(D[a, b]) for a, b in itertools.combinations(c, 2))
            ref.append((-d, tuple(sorted(c, reverse=True))))
        ref.sort()
        assert [(-float(a), tuple(v)) for a, v in zip(diam, verts.tolist())] == \
            [(a, b) for a, b in ref]


# ---------------------------------------------------------------------------
# apparent pairs


def _explicit_apparent(D, p, t=math.inf):
    """Apparent pairs read off an explicit coboundary matrix: entry (tau, sigma)
    that is the lowest nonzero of column sigma and has only zeros to its left in
    row tau (Sec. 'The Apparent Pairs Lemma'). Columns/rows in reverse
    filtration order, built with itertools and Python sorting."""
    n = D.shape[0]

    def diam(c):
        return max((float(D[a, b]) for a, b in itertools.combinations(c, 2)), default=0.0)

    def order_key(c):  # reverse filtration: decreasing diam, then increasing colex
        return (-diam(c), tuple(sorted(c, reverse=True)))

    cols = sorted([c for c in itertools.combinations(range(n), p + 1) if diam(c) <= t], key=order_key)
    rows = sorted([c for c in itertools.combinations(range(n), p + 2) if diam(c) <= t], key=order_key)
    ci = {c: i for i, c in enumerate(cols)}
    M = np.zeros((len(rows), len(cols)), dtype=bool)
    for r, tau in enumerate(rows):
        for k in range(p + 2):
            f = tau[:k] + tau[k + 1:]
            if f in ci:
                M[r, ci[f]] = True
    out = set()
    for j in range(len(cols)):
        nz = np.nonzero(M[:, j])[0]
        if len(nz) == 0:
            continue
        low = nz[-1]
        if not M[low, :j].any():
            out.add((tuple(sorted(cols[j], reverse=True)), tuple(sorted(rows[low], reverse=True))))
    return out


def _oracle_apparent_set(D, p, t=math.inf):
    s, tau = O.apparent_pairs(D, p, t)
    return {(tuple(a), tuple(b)) for a, b in zip(s.tolist(), tau.tolist())}


@pytest.mark.parametrize("idx", range(13))
def test_apparent_definition_equals_explicit_matrix_criterion(idx):
    name, D = _small_inputs()[idx]
    for p in (1, 2):
        assert _oracle_apparent_set(D, p) == _explicit_apparent(D, p), (name, p)
    vals = np.unique(D[np.triu_indices(D.shape[0], 1)])
    t = float(vals[len(vals) // 2])
    assert _oracle_apparent_set(D, 1, t) == _explicit_apparent(D, 1, t)


def test_apparent_pairs_are_zero_persistence_pairs():
    for name, D in _small_inputs():
        P = O.barcodes(D, 2, math.inf, O.MODE_HOM)
        pairs = {(tuple(b[b >= 0]), tuple(d[d >= 0])) for b, d in zip(P.bverts, P.dverts)}
        for p in (1, 2):
            for s, tau in _oracle_apparent_set(D, p):
                assert (s, tau) in pairs
                d = lambda c: max(float(D[a, b]) for a, b in itertools.combinations(c, 2))
                assert d(s) == d(tau)


def test_apparent_count_all_equal_diameters():
    """All diameters equal: exactly C(n-1, p+1) apparent (p, p+1) pairs (tightness
    of the upper bound, Theorem 'Equal Diameter Bound'; the 5-point figure shows
    C(4,2) = 6)."""
    for n in (5, 7, 9):
        D = np.ones((n, n), dtype=np.float32)
        np.fill_diagonal(D, 0)
        for p in (1, 2):
            assert len(_oracle_apparent_set(D, p)) == math.comb(n - 1, p + 1)


def test_apparent_count_decreasing_lex_assignment():
    """Distances decreasing along increasing lexicographic edge order reach the
    upper bound C(n-1, 2) in dimension 1 (Sec. 'The Upper Bound Under Differing
    Diameters'; recurrence T(n) = T(n-1) + n - 2, T(3) = 1)."""
    T = {3: 1}
    for n in range(4, 12):
        T[n] = T[n - 1] + n - 2
    for n in range(3, 12):
        D = I.decreasing_lex_distances(n)
        assert len(_oracle_apparent_set(D, 1)) == math.comb(n - 1, 2) == T[n]


def test_single_triangle_has_one_apparent_pair():
    """A single 2-simplex has exactly one (1, 2) apparent pair (lower-bound
    tightness example)."""
    for seed in range(5):
        D = O.distance_matrix(I.uniform_cube(3, 2, seed))
        assert len(_oracle_apparent_set(D, 1)) == 1
    D = np.array([[0, 3, 5], [3, 0, 4], [5, 4, 0]], dtype=np.float32)
    assert _oracle_apparent_set(D, 1) == {((2, 0), (2, 1, 0))}


def test_apparent_rate_bounds_full_filtration():
    """Upper bound (n-p-1)/n of the apparent rate (Theorem 'Equal Diameter Bound',
    which holds in general through the pair count); the 1/(p+2) lower bound is
    checked where the theorem's hypothesis holds (all diameters equal)."""
    for name, D in _small_inputs():
        n = D.shape[0]
        for p in (1, 2):
            k = len(_oracle_apparent_set(D, p))
            assert k <= math.comb(n - 1, p + 1)
    for n in (5, 8):
        D = np.ones((n, n), dtype=np.float32)
        np.fill_diagonal(D, 0)
        for p in (1, 2):
            assert len(_oracle_apparent_set(D, p)) >= math.comb(n, p + 1) / (p + 2)


def test_apparent_edges_are_not_mst_edges():
    """GMST lemma: the longest edge of an apparent simplex is a complementary
    edge, never a minimum-spanning-tree edge. The spanning tree is Kruskal's in
    the filtration order; 'longest' is the youngest edge in that order."""
    for seed in range(5):
        for D in (O.distance_matrix(I.uniform_cube(25, 3, seed)), I.integer_distances(16, 4, seed)):
            K = O.kruskal(D)
            mst = {tuple(v[:2]) for v in K.dverts[np.isfinite(K.death)].tolist()}
            for p in (1, 2):
                for s, _ in _oracle_apparent_set(D, p):
                    edges = [tuple(sorted(e, reverse=True)) for e in itertools.combinations(s, 2)]
                    youngest = max(edges, key=lambda e: (float(D[e[0], e[1]]), tuple(-x for x in e)))
                    assert youngest not in mst


def test_p1_sufficient_condition_without_equidistant_points():
    """Lemma 'Sufficient Condition for an Apparent Pair': with no two equal
    distances, an edge is apparent iff it has a cofacet of equal diameter."""
    for seed in range(3):
        D = I.permutation_distances(12, seed)
        app = {s for s, _ in _oracle_apparent_set(D, 1)}
        for a, b in itertools.combinations(range(12), 2):
            d = D[a, b]
            has = any(max(D[a, c], D[b, c]) <= d for c in range(12) if c not in (a, b))
            assert has == ((b, a) in app)


def test_cofacet_lexicographic_property():
    """Lemma 'Cofacet Lexicographic Property': if every p-simplex containing
    vertex n-1 is no longer than every other p-simplex, the oldest cofacet of a
    simplex without n-1 contains n-1 (and so the pair is apparent)."""
    rng = np.random.default_rng(0)
    for n in (6, 9):
        D = np.zeros((n, n), dtype=np.float32)
        for a, b in itertools.combinations(range(n), 2):
            v = 1.0 + rng.integers(0, 3) if b != n - 1 else 0.5
            D[a, b] = D[b, a] = v
        for c in itertools.combinations(range(n - 1), 2):
            tau = O.apparent_one(D, 1, c)
            assert tau is not None and tau[0] == n - 1


def test_torus300_golden_no_clearing_equals_clearing_mode():
    """The stored 300-point torus barcodes were computed by the coboundary
    reduction WITHOUT clearing (COHOM); the clearing mode, which starts from
    Kruskal's H0 and skips the cleared columns (Clearing Lemma), must give
    the same intervals on the same stored points."""
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "torus300_cohom.npz"))
    assert str(g["oracle_mode"]) == "COHOM"
    D = O.distance_matrix(g["points"])
    P = O.barcodes(D, 1, math.inf, O.MODE_COHOM_CLEAR)
    for q in (0, 1):
        assert np.array_equal(P.barcode(q), g[f"H{q}"]), q
