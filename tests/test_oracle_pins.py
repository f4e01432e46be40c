"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a
closed form, an invariant, exact arithmetic, a textbook routine written here
independently, brute-force enumeration, or the worked example the paper prints
(Sec. 4.4).  test_oracle_mutants.py plants mistakes in a copy of the oracle
and checks that these pins catch them.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------ helpers

def exact_d2(points, i, j):
    """Exact squared distance as a Fraction (float32 values are dyadic)."""
    return sum((Fraction(float(points[i, k])) - Fraction(float(points[j, k]))) ** 2
               for k in range(points.shape[1]))


def brute_force(points, maxdim, maxrad):
    """Enumerate every vertex subset directly (tiny n only).  Integer
    distances are exact Python integers; float distances are the oracle's
    step-1 values (pinned on their own by the rational-bound test), so this
    checks cap, ranking, enumeration, order and boundary."""
    n, d = points.shape
    is_float = points.dtype == np.float32
    d2 = {}
    for i, j in itertools.combinations(range(n), 2):
        d2[(i, j)] = oracle.pair_d2(points, i, j) if is_float else \
            sum((int(points[i, k]) - int(points[j, k])) ** 2 for k in range(d))
    r2 = maxrad * maxrad
    if is_float:
        kept = {e: v for e, v in d2.items() if v <= r2}
    else:
        lim = math.inf if math.isinf(r2) else math.floor(r2)
        kept = {e: v for e, v in d2.items() if v <= lim}
    values = sorted(set([0] + list(kept.values())))
    gidx = {v: g for g, v in enumerate(values)}
    eg = {e: gidx[v] for e, v in kept.items()}
    edges = sorted(kept, key=lambda e: (eg[e], e[0], e[1]))
    ordr = {e: t for t, e in enumerate(edges)}
    tris = []
    for a, b, c in itertools.combinations(range(n), 3):
        if (a, b) in kept and (a, c) in kept and (b, c) in kept:
            tris.append((max(eg[(a, b)], eg[(a, c)], eg[(b, c)]), a, b, c))
    tris.sort()
    return values, edges, [eg[e] for e in edges], ordr, tris


def check_against_brute(points, maxdim, maxrad):
    cx = oracle.vr_build(points, maxdim, maxrad)
    values, edges, grades, ordr, tris = brute_force(points, maxdim, maxrad)
    n = points.shape[0]
    assert cx.dims[0].count == n
    assert cx.dims[0].verts[:, 0].tolist() == list(range(n))
    assert cx.dims[0].grade.tolist() == [0] * n
    assert cx.grade_value.tolist() == [float(v) for v in values]
    if maxdim >= 1:
        d1 = cx.dims[1]
        assert [tuple(x) for x in d1.verts.tolist()] == edges
        assert d1.grade.tolist() == grades
        assert d1.colptr.tolist() == [2 * t for t in range(len(edges) + 1)]
        assert d1.rowidx.tolist() == [v for e in edges for v in e]
    if maxdim >= 2:
        d2 = cx.dims[2]
        assert [tuple(x) for x in d2.verts.tolist()] == [t[1:] for t in tris]
        assert d2.grade.tolist() == [t[0] for t in tris]
        assert d2.colptr.tolist() == [3 * t for t in range(len(tris) + 1)]
        rows = []
        for _, a, b, c in tris:
            rows += sorted([ordr[(b, c)], ordr[(a, c)], ordr[(a, b)]])
        assert d2.rowidx.tolist() == rows
    return cx


def kruskal_weights(points):
    """Weights (squared distance) of a minimum spanning tree, by Kruskal with
    union-find; distances from numpy (integers exactly; floats by a
    left-to-right double sum of elementwise IEEE operations)."""
    n, d = points.shape
    if points.dtype == np.float32:
        q = points.astype(np.float64)
        acc = np.zeros((n, n))
    else:
        q = points.astype(np.int64)
        acc = np.zeros((n, n), dtype=np.int64)
    for k in range(d):
        t = q[:, None, k] - q[None, :, k]
        acc = acc + t * t
    iu = np.triu_indices(n, 1)
    order = np.argsort(acc[iu], kind="stable")
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    out = []
    for t in order:
        i, j = int(iu[0][t]), int(iu[1][t])
        ri, rj = find(i), find(j)
        if ri != rj:
            parent[ri] = rj
            out.append(float(acc[i, j]))
    return sorted(out)


# ------------------------------------------------------------- the pins

def test_sortperm_worked_example():
    """Sec. 4.4: sortperm([7,3,8,4,2]) = [5,2,4,1,3]; ranking is the inverse
    of that permutation.  With 0 reserved as grade 0 the ranks are 1..5."""
    lines = [l.split() for l in open(os.path.join(HERE, "golden", "sortperm_sec4_4.txt"))
             if l.strip() and not l.startswith("#")]
    v = [float(x) for x in lines[0][1:]]
    sp = [int(x) for x in lines[1][1:]]
    ranks = oracle.dense_rank(v)
    assert (np.argsort(ranks, kind="stable") + 1).tolist() == sp
    assert sorted(ranks.tolist()) == [1, 2, 3, 4, 5]


def test_dense_rank_ties_and_zero():
    """Equal values share a rank; 0 is always rank 0."""
    assert oracle.dense_rank([5, 0, 5, 2, 9, 2]).tolist() == [2, 0, 2, 1, 3, 1]
    assert oracle.dense_rank([]).tolist() == []


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 20])
@pytest.mark.parametrize("dtype", [np.int8, np.int32, np.float32])
def test_counts_without_cap(n, dtype):
    """No cap: the number of k-simplices is C(n, k+1)."""
    pts = synth.random_cloud(n, 3, dtype, seed=100 + n)
    cx = oracle.vr_build(pts, 2)
    for k in range(3):
        assert cx.dims[k].count == math.comb(n, k + 1)
        if cx.dims[k].count and k:
            assert np.all(np.diff(cx.dims[k].verts, axis=1) > 0)


def test_config1_counts():
    c = synth.config1()
    cx = oracle.vr_build(c.points, c.maxdim, c.maxrad)
    assert [cx.dims[k].count for k in range(3)] == [64, 2016, 41664]


def test_hollow_tetrahedron():
    """Regular tetrahedron with even-parity +-1 coordinates: all six edges have
    d^2 = 8 (grade 1), the 2-skeleton is a 2-sphere: bars H0 3x[0,1) + [0,inf),
    H1 none, H2 [1,inf); Betti (1,0,1) at grade 1."""
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], np.int32)
    cx = oracle.vr_build(tet, 2, keep_handle=True)
    assert cx.grade_value.tolist() == [0.0, 8.0]
    assert sorted(map(tuple, cx.barcode(0).tolist())) == [(0, -1), (0, 1), (0, 1), (0, 1)]
    assert cx.barcode(1).tolist() == []
    assert cx.barcode(2).tolist() == [[1, -1]]
    assert oracle.betti(cx, 1) == [1, 0, 1]


def test_square():
    """Unit square on the integer grid: sides d^2=1 (grade 1), diagonals d^2=2
    (grade 2).  H1 = [1,2); at grade 2 the 2-skeleton is a hollow tetrahedron,
    so H2 = [2, inf)."""
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.int8)
    cx = oracle.vr_build(sq, 2, keep_handle=True)
    assert cx.grade_value.tolist() == [0.0, 1.0, 2.0]
    assert sorted(map(tuple, cx.barcode(0).tolist())) == [(0, -1), (0, 1), (0, 1), (0, 1)]
    assert cx.barcode(1).tolist() == [[1, 2]]
    assert cx.barcode(2).tolist() == [[2, -1]]


@pytest.mark.parametrize("n", [5, 6, 7, 8, 9, 10, 12, 13])
def test_regular_ngon(n):
    """n evenly spaced points on the unit circle: the VR complex is a circle
    while k/n < 1/3 (k = steps a chord spans) and has no H1 from k/n >= 1/3 on
    (Adamaszek-Adams), so H1 has one long bar [c_1, c_ceil(n/3)) with
    c_k = 2 sin(pi k/n); H0 has n-1 bars dying at c_1.  Coordinates are
    float32, so equal chords differ by ~1e-7 and may leave bars of that
    length; every other bar must be shorter than 1e-6."""
    pts = synth.ngon(n)
    cx = oracle.vr_build(pts, 2, keep_handle=True)
    dist = np.sqrt(cx.grade_value)
    c = lambda k: 2 * math.sin(math.pi * k / n)
    h0 = cx.barcode(0)
    fin = h0[h0[:, 1] >= 0]
    assert (h0[:, 1] < 0).sum() == 1 and len(fin) == n - 1
    assert np.allclose(dist[fin[:, 1]], c(1), atol=1e-6)
    h1 = cx.barcode(1)
    fin1 = h1[h1[:, 1] >= 0]
    assert (h1[:, 1] < 0).sum() == 0
    length = dist[fin1[:, 1]] - dist[fin1[:, 0]]
    long = fin1[length > 1e-6]
    assert len(long) == 1
    assert abs(dist[long[0, 0]] - c(1)) < 1e-6
    assert abs(dist[long[0, 1]] - c(math.ceil(n / 3))) < 1e-6


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_circle_samples(seed):
    """Dense samples of the unit circle with largest angular gap gamma (chord
    c = 2 sin(gamma/2)): the loop closes when the largest gap is bridged, so
    the one long H1 bar is born at c, and it dies when the complex stops being
    a circle, within about one gap of the 120-degree chord sqrt(3)
    (Adamaszek-Adams-Frick for finite subsets of the circle); every other H1
    bar is shorter than c."""
    n = 64
    pts = synth.circle_samples(n, seed)
    ang = np.sort(np.arctan2(pts[:, 1].astype(np.float64), pts[:, 0].astype(np.float64)))
    gaps = np.diff(np.concatenate([ang, [ang[0] + 2 * math.pi]]))
    gamma = float(gaps.max())
    chord = 2 * math.sin(gamma / 2)
    cx = oracle.vr_build(pts, 2, keep_handle=True)
    dist = np.sqrt(cx.grade_value)
    h1 = cx.barcode(1)
    assert (h1[:, 1] < 0).sum() == 0
    length = dist[h1[:, 1]] - dist[h1[:, 0]]
    long = h1[length > chord]
    assert len(long) == 1
    assert abs(dist[long[0, 0]] - chord) < 1e-6
    assert abs(dist[long[0, 1]] - math.sqrt(3)) < chord


@pytest.mark.parametrize("seed,dtype,n,cap", [
    (11, np.int8, 14, math.inf), (12, np.int8, 22, 60.0), (13, np.float32, 16, math.inf),
    (14, np.float32, 25, 90.0), (15, np.int32, 18, 120.0)])
def test_euler_characteristic_every_grade(seed, dtype, n, cap):
    """At every grade g, sum_k (-1)^k #{k-simplices of grade <= g} equals
    sum_k (-1)^k beta_k(g) (bars alive at g)."""
    pts = synth.random_cloud(n, 3, dtype, seed=seed, lo=-60, hi=60)
    cx = oracle.vr_build(pts, 2, cap, keep_handle=True)
    for g in range(len(cx.grade_value)):
        chi = sum((-1) ** k * int((cx.dims[k].grade <= g).sum()) for k in range(3))
        b = oracle.betti(cx, g)
        assert chi == b[0] - b[1] + b[2], g


@pytest.mark.parametrize("seed,dtype", [(21, np.int8), (22, np.float32), (23, np.int32)])
def test_h0_deaths_are_mst_weights(seed, dtype):
    """Dimension-0 bars die at the edges of a minimum spanning tree: the
    multiset of finite H0 deaths equals Kruskal's MST weights (zero-weight
    tree edges give zero-length bars, which are dropped)."""
    pts = synth.random_cloud(30, 4, dtype, seed=seed, lo=-5, hi=5)
    cx = oracle.vr_build(pts, 1, keep_handle=True)
    h0 = cx.barcode(0)
    deaths = sorted(cx.grade_value[h0[h0[:, 1] >= 0][:, 1]].tolist())
    mst = [w for w in kruskal_weights(pts) if w > 0]
    assert deaths == mst


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny(seed):
    """n <= 10: every subset enumerated directly; same simplices, grades,
    order and boundary."""
    g = synth.rng(500 + seed)
    n = int(g.integers(1, 11))
    dtype = [np.int8, np.int32, np.float32][seed % 3]
    lo, hi = (-4, 4) if seed % 2 else (-100, 100)
    pts = synth.random_cloud(n, int(g.integers(1, 5)), dtype, seed=600 + seed, lo=lo, hi=hi)
    cap = [math.inf, 6.0, 40.0, 3.0][seed % 4]
    for maxdim in (0, 1, 2):
        check_against_brute(pts, maxdim, cap)


def test_duplicates_and_single_point():
    pts = np.array([[3, 3], [3, 3], [0, 0]], np.int32)
    cx = check_against_brute(pts, 2, math.inf)
    assert cx.dims[1].grade.tolist()[0] == 0          # d^2 = 0 -> grade 0
    one = oracle.vr_build(np.zeros((1, 2), np.float32), 2)
    assert [one.dims[k].count for k in range(3)] == [1, 0, 0]
    assert one.grade_value.tolist() == [0.0]


def test_cap_is_inclusive():
    """An edge exactly at the cap is kept; one ulp below drops it (reading:
    the filtration includes an edge from its own length on)."""
    pts = np.array([[0, 0], [3, 4]], np.int32)
    assert oracle.vr_build(pts, 1, 5.0).dims[1].count == 1
    assert oracle.vr_build(pts, 1, math.nextafter(5.0, 0)).dims[1].count == 0
    f = np.array([[0, 0], [3, 4]], np.float32)
    assert oracle.vr_build(f, 1, 5.0).dims[1].count == 1
    assert oracle.vr_build(f, 1, math.nextafter(5.0, 0)).dims[1].count == 0


def test_float_distance_within_fp64_bound():
    """The float squared distance is within the forward error bound of its
    evaluation (one subtraction, one square, one addition per coordinate:
    gamma_{d+2} relative) of the exact value, computed here in rationals."""
    g = synth.rng(77)
    for d in (1, 3, 16, 32):
        pts = (g.normal(size=(20, d)) * 10.0 ** g.integers(-3, 4, size=(20, 1))).astype(np.float32)
        u = 2.0 ** -53
        gam = (d + 2) * u / (1 - (d + 2) * u)
        for i, j in itertools.combinations(range(20), 2):
            ex = exact_d2(pts, i, j)
            got = Fraction(oracle.pair_d2(pts, i, j))
            assert abs(got - ex) <= Fraction(gam) * ex


def test_integer_distance_exact_at_extremes():
    """Integer squared distances are exact even where doubles would round:
    int32 coordinates at the type's extremes."""
    pts = np.array([[2**31 - 1, -2**31], [-2**31, 2**31 - 1]], np.int32)
    ex = 2 * (2**32 - 1) ** 2
    assert oracle.pair_d2(pts, 0, 1) == float(ex)
    small = np.array([[0, 0, 0], [2**20, 1, 0]], np.int32)
    assert oracle.pair_d2(small, 0, 1) == float(2**40 + 1)


def test_errors():
    pts = np.zeros((3, 2), np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.vr_build(pts, 4)
    with pytest.raises(oracle.OracleError):
        oracle.vr_build(pts, 2, -1.0)
    with pytest.raises(oracle.OracleError):
        oracle.vr_build(pts, 2, float("nan"))
    bad = pts.copy()
    bad[1, 1] = np.inf
    with pytest.raises(oracle.OracleError):
        oracle.vr_build(bad, 2)


# ------------------------------------------------ distance-matrix input (Sec. 3)

def brute_force_dmat(D, maxrad):
    """Every subset of a tiny matrix's vertices enumerated directly: edges
    (i < j) with D[i][j] <= maxrad, grades ranking the values themselves."""
    n = D.shape[0]
    val = {(i, j): (float(D[i, j]) if D.dtype == np.float32 else int(D[i, j]))
           for i, j in itertools.combinations(range(n), 2)}
    kept = {e: v for e, v in val.items() if v <= maxrad}
    values = sorted(set([0] + list(kept.values())))
    gidx = {v: g for g, v in enumerate(values)}
    eg = {e: gidx[v] for e, v in kept.items()}
    edges = sorted(kept, key=lambda e: (eg[e], e[0], e[1]))
    ordr = {e: t for t, e in enumerate(edges)}
    tris = sorted((max(eg[(a, b)], eg[(a, c)], eg[(b, c)]), a, b, c)
                  for a, b, c in itertools.combinations(range(n), 3)
                  if (a, b) in kept and (a, c) in kept and (b, c) in kept)
    return values, edges, [eg[e] for e in edges], ordr, tris


def random_symmetric(n, dtype, g, hi):
    a = g.integers(0, hi, size=(n, n))
    m = np.triu(a, 1)
    m = m + m.T
    if dtype == np.float32:
        m = (m * 0.25).astype(np.float32)   # quarter steps: ties, exact in fp32
    return m.astype(dtype)


@pytest.mark.parametrize("seed", range(8))
def test_dmat_brute_force_tiny(seed):
    """n <= 9 symmetric matrices with many tied values: simplices, grades,
    order, boundary and grade values equal direct enumeration."""
    g = synth.rng(900 + seed)
    n = int(g.integers(1, 10))
    dtype = np.int32 if seed % 2 else np.float32
    D = random_symmetric(n, dtype, g, 6)
    cap = [math.inf, 2.0, 0.75, 4.0][seed % 4]
    values, edges, grades, ordr, tris = brute_force_dmat(D, cap)
    cx = oracle.vr_build_dmat(D, 2, cap)
    assert cx.grade_value.tolist() == [float(v) for v in values]
    assert [tuple(x) for x in cx.dims[1].verts.tolist()] == edges
    assert cx.dims[1].grade.tolist() == grades
    assert [tuple(x) for x in cx.dims[2].verts.tolist()] == [t[1:] for t in tris]
    assert cx.dims[2].grade.tolist() == [t[0] for t in tris]
    rows = []
    for _, a, b, c in tris:
        rows += sorted([ordr[(b, c)], ordr[(a, c)], ordr[(a, b)]])
    assert cx.dims[2].rowidx.tolist() == rows


@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_dmat_of_squared_distances_equals_point_build(dtype):
    """A matrix holding a cloud's squared distances, capped at r^2, gives the
    point build capped at r (integer d^2 below 2^24, exact in float32)."""
    p = synth.random_cloud(70, 3, np.int32, seed=41, lo=-60, hi=60)
    D = ((p[:, None, :].astype(np.int64) - p[None, :, :]) ** 2).sum(-1).astype(dtype)
    a = oracle.vr_build(p, 2, 30.0)
    b = oracle.vr_build_dmat(D, 2, 900.0)
    for k in range(3):
        for f in ("verts", "grade", "colptr", "rowidx"):
            x, y = getattr(a.dims[k], f), getattr(b.dims[k], f)
            assert (x is None and y is None) or np.array_equal(x, y), (k, f)
    assert np.array_equal(a.grade_value, b.grade_value)


def test_dmat_hamming_cube():
    """Hamming distances of {0,1}^3: the cube graph at cap 1 has 12 edges and
    no triangle; at cap 2 every pair but the 4 antipodal ones is an edge."""
    v = np.array(list(itertools.product([0, 1], repeat=3)))
    D = (v[:, None, :] != v[None, :, :]).sum(-1).astype(np.int32)
    c1 = oracle.vr_build_dmat(D, 2, 1.0)
    assert [c1.dims[k].count for k in range(3)] == [8, 12, 0]
    assert c1.grade_value.tolist() == [0.0, 1.0]
    c2 = oracle.vr_build_dmat(D, 2, 2.0)
    assert c2.dims[1].count == 28 - 4
    assert c2.grade_value.tolist() == [0.0, 1.0, 2.0]


def test_dmat_rejects_invalid_matrices():
    D = np.array([[0, 1], [2, 0]], np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.vr_build_dmat(D, 1)
    with pytest.raises(oracle.OracleError):
        oracle.vr_build_dmat(np.array([[0, -1], [-1, 0]], np.int32), 1)
    with pytest.raises(oracle.OracleError):
        oracle.vr_build_dmat(np.array([[0, np.nan], [np.nan, 0]], np.float32), 1)
    ok = oracle.vr_build_dmat(np.array([[0.0, -0.0], [0.0, 0.0]], np.float32), 1)
    assert ok.dims[1].grade.tolist() == [0]


# ------------------------------------------------------------- tetrahedra

def brute_tetra(points, maxrad):
    """Tetrahedra of a tiny cloud by direct enumeration of 4-subsets: grade =
    largest edge grade, order (grade, a, b, c, d), faces as triangle order
    indices, ascending."""
    values, edges, grades, ordr, tris = brute_force(points, 2, maxrad)
    eg = dict(zip(edges, grades))
    tord = {t[1:]: i for i, t in enumerate(tris)}
    n = points.shape[0]
    tets = sorted((max(eg[(a, b)], eg[(a, c)], eg[(a, d)], eg[(b, c)], eg[(b, d)], eg[(c, d)]), a, b, c, d)
                  for a, b, c, d in itertools.combinations(range(n), 4)
                  if all(e in eg for e in itertools.combinations((a, b, c, d), 2)))
    rows = []
    for _, a, b, c, d in tets:
        rows += sorted([tord[(b, c, d)], tord[(a, c, d)], tord[(a, b, d)], tord[(a, b, c)]])
    return tets, rows


@pytest.mark.parametrize("seed", range(6))
def test_tetrahedra_brute_force_tiny(seed):
    g = synth.rng(1300 + seed)
    n = int(g.integers(4, 11))
    dtype = [np.int8, np.int32, np.float32][seed % 3]
    pts = synth.random_cloud(n, 3, dtype, seed=1400 + seed, lo=-5, hi=5)
    cap = [math.inf, 4.0, 6.0][seed % 3]
    tets, rows = brute_tetra(pts, cap)
    cx = oracle.vr_build(pts, 3, cap)
    d3 = cx.dims[3]
    assert d3.count == len(tets)
    assert [tuple(x) for x in d3.verts.tolist()] == [t[1:] for t in tets]
    assert d3.grade.tolist() == [t[0] for t in tets]
    assert d3.colptr.tolist() == [4 * t for t in range(len(tets) + 1)]
    assert d3.rowidx.tolist() == rows


def test_counts_without_cap_dim3():
    """No cap: C(n, 4) tetrahedra."""
    pts = synth.random_cloud(11, 3, np.int32, seed=5)
    cx = oracle.vr_build(pts, 3)
    assert [cx.dims[k].count for k in range(4)] == [math.comb(11, k + 1) for k in range(4)]


def test_boundary_of_4_simplex():
    """The five standard basis vectors of R^5 are pairwise at d^2 = 2: the
    3-skeleton of the 4-simplex is a 3-sphere -- bars H0 4x[0,1) + [0,inf),
    H1 and H2 none, H3 [1,inf)."""
    pts = np.eye(5, dtype=np.int32)
    cx = oracle.vr_build(pts, 3, keep_handle=True)
    assert [cx.dims[k].count for k in range(4)] == [5, 10, 10, 5]
    assert sorted(map(tuple, cx.barcode(0).tolist())) == [(0, -1), (0, 1), (0, 1), (0, 1), (0, 1)]
    assert cx.barcode(1).tolist() == []
    assert cx.barcode(2).tolist() == []
    assert cx.barcode(3).tolist() == [[1, -1]]


@pytest.mark.parametrize("seed,dtype,n,cap", [(31, np.int8, 18, 50.0), (32, np.float32, 16, 70.0)])
def test_euler_characteristic_every_grade_dim3(seed, dtype, n, cap):
    pts = synth.random_cloud(n, 3, dtype, seed=seed, lo=-60, hi=60)
    cx = oracle.vr_build(pts, 3, cap, keep_handle=True)
    for g in range(len(cx.grade_value)):
        chi = sum((-1) ** k * int((cx.dims[k].grade <= g).sum()) for k in range(4))
        b = oracle.betti(cx, g)
        assert chi == b[0] - b[1] + b[2] - b[3], g
