"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

The bar is bit-exact: same simplices, grades, order, boundary CSC and grade
values (FP64 bit equality for float inputs), on seeded inputs that span
several 32-point tiles with ragged tails, degenerate ties, both sides of the
cap, the size limits and every value error."""
import math

import numpy as np
import pytest

import oracle
import paper_1809_04424_b300 as vr
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    return t


def gpu_build(torch, pts, maxdim, maxrad, on_device=True):
    src = torch.from_numpy(np.ascontiguousarray(pts)).cuda() if on_device else pts
    c = vr.vr_build(src, maxdim, maxrad)
    out = {"counts": c.counts()[0], "gv": c.grade_values(), "stats": c.stats()}
    for k in range(maxdim + 1):
        out[k] = c.to_host(k)
    return out


def assert_same(g, o, maxdim):
    assert g["gv"].tobytes() == o.grade_value.tobytes(), "grade values differ"
    for k in range(maxdim + 1):
        od, gd = o.dims[k], g[k]
        assert gd["count"] == od.count, (k, gd["count"], od.count)
        np.testing.assert_array_equal(gd["verts"], od.verts, err_msg=f"verts dim {k}")
        np.testing.assert_array_equal(gd["grade"], od.grade, err_msg=f"grade dim {k}")
        if k >= 1:
            np.testing.assert_array_equal(gd["colptr"], od.colptr, err_msg=f"colptr dim {k}")
            np.testing.assert_array_equal(gd["rowidx"], od.rowidx, err_msg=f"rowidx dim {k}")


def check(torch, pts, maxdim, maxrad, on_device=True):
    g = gpu_build(torch, pts, maxdim, maxrad, on_device)
    o = oracle.vr_build(pts, maxdim, maxrad)
    assert_same(g, o, maxdim)
    return g


def test_config1_plain_cloud(torch):
    c = synth.config1()
    g = check(torch, c.points, c.maxdim, c.maxrad)
    assert g["counts"] == [64, 2016, 41664]


def test_config2_torus_int8(torch):
    c = synth.config2()
    g = check(torch, c.points, c.maxdim, c.maxrad)
    assert g["counts"][2] > 100000


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 65, 100, 257])
@pytest.mark.parametrize("dtype", [np.int8, np.int32, np.float32])
def test_random_clouds_no_cap(torch, n, dtype):
    pts = synth.random_cloud(n, 3, dtype, seed=1000 + n)
    check(torch, pts, 2, math.inf)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("dtype", [np.int8, np.int32, np.float32])
def test_random_clouds_capped(torch, seed, dtype):
    g = synth.rng(2000 + seed)
    n = int(g.integers(50, 700))
    d = int(g.integers(1, 9))
    pts = synth.random_cloud(n, d, dtype, seed=3000 + seed, lo=-50, hi=50)
    cap = float(g.uniform(10, 60))
    for maxdim in (0, 1, 2):
        check(torch, pts, maxdim, cap)


def test_cap_edge_exactly_at_radius(torch):
    pts = np.array([[0, 0], [3, 4], [6, 8], [0, 5]], np.int32)
    check(torch, pts, 2, 5.0)
    check(torch, pts, 2, math.nextafter(5.0, 0))
    f = pts.astype(np.float32)
    check(torch, f, 2, 5.0)
    check(torch, f, 2, math.nextafter(5.0, 0))


@pytest.mark.parametrize("n", [40, 90])
def test_all_points_equal_int(torch, n):
    """Every pair at d^2 = 0: one grade holds everything; the triangle tie
    merge runs its large-segment path (C(90,3) > 4096)."""
    pts = np.full((n, 3), 7, np.int8)
    check(torch, pts, 2, math.inf)


@pytest.mark.parametrize("n", [8, 50, 70, 110])
def test_all_points_equal_float(torch, n):
    """Float repair groups of every size class (thread, CTA, global sort)."""
    pts = np.full((n, 4), 0.25, np.float32)
    check(torch, pts, 2, math.inf)


def test_lattice_many_ties(torch):
    """Integer lattice: massive distance ties, multi-edge grade groups."""
    ax = np.arange(-4, 5)
    pts = np.stack(np.meshgrid(ax, ax, ax[:4]), -1).reshape(-1, 3).astype(np.int32)
    check(torch, pts, 2, 2.5)
    check(torch, pts, 2, math.inf)


@pytest.mark.parametrize("n", [12, 60, 200])
def test_float_ngon_near_ties(torch, n):
    """Equal chords of a regular polygon differ only by fp32 rounding: the
    first-pass order must be repaired to the FP64 order."""
    pts = synth.ngon(n, 3.0)
    g = check(torch, pts, 2, 2.0)
    assert g["stats"]["max_rel_dist_err"] <= 1e-6


def test_float_config3_small(torch):
    """The 32-dimensional Gaussian-mixture shape at n = 700."""
    c = synth.config3(n=700)
    g = check(torch, c.points, 2, c.maxrad)
    assert g["stats"]["max_rel_dist_err"] <= 1e-6


def test_host_pointer_input(torch):
    c = synth.config1()
    g = gpu_build(torch, c.points, 2, c.maxrad, on_device=False)
    assert_same(g, oracle.vr_build(c.points, 2, c.maxrad), 2)


def test_max_size_sampled(torch):
    """n = 8192 (the id-field limit) with a small cap: full parity."""
    g = synth.rng(8192)
    pts = g.integers(-127, 128, size=(8192, 3)).astype(np.int8)
    check(torch, pts, 2, 9.0)


@pytest.mark.parametrize("n", [4096, 4097])
def test_dense_edge_table_boundary(torch, n):
    """Lex-order triangles on both sides of 4096 points (above it the lex
    order is forced; the dense edge tables serve both)."""
    g = synth.rng(4096 + n)
    pts = g.integers(-20, 21, size=(n, 3)).astype(np.int8)
    c = check(torch, pts, 2, 4.0)
    assert len(c[2]["grade"]) > 10000


def test_lex_mode_beyond_early_triangle_limit(torch):
    """Tie-heavy integer cloud with about 199k kept edges (more than 2^17) and
    8.8M triangles: lex order with the triangle keys allocated after the
    triangle count is read (not from the all-graphs bound), in full."""
    g = synth.rng(1800)
    pts = g.integers(-12, 13, size=(1800, 3)).astype(np.int8)
    c = check(torch, pts, 2, 9.0)
    assert len(c[1]["grade"]) > (1 << 17)


@pytest.mark.parametrize("box,r,maxdim", [(15, 5.0, 2), (20, 4.0, 3)])
def test_sparse_rows_lex_mode(torch, box, r, maxdim):
    """Tie-heavy int8 clouds whose average degree (about 36 and 8) is below
    the 79 bitmap words per row: lex order, with the candidates of each edge
    taken from the lexicographic edge list (one bit test each), in full."""
    g = synth.rng(1811)
    pts = g.integers(-box, box + 1, size=(2500, 3)).astype(np.int8)
    c = check(torch, pts, maxdim, r)
    E = len(c[1]["grade"])
    assert 2 * E < 2500 * ((2500 + 31) // 32)  # sparse rows
    assert len(c[2]["grade"]) > 10000


def test_worldmap_shaped_cloud(torch):
    """The WorldMap-shaped single cloud (n = 7322 float32 on the unit sphere,
    cap 0.15): 280,777 edges and 5,878,554 triangles, in full."""
    c = synth.worldmap()
    g = check(torch, c.points, 2, c.maxrad)
    assert g["counts"] == [7322, 280777, 5878554]
    assert g["stats"]["max_rel_dist_err"] <= 1e-6


def test_value_errors(torch):
    bad = np.zeros((5, 2), np.float32)
    bad[2, 1] = np.nan
    with pytest.raises(vr.VRError) as e:
        vr.vr_build(torch.from_numpy(bad).cuda(), 2)
    assert e.value.status == vr.VR_ERR_ARG
    big = np.zeros((5, 2), np.float32)
    big[1, 0] = 1e20
    with pytest.raises(vr.VRError) as e:
        vr.vr_build(torch.from_numpy(big).cuda(), 2)
    assert e.value.status == vr.VR_ERR_RANGE
    huge = np.array([[0, 0], [2**20, 0]], np.int32)
    with pytest.raises(vr.VRError) as e:
        vr.vr_build(torch.from_numpy(huge).cuda(), 2)
    assert e.value.status == vr.VR_ERR_RANGE
    # the same pair beyond the cap is not an error
    ok = vr.vr_build(torch.from_numpy(huge).cuda(), 2, 10.0)
    assert ok.counts()[0] == [2, 0, 0]


def test_repeat_builds_identical(torch):
    c = synth.config2()
    a = gpu_build(torch, c.points, 2, c.maxrad)
    b = gpu_build(torch, c.points, 2, c.maxrad)
    for k in range(3):
        for f in ("verts", "grade", "colptr", "rowidx"):
            if a[k][f] is not None:
                np.testing.assert_array_equal(a[k][f], b[k][f])


@pytest.mark.parametrize("cluster,spread", [(12, 600), (30, 1000), (60, 2000)])
def test_rare_ties_merge_paths(torch, cluster, spread):
    """Few tied edges (max-edge enumeration) but one grade group -- the
    duplicated points' d^2 = 0 -- spanning many edges with triangles: C(12,3),
    C(30,3) and C(60,3) triangles exercise the small, mid and large merges."""
    g = synth.rng(4000 + cluster)
    pts = g.integers(-20000, 20001, size=(spread, 3)).astype(np.int64)
    pts[:cluster] = 100000          # far beyond the cap from every other point
    iu = np.triu_indices(spread, 1)
    d2 = ((pts[iu[0]] - pts[iu[1]]) ** 2).sum(1)
    want = 25 * cluster * (cluster - 1) // 2              # tied edges stay near 4%
    cap2 = np.partition(d2, want)[want]
    pts = pts.astype(np.int32)
    check(torch, pts, 2, math.sqrt(float(cap2)))


def test_both_enumeration_orders_on_one_cloud(torch):
    """The same torus cloud through both orders: lex order (ties, default cap)
    and, with a cap so small that few edges tie, max-edge order."""
    c = synth.config2(n=400)
    assert check(torch, c.points, 2, c.maxrad)["stats"]["tri_order"] == 1
    check(torch, c.points, 2, 6.0)


@pytest.mark.parametrize("width", [0, 8])
def test_max_edge_key_widths(torch, width):
    """1200 float32 points in d = 32 at the 5% cap (about 36k kept edges and
    dense rows: max-edge order) with the triangle keys in 32 bits (automatic)
    and forced to 64 bits, both in full."""
    c = synth.config3(n=1200)
    vr.vr_set_tri_key_width(width)
    try:
        g = check(torch, c.points, 2, c.maxrad)
    finally:
        vr.vr_set_tri_key_width(0)
    E = len(g[1]["grade"])
    assert E >= (1 << 15) and 2 * E >= 1200 * ((1200 + 31) // 32)


def test_float_ties_lex_order_without_dense_tables(torch):
    """The 1000-point torus cloud as float32: its squared distances are
    integers, so most edges tie.  The host, seeing float input with dense
    rows, takes the claimed max-edge path and leaves out the dense order
    tables; the device finds the ties and takes lex order, whose kernels then
    look faces up through the neighbour CSR.  Every output in full."""
    c = synth.config2()
    g = check(torch, c.points.astype(np.float32), 2, c.maxrad)
    assert g["stats"]["tri_order"] == 1 and g["counts"][2] > 100000


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_max_edge_key_space_modes(torch, mode):
    """The 1200-point float cloud (max-edge order) with its keys in claimed
    space (the generator before any count, then a compaction into keys in
    output order), counted (count, scan, generator), and claimed with sub-buffers too
    small for the claims (the counted generator takes over from the claiming
    run's counts): every output in full."""
    c = synth.config3(n=1200)
    vr.vr_set_tri_claim(mode)
    try:
        g = check(torch, c.points, 2, c.maxrad)
    finally:
        vr.vr_set_tri_claim(0)
    assert g["stats"]["tri_order"] == (3 if mode == 0 else 2)  # max-edge, claimed or counted


def test_max_edge_claimed_ragged_chunks(torch):
    """1500 uniform float32 points in d = 32 capped at 4% of pairs: few
    triangles per edge and many edges with none, so each 32-edge group of the
    compaction of claimed third vertices has short, uneven runs; a ragged
    triangle count.  Max-edge order, claimed key space, in full."""
    pts = synth.rng(77).uniform(-1.0, 1.0, size=(1500, 32)).astype(np.float32)
    d2 = ((pts[:, None, :].astype(np.float64) - pts[None, :, :]) ** 2).sum(-1)[np.triu_indices(1500, 1)]
    cap2 = float(np.quantile(d2, 0.04))
    g = check(torch, pts, 2, math.sqrt(cap2))
    T = len(g[2]["grade"])
    E = len(g[1]["grade"])
    assert E >= (1 << 15) and 2 * E >= 1500 * ((1500 + 31) // 32)  # max-edge order
    assert T % 128 != 0 and T < 32 * E


@pytest.mark.parametrize("n", [4500, 6200])
def test_max_edge_wide_rows(torch, n):
    """Gaussian-mixture clouds (d = 32, 5% cap) whose snapshot rows take 3
    and 4 16-byte chunks per generator lane (144 and 196 words): 506k edges
    and 28M triangles with 32-bit keys; 961k edges (more than a 13-bit vertex
    leaves room for) and 73M triangles with 64-bit keys; in full."""
    c = synth.config3(n=n)
    g = check(torch, c.points, 2, c.maxrad)
    E = len(g[1]["grade"])
    assert 2 * E >= n * ((n + 31) // 32)  # dense rows: max-edge order
    assert (E > 1 << 19) == (n == 6200)
    # The host takes claimed key space while the wedge-bound buffer (T_wedge
    # keys of 4 B, or 8 B when the edge index does not fit beside the vertex)
    # stays within 1 GB, else the counted path.
    deg = np.bincount(g[1]["verts"].ravel(), minlength=n).astype(np.int64)
    t_wedge = int((deg * (deg - 1) // 2).sum()) // 3 + 1
    key_bytes = 4 if E <= 1 << (32 - (n - 1).bit_length()) else 8
    assert g["stats"]["tri_order"] == (3 if t_wedge * key_bytes <= 1 << 30 else 2)


@pytest.mark.parametrize("maxdim", [2, 1])
def test_config3_gaussian_mixture_full(torch, maxdim):
    """Full size: 4000 float32 points in d = 32, cap keeping 5% of pairs
    (about 0.4M edges and 19.8M triangles), every output bit-exact."""
    c = synth.config3(maxdim=maxdim)
    g = check(torch, c.points, maxdim, c.maxrad)
    assert g["stats"]["max_rel_dist_err"] <= 1e-6
    assert g["stats"]["tri_order"] == (3 if maxdim == 2 else 0)  # max-edge order, claimed key space


def test_config3_counted_path_full(torch):
    """The full 4000-point float cloud through the counted max-edge path
    (triangle count, scan, generator at the scanned offsets, key-reading final
    write, dense order tables): every output bit-exact, as on the claimed
    path."""
    c = synth.config3()
    vr.vr_set_tri_claim(1)
    try:
        g = check(torch, c.points, 2, c.maxrad)
    finally:
        vr.vr_set_tri_claim(0)
    assert g["stats"]["tri_order"] == 2


@pytest.mark.parametrize("seed", [1, 2])
def test_float_wide_dynamic_range(torch, seed):
    """Coordinates spanning many binades, zeros included: the integer
    evaluation of the FP64 sequence and its hardware fallback (exponents more
    than 29 apart) must both reproduce the oracle's doubles exactly."""
    g = synth.rng(7000 + seed)
    pts = g.normal(size=(300, 6)) * 10.0 ** g.integers(-12, 6, size=(300, 6))
    pts[g.random(size=pts.shape) < 0.2] = 0.0
    pts = pts.astype(np.float32)
    check(torch, pts, 2, math.inf if seed == 1 else 1e-3)


@pytest.mark.parametrize("dtype", [np.int8, np.float32])
def test_zero_radius_keeps_duplicates(torch, dtype):
    """maxrad = 0: only coincident points are joined (d^2 = 0 <= 0)."""
    pts = synth.random_cloud(40, 2, np.int8, seed=91, lo=-3, hi=3).astype(dtype)
    g = check(torch, pts, 2, 0.0)
    assert g["counts"][1] > 0
