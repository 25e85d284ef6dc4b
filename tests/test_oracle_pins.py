"""Pins of the oracle against facts fixed by the paper and by the mathematics.

Each test checks the exact CPU oracle (``oracle/``) against something other
than itself: closed-form cells, an independent exact half-plane clipper, the
empty-circle definition of the Delaunay graph, global invariants (Euler's
relation, total area, equidistance, the bound on Delaunay edges) and the
counting lemmas of the paper's correctness proof.
"""

from fractions import Fraction as F

import numpy as np
import pytest

import oracle
import synth
from bruteforce import halfplane_cell, polygon_area, restricted_delaunay

MODES = ["plain", "bucketed"]


def _cell(res, i):
    a, b = res["cell_ptr"][i], res["cell_ptr"][i + 1]
    return [int(v) for v in res["labels"][a:b]], oracle.vertices_exact(res, i)


def _tiny(n, seed, box):
    """n distinct integer sites strictly inside [0, box]^2."""
    return synth.uniform_sites(n, seed=seed, box=box)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("mode", MODES)
def test_single_site_is_the_box(mode):
    # n = 1: the cell is X itself; edges ordered right, top, left, bottom.
    xy = np.array([[300, 700]], dtype=np.int32)
    r = oracle.cells(xy, (1000, 800), mode, bucket_side=100, beta=1)
    labels, verts = _cell(r, 0)
    assert labels == [-2, -3, -4, -1]
    assert verts == [(1000, 800), (0, 800), (0, 0), (1000, 0)]
    assert r["delaunay"].shape[0] == 0


@pytest.mark.parametrize("mode", MODES)
def test_two_sites_split_by_their_bisector(mode):
    xy = np.array([[100, 500], [300, 500]], dtype=np.int32)
    r = oracle.cells(xy, 1000, mode, bucket_side=50, beta=1)
    assert _cell(r, 0) == ([1, -3, -4, -1], [(200, 1000), (0, 1000), (0, 0), (200, 0)])
    assert _cell(r, 1) == ([-2, -3, 0, -1], [(1000, 1000), (200, 1000), (200, 0), (1000, 0)])
    assert r["delaunay"].tolist() == [[0, 1]]


@pytest.mark.parametrize("mode", MODES)
def test_bisector_through_two_corners(mode):
    # p = (1,3), a = (3,1) in [0,4]^2: the bisector is the diagonal y = x.
    xy = np.array([[1, 3], [3, 1]], dtype=np.int32)
    r = oracle.cells(xy, 4, mode, bucket_side=1, beta=1)
    assert _cell(r, 0) == ([-3, -4, 1], [(0, 4), (0, 0), (4, 4)])
    assert _cell(r, 1) == ([-2, 0, -1], [(4, 4), (0, 0), (4, 0)])
    # both cells have two vertices where three lines meet (box corners)
    assert r["stats"][:, 5].tolist() == [2, 2]


@pytest.mark.parametrize("mode", MODES)
def test_lattice_cells_are_squares(mode):
    # k x k lattice at odd offsets: every cell is a square (the most
    # degenerate input: four sites on every circle through a vertex) and the
    # Delaunay graph is the 4-neighbour grid graph.
    k, sp, off = 6, 20, 10
    xy = synth.lattice_sites(k, sp, off)
    r = oracle.cells(xy, k * sp, mode, bucket_side=16, beta=1)
    for idx in range(k * k):
        i, j = divmod(idx, k)
        labels, verts = _cell(r, idx)
        x0, x1, y0, y1 = i * sp, (i + 1) * sp, j * sp, (j + 1) * sp
        right = (i + 1) * k + j if i + 1 < k else -2
        top = i * k + j + 1 if j + 1 < k else -3
        left = (i - 1) * k + j if i > 0 else -4
        bottom = i * k + j - 1 if j > 0 else -1
        assert labels == [right, top, left, bottom]
        assert verts == [(x1, y1), (x0, y1), (x0, y0), (x1, y0)]
    want = sorted([(a, a + 1) for a in range(k * k) if (a + 1) % k != 0] +
                  [(a, a + k) for a in range(k * k - k)])
    assert sorted(map(tuple, r["delaunay"].tolist())) == want
    # interior lattice vertices lie on four lines of each incident cell
    interior = r["stats"][:, 5]
    assert interior[(k // 2) * k + k // 2] == 4


@pytest.mark.parametrize("mode", MODES)
def test_collinear_sites_give_strips(mode):
    # sites on one horizontal line: parallel bisectors (the det(B) = 0,
    # L1 != L2 case of Algorithm 1)
    xs = [100, 300, 500, 700]
    xy = np.array([[x, 400] for x in xs], dtype=np.int32)
    r = oracle.cells(xy, (800, 800), mode, bucket_side=40, beta=1)
    bounds = [0, 200, 400, 600, 800]
    for i in range(4):
        labels, verts = _cell(r, i)
        right = i + 1 if i < 3 else -2
        left = i - 1 if i > 0 else -4
        assert labels == [right, -3, left, -1]
        x0, x1 = bounds[i], bounds[i + 1]
        assert verts == [(x1, 800), (x0, 800), (x0, 0), (x1, 0)]
    assert r["delaunay"].tolist() == [[0, 1], [1, 2], [2, 3]]


@pytest.mark.parametrize("mode", MODES)
def test_ray_through_a_degenerate_vertex(mode):
    # The projector corner (0,1) from p = (50,50) meets v = (50,60), which is
    # equidistant from p and the three sites (60,60), (40,60), (50,70).  The
    # bisector of p and (50,70) touches the cell only at v (Remark A.4).
    xy = np.array([[50, 50], [60, 60], [40, 60], [50, 70]], dtype=np.int32)
    r = oracle.cells(xy, 100, mode, bucket_side=10, beta=1)
    labels, verts = _cell(r, 0)
    assert labels == [-2, 1, 2, -4, -1]
    assert verts[:3] == [(100, 10), (50, 60), (0, 10)]
    for k in range(4):
        assert _cell(r, k) == halfplane_cell(xy, k, 100, 100)
    cc, cw, ties, t, _ = oracle.endpoint(xy, 100, 0, (0, 1), mode, bucket_side=10, beta=1)
    assert (cc, cw, ties, t) == (2, 1, 3, 10)


def test_input_validation():
    box = 100
    with pytest.raises(oracle.OracleError) as e:
        oracle.cells(np.array([[0, 5], [3, 4]], dtype=np.int32), box)
    assert e.value.code == -2
    with pytest.raises(oracle.OracleError) as e:
        oracle.cells(np.array([[5, 100], [3, 4]], dtype=np.int32), box)
    assert e.value.code == -2
    with pytest.raises(oracle.OracleError) as e:
        oracle.cells(np.array([[5, 5], [3, 4], [5, 5]], dtype=np.int32), box)
    assert e.value.code == -3
    with pytest.raises(oracle.OracleError) as e:
        oracle.cells(np.array([[5, 5]], dtype=np.int32), (1 << 20) + 1)
    assert e.value.code == -4


# ------------------------------------------------- independent brute force

@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed", range(40))
def test_cells_equal_halfplane_intersection(mode, seed):
    n = 3 + seed % 20
    box = 64 if seed % 3 == 0 else 4096
    xy = _tiny(n, 7000 + seed, box)
    r = oracle.cells(xy, box, mode, bucket_side=max(1, box // 8), beta=1 + seed % 3)
    for k in range(n):
        assert _cell(r, k) == halfplane_cell(xy, k, box, box), (seed, k)


@pytest.mark.parametrize("seed", range(25))
def test_delaunay_equals_empty_circle_rule(seed):
    n = 4 + seed % 14
    box = 48 if seed % 2 else 1 << 20
    xy = _tiny(n, 9100 + seed, box)
    r = oracle.cells(xy, box, "plain")
    got = sorted(map(tuple, r["delaunay"].tolist()))
    assert got == restricted_delaunay(xy, box, box), seed
    if n >= 3:
        assert len(got) <= 3 * n - 6


def test_extreme_coordinates():
    # sites at the bit-budget extremes of the 2^20 world
    M = (1 << 20) - 1
    xy = np.array([[1, 1], [M, M], [1, M], [M, 1], [2, 1], [1, 2], [M - 1, M],
                   [1 << 19, 1 << 19], [(1 << 19) + 1, 1 << 19], [3, M - 5]], dtype=np.int32)
    box = 1 << 20
    for mode in MODES:
        r = oracle.cells(xy, box, mode, bucket_side=1 << 16, beta=2)
        for k in range(len(xy)):
            assert _cell(r, k) == halfplane_cell(xy, k, box, box), (mode, k)


# ----------------------------------------------------- Theorem 2.2 property

@pytest.mark.parametrize("mode", MODES)
def test_endpoint_is_ray_exit_of_the_cell(mode):
    # T(p, theta) of eq. (2.1): the ray leaves the cell R_k at the endpoint.
    rng = np.random.default_rng(5)
    box = 10_000
    xy = _tiny(25, 4242, box)
    for k in range(0, 25, 3):
        labels, verts = halfplane_cell(xy, k, box, box)
        px, py = int(xy[k][0]), int(xy[k][1])
        for _ in range(12):
            th = tuple(int(v) for v in rng.integers(-(1 << 40), 1 << 40, size=2))
            ccw, cw, ties, t, _ = oracle.endpoint(xy, box, k, th, mode, bucket_side=625, beta=1)
            # exit parameter of the ray from the polygon, by its edges
            best = None
            m = len(verts)
            for i in range(m):
                A, B = verts[i - 1], verts[i]
                # solve p + t th = A + s (B - A)
                ex, ey = B[0] - A[0], B[1] - A[1]
                det = th[0] * (-ey) + ex * th[1]
                if det == 0:
                    continue
                rx, ry = A[0] - px, A[1] - py
                tt = (rx * (-ey) + ex * ry) / det
                ss = (th[0] * ry - th[1] * rx) / det
                if tt > 0 and 0 <= ss <= 1:
                    best = tt if best is None else min(best, tt)
            assert t == best
            assert ccw in labels and cw in labels


# ------------------------------------------------------- global invariants

def _invariants(xy, box, r):
    n = len(xy)
    V = set()
    E = set()
    area = F(0)
    nb = {k: set() for k in range(n)}
    for k in range(n):
        labels, verts = _cell(r, k)
        area += polygon_area(verts)
        m = len(verts)
        for i in range(m):
            V.add(verts[i])
            E.add(frozenset((verts[i - 1], verts[i])))
            if labels[i] >= 0:
                nb[k].add(labels[i])
        px, py = int(xy[k][0]), int(xy[k][1])
        for i in range(m):
            a, b = labels[i], labels[(i + 1) % m]
            if a >= 0 and b >= 0:
                vx, vy = verts[i]
                d0 = (vx - px) ** 2 + (vy - py) ** 2
                for s in (a, b):
                    assert (vx - int(xy[s][0])) ** 2 + (vy - int(xy[s][1])) ** 2 == d0
    assert len(V) - len(E) + n == 1, "Euler's relation V - E + F = 1"
    assert area == F(box) * F(box), "cell areas sum to the area of X"
    for k in range(n):
        for j in nb[k]:
            assert k in nb[j], "neighbour relation is symmetric"
    if n >= 3:
        assert r["delaunay"].shape[0] <= 3 * n - 6


@pytest.mark.parametrize("seed", range(6))
def test_global_invariants_random(seed):
    box = 1 << 20
    xy = synth.uniform_sites(300 + 50 * seed, seed=100 + seed)
    r = oracle.cells(xy, box, "bucketed")
    _invariants(xy, box, r)


def test_global_invariants_clustered():
    box = 1 << 20
    xy = synth.gaussian_mixture_sites(800, seed=77, sigma=3000.0)
    r = oracle.cells(xy, box, "bucketed")
    _invariants(xy, box, r)


def test_global_invariants_degenerate_lattice():
    k, sp = 9, 1000
    xy = synth.lattice_sites(k, sp, sp // 2)
    r = oracle.cells(xy, k * sp, "plain")
    _invariants(xy, k * sp, r)


# ------------------------------------------------ counting lemmas (Sec. 8)

@pytest.mark.parametrize("mode", MODES)
def test_algorithm_counters(mode):
    box = 1 << 20
    n = 2000
    xy = synth.uniform_sites(n, seed=31)
    r = oracle.cells(xy, box, mode)
    st = r["stats"]
    rays, nodes, e = st[:, 0], st[:, 1], st[:, 6]
    assert np.all(rays <= e + 1), "Lemma BoundShotRays: rho_k <= e_k + 1"
    assert np.all(nodes <= 2 * e), "Lemma e_k: at most 2 e_k tree nodes"
    assert e.sum() <= 10 * n, "sum of e_k <= (|X_e| + 6) n"
    assert rays.sum() <= 11 * n, "sum of rho_k <= (|X_e| + 7) n"
    assert np.all(st[:, 7] == 0), "Lemma IntermediateRay"
    assert np.all(st[:, 2] == 2 * (nodes - 1)), "two endpoints per subedge"
    # a subedge tree is binary: one extra node per split, two nodes per ray added
    assert np.all(nodes == 1 + 3 + 2 * (rays - 3))


def test_plain_equals_bucketed_at_scale():
    box = 1 << 20
    xy = synth.uniform_sites(20000, seed=12)
    a = oracle.cells(xy, box, "bucketed")
    sel = np.arange(0, 20000, 97)
    b = oracle.cells(xy, box, "plain", sel=sel)
    for i, k in enumerate(sel):
        assert _cell(b, i) == _cell(a, int(k))
    # bucketed: distance comparisons per ray stay far below n (Method A.6)
    assert a["stats"][:, 3].sum() / a["stats"][:, 0].sum() < 500


@pytest.mark.parametrize("beta,side", [(1, None), (1, 2000), (2, 50000), (4, None)])
def test_bucketed_output_is_independent_of_beta_and_side(beta, side):
    # Method A.6 takes any bucket side s > 0 and any integer beta > 0;
    # Proposition A.8: the endpoint is the exact first hit for every such
    # choice, so every choice returns the plain method's cells.  (The stored
    # digests of the large clustered workloads use beta = 1.)
    box = 1 << 20
    xy = synth.gaussian_mixture_sites(3000, seed=77, sigma=3000.0)
    ref = oracle.cells(xy, box, "plain")
    got = oracle.cells(xy, box, "bucketed", beta=beta, bucket_side=side)
    for key in ("cell_ptr", "labels", "vnum", "delaunay"):
        assert np.array_equal(got[key], ref[key]), key


# ---------------------------------------------------- Method A.6 worked example

def test_si_worked_example():
    # Appendix 3, proof of Theorem 8.1(e): X = [0,300]^2, s = 1, beta = 3,
    # y~ = (0.4, 50.2), 4 sqrt(2)(beta + 1.01) ~ 22.68.  The golden file holds
    # the printed values.
    gold = {}
    with open(__file__.replace("test_oracle_pins.py", "golden/si_example.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                key, val = line.split("=")
                gold[key.strip()] = [int(v) for v in val.split(",")]
    # eta is the integer ceiling of 22.68...
    assert oracle.eta(3, 1) == 23
    x0, x1, y0, y1 = oracle.si_rect((F(2, 5), F(251, 5)), F(2268, 100), 1)
    # intersected with X, the x-range is the printed [0, 24]
    assert [max(x0, 0), min(x1, 300)] == gold["x_range_printed"]
    # eq. (A.3) gives y-range [floor(27.52), floor(72.88) + 1] = [27, 73];
    # the printed upper end 72 is one less (see the reading in the fixture)
    assert [y0, y1] == gold["y_range_eq_A3"]
    assert gold["y_range_printed"][0] == y0 and gold["y_range_printed"][1] == y1 - 1
