"""GPU parity: the CUDA path (through the C ABI) against the exact oracle.

Combinatorial output (cell offsets, edge labels in canonical order, Delaunay
pairs) must be bit-identical; float64 vertices within 1e-9 relative of the
oracle's exact rationals.
"""

import numpy as np
import pytest

import oracle
import synth
from parity import (assert_full_parity, assert_sampled_parity, assert_shared_vertices_identical,
                    delaunay_symmetric_ok, to_numpy)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1212_1095_gb300 as vg  # noqa: E402

BOX = 1 << 20


def gpu(xy, box, **opts):
    t = torch.from_numpy(np.ascontiguousarray(xy, dtype=np.int32)).cuda()
    return to_numpy(vg.build(t, box, **opts))


# ----------------------------------------------------------- closed forms

def test_single_site():
    d = gpu(np.array([[300, 700]]), (1000, 800))
    assert d["labels"].tolist() == [-2, -3, -4, -1]
    assert d["vx"].tolist() == [1000, 0, 0, 1000] and d["vy"].tolist() == [800, 800, 0, 0]
    assert d["delaunay"].shape[0] == 0


@pytest.mark.parametrize("lanes", [2, 4, 8, 16, 32])
def test_lattice_and_degenerate_layouts(lanes):
    cases = [
        (synth.lattice_sites(7, 20, 10), 140),
        (np.array([[x, 400] for x in (100, 300, 500, 700)]), 800),
        (np.array([[1, 3], [3, 1]]), 4),
        (np.array([[50, 50], [60, 60], [40, 60], [50, 70]]), 100),
        (synth.lattice_sites(12, 1000, 500), 12000),
    ]
    for xy, box in cases:
        for exact_only in (0, 1):
            d = gpu(xy, box, lanes_per_cell=lanes, exact_only=exact_only)
            assert_full_parity(d, oracle.cells(xy, box, "plain"))


@pytest.mark.parametrize("seed", range(12))
def test_small_random_sets(seed):
    n = [1, 2, 3, 5, 8, 13, 40, 77, 150, 333, 512, 999][seed]
    box = [64, 1000, 4096, 1 << 20][seed % 4]
    xy = synth.uniform_sites(n, seed=500 + seed, box=box)
    r = oracle.cells(xy, box, "plain")
    for lanes in (4, 8, 32):
        assert_full_parity(gpu(xy, box, lanes_per_cell=lanes), r)


def test_uniform_1k_all_variants():
    # n = 1,000 uniform sites, no four co-circular; every kernel variant
    xy = synth.workload("uniform_1k")
    r = oracle.cells(xy, BOX, "plain")
    assert r["stats"][:, 5].sum() == 0, "general position"
    for lanes in (2, 4, 8, 16, 32):
        for target in (6, 20, 40):
            assert_full_parity(gpu(xy, BOX, lanes_per_cell=lanes, target=target), r)
    assert_full_parity(gpu(xy, BOX, exact_only=1), r)
    for block in (32, 128):                            # block shapes of the first pass
        assert_full_parity(gpu(xy, BOX, block_threads=block), r)
    # tiny buckets force certificate reruns, huge buckets the large-cell pass
    for side in (2000, 8000, 200000, 1 << 20):
        assert_full_parity(gpu(xy, BOX, bucket_side=side), r)
    # adaptive buckets: none divided, every bucket of 4+ sites divided, and
    # large buckets divided into up to 16 x 16 sub-buckets
    for side in (0, 65536, 200000, 1 << 20):
        for split in (0, 4, 12, 64):
            assert_full_parity(gpu(xy, BOX, bucket_side=side, fine_split=split), r)


def test_extreme_coordinates():
    M = BOX - 1
    xy = np.array([[1, 1], [M, M], [1, M], [M, 1], [2, 1], [1, 2], [M - 1, M],
                   [1 << 19, 1 << 19], [(1 << 19) + 1, 1 << 19], [3, M - 5]])
    assert_full_parity(gpu(xy, BOX), oracle.cells(xy, BOX, "plain"))


@pytest.fixture(scope="module")
def clustered_60k():
    xy = synth.gaussian_mixture_sites(60000, seed=4242, sigma=2000.0)
    return xy, oracle.cells(xy, BOX, "bucketed")


@pytest.mark.parametrize("split", [0, 4, 12])
def test_clustered_medium(clustered_60k, split):
    xy, r = clustered_60k
    t = torch.from_numpy(np.ascontiguousarray(xy, dtype=np.int32)).cuda()
    res = vg.build(t, BOX, collect_stats=1, fine_split=split)
    assert_full_parity(to_numpy(res), r)
    # the cluster cores are dense enough for the adaptive buckets to divide
    assert (res.stats["divided_buckets"] > 0) == (split != 0)


def test_cells_with_hundreds_of_edges():
    # three hubs (indices 0..2), each ringed by 200 sites: every hub's cell is
    # a 200-gon, so the first 32 cells hold 745 edges, more than one warp of
    # the compaction stages (512); those cells go through its per-lane path
    # after the medium and large tiers
    pts = [[200000, 500000], [500000, 500000], [800000, 500000]]
    for cx, cy in list(pts):
        a = 2 * np.pi * (np.arange(200) + 0.25) / 200
        ring = np.stack([np.rint(cx + 20000 * np.cos(a)), np.rint(cy + 20000 * np.sin(a))], 1)
        pts += ring.astype(np.int64).tolist()
    xy = np.array(pts, dtype=np.int32)
    r = oracle.cells(xy, BOX, "plain")
    assert np.diff(r["cell_ptr"])[:3].tolist() == [200, 200, 200]
    assert_full_parity(gpu(xy, BOX), r)


def test_errors_are_reported():
    with pytest.raises(vg.VorError) as e:
        gpu(np.array([[0, 5], [3, 4]]), 100)
    assert e.value.code == -2
    with pytest.raises(vg.VorError) as e:
        gpu(np.array([[5, 5], [3, 4], [5, 5]]), 100)
    assert e.value.code == -3
    with pytest.raises(vg.VorError) as e:
        gpu(np.array([[5, 5]]), (1 << 20) + 1)
    assert e.value.code in (-1, -4)
    # one equal pair among 1,000 sites: found by the first pass's gather
    # (one lane per cell) and by the per-bucket comparison (8 lanes)
    xy = synth.workload("uniform_1k").copy()
    xy[777] = xy[123]
    for lanes in (1, 8):
        with pytest.raises(vg.VorError) as e:
            gpu(xy, BOX, lanes_per_cell=lanes)
        assert e.value.code == -3
    # the context stays usable after device-detected errors
    d = gpu(np.array([[30, 40], [60, 20]]), 100)
    assert d["cell_ptr"][-1] > 0


def test_uniform_1m_full_parity():
    # n = 1,048,576 uniform sites (the benchmark workload), whole diagram
    xy = synth.workload("uniform_1m")
    d = gpu(xy, BOX, collect_stats=1)
    r = oracle.cells(xy, BOX, "bucketed")
    assert r["stats"][:, 5].sum() == 0, "general position"
    assert_full_parity(d, r)
    delaunay_symmetric_ok(d, xy.shape[0])


def test_host_entry_point_matches_device_entry_point():
    xy = synth.uniform_sites(20000, seed=99)
    a = gpu(xy, BOX)
    b = to_numpy(vg.build_host(xy, BOX))
    for key in ("cell_ptr", "labels", "vx", "vy", "delaunay"):
        assert np.array_equal(a[key], b[key]), key


def _hub_rows(cx, cy, d, m):
    """m sites on four rows around the hub (cx, cy), each row at distance d
    from it and its sites within 0.4 d of the row's foot: the bisectors of
    the hub with the sites of a row all touch one parabola (focus the hub),
    so every site of every row carries an edge of the hub's cell, which has
    exactly m edges."""
    k = m // 4
    step = max(1, int(0.8 * d) // k)
    t = np.round((np.arange(k) - (k - 1) / 2.0) * step).astype(np.int64)
    rows = [np.stack([t, np.full(k, -d)], 1), np.stack([np.full(k, d), t], 1),
            np.stack([-t, np.full(k, d)], 1), np.stack([np.full(k, -d), -t], 1)]
    return np.concatenate(rows) + np.array([cx, cy])


@pytest.mark.parametrize("m", [1000, 5000])
def test_hub_cells_with_thousands_of_edges(m):
    # one cell with m edges: beyond the shared-memory capacities of the
    # block-per-cell tier for m = 5000 (its global-memory mode), within them
    # for m = 1000; the oracle has no size limit and neither has the library
    u = synth.uniform_sites(3000, seed=m)
    u = u[np.maximum(np.abs(u[:, 0] - 500000), np.abs(u[:, 1] - 500000)) > 25000]
    xy = np.concatenate([[[500000, 500000]], _hub_rows(500000, 500000, 10000, m), u]).astype(np.int32)
    r = oracle.cells(xy, BOX, "bucketed", beta=1)
    assert np.diff(r["cell_ptr"])[0] == m
    d = gpu(xy, BOX, collect_stats=1)
    assert_full_parity(d, r)
    # and inside a batch, next to an ordinary set
    u = synth.uniform_sites(2000, seed=7)
    ptr = np.array([0, xy.shape[0], xy.shape[0] + u.shape[0]], np.int64)
    B = vg.build_batch(torch.from_numpy(np.concatenate([xy, u])).cuda(), ptr,
                       np.full((2, 2), BOX, np.int32))
    assert_full_parity(to_numpy(B.set(0)), r)
    assert_full_parity(to_numpy(B.set(1)), oracle.cells(u, BOX, "plain"))


def test_shared_vertices_are_identical():
    # a vertex shared by two or three cells has identical float64
    # coordinates in every cell (uniform and clustered sites, and sites on a
    # lattice, where four cells meet at every lattice vertex and the owner's
    # list may not hold the pair)
    for xy, box in ((synth.uniform_sites(50000, seed=11), BOX),
                    (synth.gaussian_mixture_sites(50000, seed=12, sigma=3000.0), BOX),
                    (synth.lattice_sites(30, 1000, 500), 30000)):
        # every cell computes a vertex from its owner's lines (the default),
        # or the owner computes it once and the others copy it
        d0 = gpu(xy, box)
        d1 = gpu(xy, box, share_vertices=1)
        for d in (d0, d1):
            assert_shared_vertices_identical(d)
        for key in ("cell_ptr", "labels", "vx", "vy", "delaunay"):
            assert np.array_equal(d0[key], d1[key]), key
        if xy.shape[0] <= 1000:
            assert_full_parity(d0, oracle.cells(xy, box, "plain"))
