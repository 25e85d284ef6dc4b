"""GPU parity at the full sizes of the clustered and batched workloads.

The clustered 4,194,304-site build is compared with the exact oracle on a
sample of cells (random ones, the hull cells at the extreme coordinates,
and the cells with the most edges or the widest extent in the GPU output,
chosen only as a sample) and checked as a whole against properties that
hold at any size.  The batch of 4,096 sets is compared set by set on a
sample of sets spanning the size range.
"""

import numpy as np
import pytest

import oracle
import synth
from parity import assert_full_parity, assert_sampled_parity, delaunay_symmetric_ok, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1212_1095_gb300 as vg  # noqa: E402

BOX = synth.WORLD


def _cell_extents(d):
    """Per cell: number of edges and the larger side of its vertex bounding box."""
    cp, vx, vy = d["cell_ptr"], d["vx"], d["vy"]
    e = np.diff(cp)
    idx = np.repeat(np.arange(len(e)), e)
    xmin = np.full(len(e), np.inf)
    xmax = np.full(len(e), -np.inf)
    ymin = np.full(len(e), np.inf)
    ymax = np.full(len(e), -np.inf)
    np.minimum.at(xmin, idx, vx)
    np.maximum.at(xmax, idx, vx)
    np.minimum.at(ymin, idx, vy)
    np.maximum.at(ymax, idx, vy)
    return e, np.maximum(xmax - xmin, ymax - ymin)


def _areas(d):
    cp, vx, vy = d["cell_ptr"], d["vx"], d["vy"]
    nxt = np.arange(len(vx)) + 1
    nxt[cp[1:] - 1] = cp[:-1]                      # each cell's last vertex wraps to its first
    cross = vx * vy[nxt] - vx[nxt] * vy
    return np.add.reduceat(cross, cp[:-1]) / 2.0


def test_gauss_4m_sampled_parity_and_invariants():
    xy = synth.workload("gauss_4m")
    n = xy.shape[0]
    d = to_numpy(vg.build(torch.from_numpy(xy).cuda(), BOX))
    # sample: random cells, extreme-coordinate hull cells, most edges, widest
    e, ext = _cell_extents(d)
    rng = np.random.default_rng(1212)
    parts = [rng.choice(n, 3000, replace=False),
             np.argsort(xy[:, 0])[:25], np.argsort(-xy[:, 0])[:25],
             np.argsort(xy[:, 1])[:25], np.argsort(-xy[:, 1])[:25],
             np.argsort(-e)[:100], np.argsort(-ext)[:200]]
    sel = np.unique(np.concatenate(parts))
    assert_sampled_parity(d, oracle.cells(xy, BOX, "bucketed", sel=sel), sel)
    # whole-diagram properties
    assert e.min() >= 3
    area = _areas(d)
    assert np.all(area > 0)
    assert abs(area.sum() - float(BOX) * BOX) <= 1e-8 * float(BOX) * BOX
    delaunay_symmetric_ok(d, n)
    # each Delaunay pair appears as a neighbour label in both cells
    lab = d["labels"]
    owner = np.repeat(np.arange(n), e)
    nb = lab >= 0
    pairs = np.stack([np.minimum(owner[nb], lab[nb]), np.maximum(owner[nb], lab[nb])], 1)
    key = np.unique(pairs[:, 0].astype(np.int64) * n + pairs[:, 1])
    dk = d["delaunay"][:, 0].astype(np.int64) * n + d["delaunay"][:, 1]
    assert np.array_equal(key, dk)
    # and every such pair was listed from both sides (2 labels per pair)
    assert nb.sum() == 2 * dk.size


def test_batch_4096_sampled_sets():
    xy, ptr = synth.batch_workload()
    S = ptr.shape[0] - 1
    bx = np.full((S, 2), BOX, np.int32)
    B = vg.build_batch(torch.from_numpy(xy).cuda(), ptr, bx)
    sizes = np.diff(ptr)
    order = np.argsort(sizes)
    # sets across the size range (both kinds), the largest of each kind
    pick = list(order[np.linspace(0, S - 1, 14).astype(int)])
    pick += [int(order[np.nonzero(order % 2 == 0)[0][-1]]), int(order[np.nonzero(order % 2 == 1)[0][-1]])]
    for j in sorted(set(int(p) for p in pick)):
        s = xy[ptr[j]:ptr[j + 1]]
        mode = "plain" if s.shape[0] <= 2000 else "bucketed"
        assert_full_parity(to_numpy(B.set(j)), oracle.cells(s, BOX, mode))


def test_large_clustered_request_with_many_large_cells():
    # request 842 of the saturated serving stream: 963,722 clustered sites
    # (a slice of the Gaussian-mixture pool); its cluster-hull cells reach the
    # large tier, whose row scan once read overlapping ranges twice
    pools = synth.serve_pools()
    seed = synth.SEED_BASE + 51
    _, sizes, kinds = synth.poisson_requests(2000, 100.0, seed=seed)
    xy = synth.serve_request(842 + seed * 100000, sizes[842], kinds[842], pools)
    n = xy.shape[0]
    d = to_numpy(vg.build(torch.from_numpy(xy).cuda(), BOX))
    e, ext = _cell_extents(d)
    rng = np.random.default_rng(842)
    k = np.nonzero((xy[:, 0] == 705893) & (xy[:, 1] == 388283))[0]
    sel = np.unique(np.concatenate([rng.choice(n, 2000, replace=False), k,
                                    np.argsort(-ext)[:300], np.argsort(-e)[:50]]))
    assert_sampled_parity(d, oracle.cells(xy, BOX, "bucketed", sel=sel), sel)
    area = _areas(d)
    assert abs(area.sum() - float(BOX) * BOX) <= 1e-8 * float(BOX) * BOX
