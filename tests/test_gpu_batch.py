"""GPU parity of batch builds: many independent sets in one build.

Every set of a batch must come out bit-identical to the oracle's diagram of
that set alone (labels local to the set), and to a single build of the set.
"""

import numpy as np
import pytest

import oracle
import synth
from parity import assert_full_parity, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1212_1095_gb300 as vg  # noqa: E402


def _mixed_sets():
    """Sets of ragged sizes (empty, one site, tiny, medium, clustered) in
    boxes of different shapes; set 5 repeats the sites of set 3 (equal
    sites in different sets are not duplicates)."""
    sets, boxes = [], []

    def add(xy, box):
        sets.append(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
        boxes.append(box)

    add(synth.uniform_sites(1, seed=901, box=64), (64, 64))
    add(np.zeros((0, 2), np.int32), (100, 100))
    add(synth.uniform_sites(2, seed=902, box=1000), (1000, 1000))
    add(synth.uniform_sites(300, seed=903, box=4096), (4096, 4096))
    add(synth.lattice_sites(6, 30, 15), (180, 180))
    add(sets[3], (4096, 4096))
    xy = synth.uniform_sites(500, seed=904, box=900)
    add(xy, (900, 5000))                                     # a tall box
    add(synth.gaussian_mixture_sites(3000, seed=905), (1 << 20, 1 << 20))
    add(np.zeros((0, 2), np.int32), (2, 2))
    add(synth.uniform_sites(7000, seed=906), (1 << 20, 1 << 20))
    add(synth.uniform_sites(3, seed=907, box=8), (8, 8))
    return sets, boxes


def _pack(sets, boxes):
    ptr = np.zeros(len(sets) + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([s.shape[0] for s in sets])
    xy = np.concatenate(sets).astype(np.int32) if ptr[-1] > 0 else np.zeros((0, 2), np.int32)
    return xy, ptr, np.asarray(boxes, dtype=np.int32)


def _oracle(xy, box):
    mode = "plain" if xy.shape[0] <= 2000 else "bucketed"
    return oracle.cells(xy, box, mode)


def test_batch_sets_match_oracle_and_single_builds():
    sets, boxes = _mixed_sets()
    xy, ptr, bx = _pack(sets, boxes)
    B = vg.build_batch(torch.from_numpy(xy).cuda(), ptr, bx)
    for j, (s, box) in enumerate(zip(sets, boxes)):
        d = to_numpy(B.set(j))
        if s.shape[0] == 0:
            assert d["cell_ptr"].tolist() == [0] and d["labels"].size == 0
            assert d["delaunay"].shape[0] == 0
            continue
        assert_full_parity(d, _oracle(s, box))
        single = to_numpy(vg.build(torch.from_numpy(s).cuda(), box))
        for key in ("cell_ptr", "labels", "vx", "vy", "delaunay"):
            assert np.array_equal(d[key], single[key]), (j, key)


@pytest.mark.parametrize("opts", [dict(lanes_per_cell=8), dict(bucket_side=3000),
                                  dict(exact_only=1), dict(target=10)])
def test_batch_options(opts):
    sets, boxes = _mixed_sets()
    keep = [3, 4, 6, 7, 9]
    sets = [sets[j] for j in keep]
    boxes = [boxes[j] for j in keep]
    xy, ptr, bx = _pack(sets, boxes)
    B = vg.build_batch(torch.from_numpy(xy).cuda(), ptr, bx, **opts)
    for j, (s, box) in enumerate(zip(sets, boxes)):
        assert_full_parity(to_numpy(B.set(j)), _oracle(s, box))


def test_batch_of_generated_sets_sampled():
    # a slice of the batched workload: log-uniform sizes, uniform and clustered
    xy, ptr = synth.batch_sets(n_sets=24, lo=16, hi=4096)
    bx = np.full((24, 2), synth.WORLD, dtype=np.int32)
    B = vg.build_batch(torch.from_numpy(xy).cuda(), ptr, bx)
    for j in range(24):
        s = xy[ptr[j]:ptr[j + 1]]
        assert_full_parity(to_numpy(B.set(j)), _oracle(s, synth.WORLD))


def test_batch_all_empty():
    ptr = np.zeros(4, dtype=np.int64)
    bx = np.full((3, 2), 100, dtype=np.int32)
    B = vg.build_batch(torch.zeros((0, 2), dtype=torch.int32, device="cuda"), ptr, bx)
    assert B.labels.numel() == 0 and B.delaunay.shape[0] == 0
    assert B.cell_ptr[:1].cpu().tolist() == [0]
    assert B.del_set_ptr.cpu().tolist() == [0, 0, 0, 0]


def test_batch_errors_fail_the_batch():
    sets = [synth.uniform_sites(50, seed=911, box=1000), synth.uniform_sites(50, seed=912, box=1000)]
    # a site of set 1 lies outside set 1's (smaller) box
    xy, ptr, bx = _pack(sets, [(1000, 1000), (500, 500)])
    with pytest.raises(vg.VorError) as e:
        vg.build_batch(torch.from_numpy(xy).cuda(), ptr, bx)
    assert e.value.code == -2
    # a duplicate inside set 0
    s0 = sets[0].copy()
    s0[7] = s0[3]
    xy, ptr, bx = _pack([s0, sets[1]], [(1000, 1000), (1000, 1000)])
    with pytest.raises(vg.VorError) as e:
        vg.build_batch(torch.from_numpy(xy).cuda(), ptr, bx)
    assert e.value.code == -3


def test_batch_device_offsets_must_match_host():
    sets = [synth.uniform_sites(40, seed=913, box=1000), synth.uniform_sites(60, seed=914, box=1000)]
    xy, ptr, bx = _pack(sets, [(1000, 1000), (1000, 1000)])
    ws = vg.BatchWorkspace(ptr, bx, vg.vor_opts_default())
    ws.d_set_ptr[-1] = int(ptr[-1]) - 1          # device total differs from the host's
    ws.launch(torch.from_numpy(xy).cuda())
    with pytest.raises(vg.VorError) as e:
        ws.finish()
    assert e.value.code == -1
    ws.d_set_ptr.copy_(torch.from_numpy(ptr))
    ws.launch(torch.from_numpy(xy).cuda())
    B = ws.finish()
    for j, s in enumerate(sets):
        assert_full_parity(to_numpy(B.set(j)), _oracle(s, 1000))


def test_batch_graph_capture_and_replay():
    xy, ptr = synth.batch_sets(n_sets=12, lo=16, hi=2048, seed=synth.SEED_BASE + 40)
    bx = np.full((12, 2), synth.WORLD, dtype=np.int32)
    # a second input of the same set sizes: each set mirrored in x
    xy2 = xy.copy()
    xy2[:, 0] = synth.WORLD - xy[:, 0]
    ws = vg.BatchWorkspace(ptr, bx, vg.vor_opts_default())
    buf = torch.from_numpy(xy).cuda()
    ws.launch(buf)                                  # warm-up outside the capture
    ws.finish()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ws.launch(buf)
    for inp in (xy2, xy):
        buf.copy_(torch.from_numpy(inp))
        g.replay()
        B = ws.finish()
        for j in range(12):
            s = inp[ptr[j]:ptr[j + 1]]
            assert_full_parity(to_numpy(B.set(j)), _oracle(s, synth.WORLD))


def test_bucket_load_option_keeps_results():
    sets, boxes = _mixed_sets()
    keep = [3, 6, 7, 9]
    sets = [sets[j] for j in keep]
    boxes = [boxes[j] for j in keep]
    xy, ptr, bx = _pack(sets, boxes)
    ref = None
    for load in (25, 100, 400, 1600):
        B = vg.build_batch(torch.from_numpy(xy).cuda(), ptr, bx, bucket_load_pct=load)
        got = [to_numpy(B.set(j)) for j in range(len(sets))]
        if ref is None:
            ref = got
            for j, (s, box) in enumerate(zip(sets, boxes)):
                assert_full_parity(got[j], _oracle(s, box))
        else:
            for a, b in zip(ref, got):
                for key in a:
                    assert np.array_equal(a[key], b[key])


def test_autotune_returns_the_fastest_valid_candidate():
    xy, ptr = synth.batch_sets(n_sets=32, lo=16, hi=4096, seed=synth.SEED_BASE + 41)
    bx = np.full((32, 2), synth.WORLD, dtype=np.int32)
    cands = [vg.vor_opts_default(), vg.vor_opts_default(lanes_per_cell=8, target=16),
             vg.vor_opts_default(bucket_load_pct=400)]
    best, table = vg.autotune_batch(torch.from_numpy(xy).cuda(), ptr, bx, candidates=cands, reps=1)
    ms = [m for _, m in table]
    assert all(np.isfinite(ms))
    assert best.as_dict() == cands[int(np.argmin(ms))].as_dict()
    B = vg.build_batch(torch.from_numpy(xy).cuda(), ptr, bx, **{
        k: v for k, v in best.as_dict().items() if k in ("lanes_per_cell", "target",
                                                          "bucket_load_pct")})
    for j in range(32):
        assert_full_parity(to_numpy(B.set(j)), _oracle(xy[ptr[j]:ptr[j + 1]], synth.WORLD))
