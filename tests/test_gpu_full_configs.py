"""GPU parity on the whole of the full-size clustered workloads.

Every cell of the 4,194,304-site Gaussian-mixture build, every set of the
4,096-set batch and every request of a 200-request served Poisson stream is
compared with the exact oracle: the combinatorial output (edge counts,
canonical edge labels, Delaunay pairs) through the digests that
tests/golden/make_digests.py stored from the oracle (bit-exact), and the
float64 vertices against the meeting point of their two lines, computed
exactly from the verified labels (1e-9 relative).  When an input differs from
the one a digest was made for (another platform's floating-point library in
the Gaussian generator), the oracle is run here instead.

The cells the oracle marks degenerate in the 4M build (a vertex with more
than three equidistant sites: co-circular sites are allowed there) are also
compared one by one with the oracle, and counted.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth
from parity import (assert_full_parity, assert_sampled_parity, assert_vertices_from_labels,
                    cells_digest, chunk_digests, delaunay_symmetric_ok, input_digest, to_numpy)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1212_1095_gb300 as vg  # noqa: E402

BOX = synth.WORLD
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _oracle(xy, **kw):
    # the digests' oracle configuration (Method A.6, beta = 1)
    return oracle.cells(xy, BOX, "bucketed", beta=1, **kw)


def _areas(d):
    cp, vx, vy = d["cell_ptr"], d["vx"], d["vy"]
    nxt = np.arange(len(vx)) + 1
    nxt[cp[1:] - 1] = cp[:-1]                      # each cell's last vertex wraps to its first
    cross = vx * vy[nxt] - vx[nxt] * vy
    return np.add.reduceat(cross, cp[:-1]) / 2.0


def _first_bad_cells(d, xy, lo, hi, count=64):
    """Oracle comparison of the first cells of a chunk whose digest differs
    (for a readable failure message)."""
    sel = np.arange(lo, min(hi, lo + count))
    assert_sampled_parity(d, _oracle(xy, sel=sel), sel)


@pytest.fixture(scope="module")
def gauss_4m():
    xy = synth.workload("gauss_4m")
    d = to_numpy(vg.build(torch.from_numpy(xy).cuda(), BOX, collect_stats=1))
    return xy, d


def test_gauss_4m_whole_diagram_parity(gauss_4m):
    xy, d = gauss_4m
    n = xy.shape[0]
    g = _golden("gauss_4m.json")
    if input_digest(xy) != g["input_sha256"]:
        assert_full_parity(d, _oracle(xy))
    else:
        assert d["labels"].shape[0] == g["n_edges"] and d["delaunay"].shape[0] == g["n_del"]
        got = chunk_digests(d["cell_ptr"], d["labels"], d["delaunay"], n, g["chunk"])
        bad = [c for c, (a, b) in enumerate(zip(got, g["chunks"])) if a != b]
        if bad:
            lo = bad[0] * g["chunk"]
            _first_bad_cells(d, xy, lo, lo + g["chunk"])
        assert not bad, f"{len(bad)} of {len(got)} chunks differ from the oracle, first {bad[:8]}"
        assert_vertices_from_labels(xy, BOX, d)
    # whole-diagram properties
    assert np.diff(d["cell_ptr"]).min() >= 3
    area = _areas(d)
    assert np.all(area > 0)
    assert abs(area.sum() - float(BOX) * BOX) <= 1e-8 * float(BOX) * BOX
    delaunay_symmetric_ok(d, n)


def test_gauss_4m_degenerate_cells(gauss_4m):
    xy, d = gauss_4m
    g = _golden("gauss_4m.json")
    deg = np.array(g["degenerate_cells"], dtype=np.int64)
    if input_digest(xy) != g["input_sha256"]:
        st = _oracle(xy)["stats"]
        deg = np.nonzero(st[:, 5] > 0)[0]
    print(f"gauss_4m: {deg.shape[0]} cells with a degenerate vertex (4+ equidistant sites)")
    assert deg.shape[0] > 0, "the clustered workload keeps co-circular sites"
    assert_sampled_parity(d, _oracle(xy, sel=deg), deg)


def test_batch_4096_every_set():
    xy, ptr = synth.batch_workload()
    S = ptr.shape[0] - 1
    g = _golden("batch_4096.json")
    same_input = (input_digest(xy) == g["input_sha256"]
                  and input_digest(ptr.astype(np.int32)) == g["set_ptr_sha256"])
    bx = np.full((S, 2), BOX, np.int32)
    B = vg.build_batch(torch.from_numpy(xy).cuda(), ptr, bx)
    cp = B.cell_ptr.cpu().numpy()
    lab = B.labels.cpu().numpy()
    vx, vy = B.vx.cpu().numpy(), B.vy.cpu().numpy()
    dl = B.delaunay.cpu().numpy().reshape(-1, 2)
    dsp = B.del_set_ptr.cpu().numpy()
    bad = []
    for j in range(S):
        a, b = int(ptr[j]), int(ptr[j + 1])
        e0, e1 = int(cp[a]), int(cp[b])
        d = {"cell_ptr": cp[a:b + 1] - e0, "labels": lab[e0:e1], "vx": vx[e0:e1], "vy": vy[e0:e1],
             "delaunay": dl[dsp[j]:dsp[j + 1]]}
        s = xy[a:b]
        if not same_input:
            assert_full_parity(d, _oracle(s))
            continue
        if cells_digest(d["cell_ptr"], d["labels"], d["delaunay"], 0, b - a) != g["sets"][j]:
            bad.append(j)
            if len(bad) == 1:
                assert_full_parity(d, _oracle(s))
        assert_vertices_from_labels(s, BOX, d)
    assert not bad, f"{len(bad)} of {S} sets differ from the oracle: {bad[:16]}"


def test_served_poisson_stream_every_request():
    from golden import make_digests
    g = _golden("serve_stream.json")
    sizes, kinds, reqs = make_digests.serve_stream_requests()
    assert [int(s) for s in sizes] == g["sizes"] and [int(k) for k in kinds] == g["kinds"]
    # Poisson arrivals at 400 requests/s (the sizes and kinds do not depend
    # on the rate); results are read as they complete
    import threading
    import time
    arrivals, _, _ = synth.poisson_requests(len(reqs), 400.0, seed=make_digests.SERVE_SEED)
    tickets = [None] * len(reqs)
    with vg.Server(device_bytes=24 << 30, host_bytes=8 << 30, max_inflight=4,
                   max_wave_requests=64, max_wave_sites=8 << 20) as srv:
        t0 = time.perf_counter()

        def submitter():
            for j, xy in enumerate(reqs):
                dt = t0 + arrivals[j] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets[j] = srv.submit(xy, BOX, timeout=600.0)

        th = threading.Thread(target=submitter)
        th.start()
        bad, waves = [], []
        for j, xy in enumerate(reqs):
            while tickets[j] is None:
                time.sleep(0.0005)
            r = srv.wait(tickets[j], timeout=600.0)
            assert r["status"] == 0, vg.vor_strerror(r["status"])
            waves.append(r["wave_requests"])
            if input_digest(xy)[:32] != g["inputs"][j]:
                assert_full_parity(r, _oracle(xy))
                continue
            if cells_digest(r["cell_ptr"], r["labels"], r["delaunay"], 0, xy.shape[0]) != g["requests"][j]:
                bad.append(j)
                if len(bad) == 1:
                    assert_full_parity(r, _oracle(xy))
            assert_vertices_from_labels(xy, BOX, r)
        th.join()
    assert max(waves) > 1, "requests shared waves (continuous batching)"
    assert not bad, f"{len(bad)} of {len(reqs)} requests differ from the oracle: {bad[:16]}"


def test_large_clustered_request_with_many_large_cells():
    # request 842 of the saturated serving stream: 963,722 clustered sites
    # (a slice of the Gaussian-mixture pool); its cluster-hull cells reach the
    # large-cell tiers, whose row scan once read overlapping ranges twice
    pools = synth.serve_pools()
    seed = synth.SEED_BASE + 51
    _, sizes, kinds = synth.poisson_requests(2000, 100.0, seed=seed)
    xy = synth.serve_request(842 + seed * 100000, sizes[842], kinds[842], pools)
    n = xy.shape[0]
    d = to_numpy(vg.build(torch.from_numpy(xy).cuda(), BOX))
    cp = d["cell_ptr"]
    e = np.diff(cp)
    rng = np.random.default_rng(842)
    k = np.nonzero((xy[:, 0] == 705893) & (xy[:, 1] == 388283))[0]
    sel = np.unique(np.concatenate([rng.choice(n, 2000, replace=False), k, np.argsort(-e)[:300]]))
    assert_sampled_parity(d, _oracle(xy, sel=sel), sel)
    assert_vertices_from_labels(xy, BOX, d)
    area = _areas(d)
    assert abs(area.sum() - float(BOX) * BOX) <= 1e-8 * float(BOX) * BOX
