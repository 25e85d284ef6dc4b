"""GPU tests of the request server (continuous batching).

Each result must be the same alone and in the mix: a request's diagram from
the server equals the single build of its sites, bit for bit, whatever wave
it ran in.  Errors stay with the request that caused them; memory budgets
bound admission; injected host-side failures and cancellations leave no
memory behind.
"""

import numpy as np
import pytest

import oracle
import synth
from parity import assert_full_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1212_1095_gb300 as vg  # noqa: E402

BOX = synth.WORLD
KEYS = ("cell_ptr", "labels", "vx", "vy", "delaunay")


def _single(xy, box):
    d = vg.build(torch.from_numpy(np.ascontiguousarray(xy, np.int32)).cuda(), box)
    return {"cell_ptr": d.cell_ptr.cpu().numpy(), "labels": d.labels.cpu().numpy(),
            "vx": d.vx.cpu().numpy(), "vy": d.vy.cpu().numpy(),
            "delaunay": d.delaunay.cpu().numpy().reshape(-1, 2)}


def _requests(count, seed, hi=20000):
    """Uniform and clustered requests of log-uniform size, some in small boxes."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(np.exp(rng.uniform(np.log(20), np.log(hi))))
        if q % 5 == 4:
            box = 4096
            xy = synth.uniform_sites(min(n, 2000), seed=seed * 1000 + q, box=box)
        elif q % 2:
            box = BOX
            xy = synth.gaussian_mixture_sites(n, seed=seed * 1000 + q)
        else:
            box = BOX
            xy = synth.uniform_sites(n, seed=seed * 1000 + q)
        out.append((xy, box))
    return out


def _same(res, ref):
    assert res["status"] == 0
    for k in KEYS:
        assert np.array_equal(res[k], ref[k]), k


def test_results_are_the_same_alone_and_in_the_mix():
    reqs = _requests(24, seed=71)
    with vg.Server(device_bytes=4 << 30, host_bytes=1 << 30, max_inflight=3,
                   max_wave_requests=8) as srv:
        # a large request first keeps the GPU busy while the rest queue up
        # and are batched
        head = synth.uniform_sites(400000, seed=72)
        tickets = [srv.submit(head, BOX)] + [srv.submit(xy, box) for xy, box in reqs]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == 25 and st["failed"] == 0
    assert st["max_wave_requests_seen"] > 1              # requests did share waves
    _same(results[0], _single(head, BOX))
    for (xy, box), r in zip(reqs, results[1:]):
        _same(r, _single(xy, box))
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]
    # and against the oracle for the small ones
    for (xy, box), r in list(zip(reqs, results[1:]))[:6]:
        if xy.shape[0] <= 3000:
            assert_full_parity(r, oracle.cells(xy, box, "plain"))


def test_a_faulty_request_fails_alone():
    reqs = _requests(10, seed=73, hi=3000)
    bad = synth.uniform_sites(100, seed=74, box=5000)     # sites up to 4999 ...
    with vg.Server(device_bytes=2 << 30, host_bytes=1 << 30, max_inflight=2,
                   max_wave_requests=16) as srv:
        head = synth.uniform_sites(300000, seed=75)
        t0 = srv.submit(head, BOX)
        ts = [srv.submit(xy, box) for xy, box in reqs[:5]]
        tb = srv.submit(bad, 1000)                         # ... in a 1000-wide box
        ts += [srv.submit(xy, box) for xy, box in reqs[5:]]
        assert srv.wait(t0)["status"] == 0
        rb = srv.wait(tb)
        assert rb["status"] == -2                          # VOR_E_SITE_OUTSIDE
        for (xy, box), t in zip(reqs, ts):
            _same(srv.wait(t), _single(xy, box))
        st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 11


def test_admission_under_a_small_budget():
    o = vg.vor_opts_default()
    one = vg.vor_workspace_bytes(50000, BOX, o)
    budget = 3 * one + (64 << 20)                          # room for about two requests
    reqs = [(synth.uniform_sites(50000, seed=80 + q), BOX) for q in range(8)]
    with vg.Server(device_bytes=budget, host_bytes=512 << 20, max_inflight=4,
                   max_wave_requests=8) as srv:
        with pytest.raises(vg.VorError) as e:              # alone larger than the budget
            srv.submit(synth.uniform_sites(400000, seed=90), BOX)
        assert e.value.code == vg.E_SERVER_FULL
        ts = [srv.submit(xy, box) for xy, box in reqs]
        for (xy, box), t in zip(reqs, ts):
            _same(srv.wait(t), _single(xy, box))
        st = srv.stats()
        assert st["device_free"] == budget and st["device_largest_free"] == budget
    assert st["completed"] == 8


def test_injected_host_allocation_failure_and_cancel_leave_no_memory_behind():
    reqs = _requests(6, seed=91, hi=5000)
    host = 256 << 20
    with vg.Server(device_bytes=1 << 30, host_bytes=host, max_inflight=1, max_wave_requests=1,
                   fail_host_alloc_at=2) as srv:
        head = synth.uniform_sites(300000, seed=92)
        t0 = srv.submit(head, BOX)
        ts = [srv.submit(xy, box) for xy, box in reqs]
        srv.cancel(ts[3])                                  # still waiting: dropped at once
        out = [srv.wait(t) for t in [t0] + ts]
        assert out[0]["status"] == 0
        assert out[1]["status"] == -5                      # the injected failure (VOR_E_OOM)
        assert out[4]["status"] == vg.E_CANCELLED
        for j in (2, 3, 5, 6):
            xy, box = reqs[j - 1]
            _same(out[j], _single(xy, box))
        st = srv.stats()
        assert st["pending"] == 0 and st["inflight"] == 0
        assert st["host_free"] == host and st["device_free"] == 1 << 30
        assert st["failed"] == 1 and st["cancelled"] == 1


def test_poll_and_timeouts():
    with vg.Server(device_bytes=1 << 30, host_bytes=256 << 20) as srv:
        xy = synth.uniform_sites(1000, seed=95)
        t = srv.submit(xy, BOX)
        r = None
        for _ in range(100000):
            r = srv.poll(t, keep=True)
            if r is not None:
                break
        r = srv.wait(t)
        _same(r, _single(xy, BOX))
        with pytest.raises(vg.VorError):
            srv.wait(t)                                    # released: unknown ticket
        e = srv.submit(np.zeros((0, 2), np.int32), BOX)    # an empty request
        r = srv.wait(e)
        assert r["status"] == 0 and r["cell_ptr"].tolist() == [0] and r["labels"].size == 0
