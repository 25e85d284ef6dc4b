"""The allocation-free build entry point, vor_build_noalloc.

Some callers cannot allocate device memory when they need a diagram (a
plug-in inside a host application whose framework owns the device memory
pool, or a real-time deployment that forbids device allocation after
start-up).  vor_build_noalloc builds with a static scratch array inside the
library instead of a caller-provided workspace.  These tests call it through
the C ABI and check its output against the regular entry point
(vor_build_async with its own workspace) on two calls in a row, so a call
that finds the previous call's contents in the shared scratch is covered.

The file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1212_1095_gb300 as vg  # noqa: E402

BOX = 1 << 20
VERTEX_RTOL = 1e-9


def _outputs(n, dev):
    ec, dc = vg.vor_edge_capacity(n), vg.vor_delaunay_capacity(n)
    bufs = {
        "cell_ptr": torch.empty(n + 1, dtype=torch.int64, device=dev),
        "labels": torch.empty(ec, dtype=torch.int32, device=dev),
        "vx": torch.empty(ec, dtype=torch.float64, device=dev),
        "vy": torch.empty(ec, dtype=torch.float64, device=dev),
        "del": torch.empty((dc, 2), dtype=torch.int32, device=dev),
        "totals": torch.zeros(2, dtype=torch.int64, device=dev),
    }
    out = vg.VorOut(bufs["cell_ptr"].data_ptr(), bufs["labels"].data_ptr(), bufs["vx"].data_ptr(),
                    bufs["vy"].data_ptr(), bufs["del"].data_ptr(), bufs["totals"].data_ptr(),
                    ec, dc)
    return bufs, out


def _call(sites, n, out):
    lib = vg.library()
    opts = vg.vor_opts_default()
    stream = torch.cuda.current_stream()
    rc = lib.vor_build_noalloc(ctypes.c_void_p(sites.data_ptr()), n, vg.VorBox(BOX, BOX),
                               ctypes.byref(opts), ctypes.byref(out),
                               ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, vg.vor_strerror(rc)


def _noalloc(xy):
    """One call of vor_build_noalloc through the C ABI; returns host arrays."""
    dev = torch.device("cuda", torch.cuda.current_device())
    sites = torch.from_numpy(np.ascontiguousarray(xy, dtype=np.int32)).to(dev)
    n = xy.shape[0]
    bufs, out = _outputs(n, dev)
    _call(sites, n, out)
    ne, nd = (int(v) for v in bufs["totals"].cpu())
    return {"cell_ptr": bufs["cell_ptr"].cpu().numpy(), "labels": bufs["labels"][:ne].cpu().numpy(),
            "vx": bufs["vx"][:ne].cpu().numpy(), "vy": bufs["vy"][:ne].cpu().numpy(),
            "delaunay": bufs["del"][:nd].cpu().numpy()}


def _regular(xy):
    d = vg.build(torch.from_numpy(np.ascontiguousarray(xy, dtype=np.int32)).cuda(), BOX)
    return {"cell_ptr": d.cell_ptr.cpu().numpy(), "labels": d.labels.cpu().numpy(),
            "vx": d.vx.cpu().numpy(), "vy": d.vy.cpu().numpy(),
            "delaunay": d.delaunay.cpu().numpy()}


def _same(a, b):
    for key in ("cell_ptr", "labels", "delaunay"):
        assert np.array_equal(a[key], b[key]), key
    for key in ("vx", "vy"):
        assert np.all(np.abs(a[key] - b[key]) <= VERTEX_RTOL * np.maximum(np.abs(b[key]), 1.0)), key


def test_noalloc_matches_regular_entry_point_on_two_calls():
    # the second call reuses the scratch the first call left behind
    first = synth.uniform_sites(80000, seed=31)
    second = synth.gaussian_mixture_sites(40000, seed=32, sigma=3000.0)
    for xy in (first, second):
        _same(_noalloc(xy), _regular(xy))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = vg.library()
    opts = vg.vor_opts_default()
    n = 1 << 20
    assert vg.vor_workspace_bytes(n, BOX, opts) > (64 << 20)
    out = vg.VorOut()
    rc = lib.vor_build_noalloc(ctypes.c_void_p(0), n, vg.VorBox(BOX, BOX), ctypes.byref(opts),
                               ctypes.byref(out), ctypes.c_void_p(0))
    assert rc == -9


def test_noalloc_allocates_no_device_memory():
    # inputs and outputs allocated up front; after one warm-up call (which
    # may load the library's scratch array), a second call leaves the free
    # device memory exactly where it was
    dev = torch.device("cuda", torch.cuda.current_device())
    xy = synth.uniform_sites(50000, seed=33)
    sites = torch.from_numpy(xy).to(dev)
    bufs, out = _outputs(xy.shape[0], dev)
    _call(sites, xy.shape[0], out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _call(sites, xy.shape[0], out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
