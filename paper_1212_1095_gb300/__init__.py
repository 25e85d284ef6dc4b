"""GB300 projector-algorithm library: Python binding of libvor.so.

A thin ctypes binding of the C ABI declared in ``include/vor.h``.  PyTorch
provides the device memory and the stream; every step of the computation runs
in the library's CUDA kernels.  There is no CPU fallback: if the library is
missing or no GPU is present, the calls raise.

Names follow the C ABI (``vor_build_async``, ``vor_status``, ...); ``build``
and ``build_host`` are the convenience forms the tests and the benchmark use.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from ._build import SO as _SO_PATH
from ._build import build_library

__all__ = ["VorOpts", "VorStats", "VorOut", "VorError", "build_library", "library",
           "vor_opts_default", "vor_workspace_bytes", "vor_build_async", "vor_status",
           "vor_edge_capacity", "vor_delaunay_capacity", "vor_host_scratch_bytes",
           "vor_build_host", "vor_build_noalloc", "vor_strerror", "vor_stage_timing",
           "vor_stage_ms", "STAGES", "build", "build_host", "Diagram", "vor_batch_edge_capacity",
           "vor_batch_delaunay_capacity", "vor_batch_workspace_bytes", "vor_build_batch_async",
           "BatchWorkspace", "BatchDiagram", "build_batch", "vor_kernel_launches",
           "vor_autotune_grid", "autotune_batch", "Server", "VorServerConfig", "vor_vertex_quotients",
           "vor_server_config_default",
           "SIDE_BOTTOM", "SIDE_RIGHT", "SIDE_TOP", "SIDE_LEFT"]

SIDE_BOTTOM, SIDE_RIGHT, SIDE_TOP, SIDE_LEFT = -1, -2, -3, -4

ERROR_NAMES = {0: "VOR_OK", -1: "VOR_E_INVALID_ARG", -2: "VOR_E_SITE_OUTSIDE",
               -3: "VOR_E_DUPLICATE", -4: "VOR_E_BOX_TOO_LARGE", -5: "VOR_E_OOM",
               -6: "VOR_E_CAPACITY", -7: "VOR_E_CUDA", -8: "VOR_E_INTERNAL",
               -9: "VOR_E_SCRATCH_LIMIT", -10: "VOR_E_SERVER_FULL", -11: "VOR_E_TIMEOUT",
               -12: "VOR_E_CANCELLED", 1: "VOR_PENDING"}
PENDING, E_SERVER_FULL, E_TIMEOUT, E_CANCELLED = 1, -10, -11, -12


class VorError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)} ({vor_strerror(code)})")


class VorSite(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int32), ("y", ctypes.c_int32)]


class VorBox(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("h", ctypes.c_int32)]


class VorOpts(ctypes.Structure):
    _fields_ = [("bucket_side", ctypes.c_int32), ("lanes_per_cell", ctypes.c_int32),
                ("target", ctypes.c_int32), ("exact_only", ctypes.c_int32),
                ("check_duplicates", ctypes.c_int32), ("collect_stats", ctypes.c_int32),
                ("bucket_load_pct", ctypes.c_int32), ("share_vertices", ctypes.c_int32),
                ("fine_split", ctypes.c_int32), ("block_threads", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class VorStats(ctypes.Structure):
    _fields_ = [("rays", ctypes.c_uint64), ("vertex_tests", ctypes.c_uint64),
                ("evals", ctypes.c_uint64), ("exact_rays", ctypes.c_uint64),
                ("annulus_sites", ctypes.c_uint64), ("reruns", ctypes.c_uint64),
                ("deferred", ctypes.c_uint64), ("candidates", ctypes.c_uint64),
                ("max_edges", ctypes.c_uint64), ("widenings", ctypes.c_uint64),
                ("evals_first_pass", ctypes.c_uint64), ("rays_first_pass", ctypes.c_uint64),
                ("evals_second_pass", ctypes.c_uint64), ("third_pass_cells", ctypes.c_uint64),
                ("medium_cells", ctypes.c_uint64),
                ("large_cells", ctypes.c_uint64), ("global_cells", ctypes.c_uint64),
                ("divided_buckets", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_ if f != "reserved"}


class VorOut(ctypes.Structure):
    _fields_ = [("cell_ptr", ctypes.c_void_p), ("edge_label", ctypes.c_void_p),
                ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p),
                ("del_edge", ctypes.c_void_p), ("totals", ctypes.c_void_p),
                ("edge_cap", ctypes.c_int64), ("del_cap", ctypes.c_int64)]


class VorServerConfig(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_int64), ("host_bytes", ctypes.c_int64),
                ("max_inflight", ctypes.c_int32), ("max_wave_requests", ctypes.c_int32),
                ("max_wave_sites", ctypes.c_int64), ("opts", VorOpts),
                ("fail_host_alloc_at", ctypes.c_int32)]


class VorRequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("wave_requests", ctypes.c_int32),
                ("n", ctypes.c_int64), ("n_edges", ctypes.c_int64), ("n_del", ctypes.c_int64),
                ("cell_ptr", ctypes.c_void_p), ("edge_label", ctypes.c_void_p),
                ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("del_edge", ctypes.c_void_p),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class VorServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "submitted", "completed", "failed", "cancelled", "waves", "split_waves", "pending",
        "inflight", "max_wave_requests_seen", "device_free", "device_largest_free",
        "host_free")] + [("reserved", ctypes.c_int64 * 4)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_ if f != "reserved"}


_lib = None


def library():
    """Load libvor.so (building it first if the sources changed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _SO_PATH if os.path.exists(_SO_PATH) else build_library()
    lib = ctypes.CDLL(path)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.vor_opts_default.argtypes = [P]
    lib.vor_opts_default.restype = None
    lib.vor_edge_capacity.argtypes = [i64]
    lib.vor_edge_capacity.restype = i64
    lib.vor_delaunay_capacity.argtypes = [i64]
    lib.vor_delaunay_capacity.restype = i64
    lib.vor_workspace_bytes.argtypes = [i64, VorBox, P]
    lib.vor_workspace_bytes.restype = i64
    lib.vor_build_async.argtypes = [P, i64, VorBox, P, P, i64, P, P]
    lib.vor_build_async.restype = i32
    lib.vor_status.argtypes = [P, P, P]
    lib.vor_status.restype = i32
    lib.vor_host_scratch_bytes.argtypes = [i64]
    lib.vor_host_scratch_bytes.restype = i64
    lib.vor_build_host.argtypes = [P, i64, VorBox, P, P, i64, P, i64, P, P, P, P, P, i64, i64,
                                   P, P, P]
    lib.vor_build_host.restype = i32
    lib.vor_stage_timing.argtypes = [i32]
    lib.vor_stage_timing.restype = i32
    lib.vor_stage_ms.argtypes = [P, i32]
    lib.vor_stage_ms.restype = i32
    lib.vor_build_noalloc.argtypes = [P, i64, VorBox, P, P, P]
    lib.vor_build_noalloc.restype = i32
    lib.vor_batch_edge_capacity.argtypes = [i64, ctypes.c_int32]
    lib.vor_batch_edge_capacity.restype = i64
    lib.vor_batch_delaunay_capacity.argtypes = [i64, ctypes.c_int32]
    lib.vor_batch_delaunay_capacity.restype = i64
    lib.vor_batch_workspace_bytes.argtypes = [P, ctypes.c_int32, P, P]
    lib.vor_batch_workspace_bytes.restype = i64
    lib.vor_build_batch_async.argtypes = [P, P, P, ctypes.c_int32, P, P, P, P, i64, P, P, P]
    lib.vor_build_batch_async.restype = i32
    lib.vor_autotune_grid.argtypes = [P, ctypes.c_int32]
    lib.vor_autotune_grid.restype = ctypes.c_int32
    lib.vor_autotune_batch.argtypes = [P, P, P, ctypes.c_int32, P, P, P, ctypes.c_int32,
                                       ctypes.c_int32, P, i64, P, P, P, P, P]
    lib.vor_autotune_batch.restype = i32
    lib.vor_server_config_default.argtypes = [P]
    lib.vor_server_config_default.restype = None
    lib.vor_server_create.argtypes = [P, P]
    lib.vor_server_create.restype = i32
    lib.vor_server_submit.argtypes = [P, P, i64, VorBox, ctypes.c_double, P]
    lib.vor_server_submit.restype = i32
    lib.vor_server_poll.argtypes = [P, ctypes.c_uint64, P]
    lib.vor_server_poll.restype = i32
    lib.vor_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_double, P]
    lib.vor_server_wait.restype = i32
    lib.vor_server_cancel.argtypes = [P, ctypes.c_uint64]
    lib.vor_server_cancel.restype = i32
    lib.vor_server_release.argtypes = [P, ctypes.c_uint64]
    lib.vor_server_release.restype = i32
    lib.vor_server_statistics.argtypes = [P, P]
    lib.vor_server_statistics.restype = i32
    lib.vor_server_now.argtypes = [P]
    lib.vor_server_now.restype = ctypes.c_double
    lib.vor_server_destroy.argtypes = [P]
    lib.vor_server_destroy.restype = i32
    lib.vor_vertex_quotients.argtypes = [P, P, i64, P, P]
    lib.vor_vertex_quotients.restype = i32
    lib.vor_kernel_launches.argtypes = []
    lib.vor_kernel_launches.restype = i64
    lib.vor_strerror.argtypes = [i32]
    lib.vor_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


# ---------------------------------------------------------------- raw ABI ----

def vor_opts_default(**kw) -> VorOpts:
    o = VorOpts()
    library().vor_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, int(v))
    return o


def _box(box) -> VorBox:
    if isinstance(box, VorBox):
        return box
    w, h = (box, box) if isinstance(box, int) else box
    return VorBox(int(w), int(h))


def vor_edge_capacity(n: int) -> int:
    return int(library().vor_edge_capacity(int(n)))


def vor_delaunay_capacity(n: int) -> int:
    return int(library().vor_delaunay_capacity(int(n)))


def vor_workspace_bytes(n: int, box, opts: VorOpts | None = None) -> int:
    return int(library().vor_workspace_bytes(int(n), _box(box),
                                             ctypes.byref(opts) if opts is not None else None))


def vor_build_async(d_sites_ptr: int, n: int, box, opts: VorOpts, ws_ptr: int, ws_bytes: int,
                    out: VorOut, stream: int) -> int:
    return int(library().vor_build_async(ctypes.c_void_p(d_sites_ptr), int(n), _box(box),
                                         ctypes.byref(opts), ctypes.c_void_p(ws_ptr),
                                         int(ws_bytes), ctypes.byref(out),
                                         ctypes.c_void_p(stream)))


def vor_status(ws_ptr: int, stream: int) -> tuple[int, VorStats]:
    st = VorStats()
    rc = library().vor_status(ctypes.c_void_p(ws_ptr), ctypes.c_void_p(stream), ctypes.byref(st))
    return int(rc), st


def vor_host_scratch_bytes(n: int) -> int:
    return int(library().vor_host_scratch_bytes(int(n)))


def vor_vertex_quotients(num, den):
    """num / den in float64 by the library's vertex conversion (torch int64
    tensors on the GPU of equal length; den holds unsigned values < 2^44)."""
    import torch
    out = torch.empty(num.shape[0], dtype=torch.float64, device=num.device)
    rc = library().vor_vertex_quotients(ctypes.c_void_p(num.data_ptr()),
                                        ctypes.c_void_p(den.data_ptr()), int(num.shape[0]),
                                        ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise VorError(rc, "vor_vertex_quotients")
    return out


def vor_kernel_launches() -> int:
    return int(library().vor_kernel_launches())


def vor_strerror(code: int) -> str:
    try:
        return library().vor_strerror(int(code)).decode()
    except OSError:
        return "library not loaded"


def vor_stage_timing(enable: bool) -> int:
    return int(library().vor_stage_timing(1 if enable else 0))


STAGES = ("bucketing", "gather_first_pass", "projector_first_pass", "second_pass",
          "large_cells", "compaction")


def vor_stage_ms() -> list[float]:
    """Device ms of the stages (see STAGES) of the last timed build."""
    buf = (ctypes.c_float * len(STAGES))()
    k = int(library().vor_stage_ms(buf, len(STAGES)))
    if k < 0:
        raise VorError(k, "vor_stage_ms")
    return [float(buf[i]) for i in range(k)]


def vor_build_noalloc(d_sites_ptr: int, n: int, box, opts: VorOpts, out: VorOut,
                      stream: int) -> int:
    """The allocation-free build (see include/vor.h): synchronous, returns the status."""
    return int(library().vor_build_noalloc(ctypes.c_void_p(d_sites_ptr), int(n), _box(box),
                                           ctypes.byref(opts), ctypes.byref(out),
                                           ctypes.c_void_p(stream)))


def vor_build_host(*args) -> int:
    return int(library().vor_build_host(*args))


def vor_batch_edge_capacity(n_total: int, n_sets: int) -> int:
    return int(library().vor_batch_edge_capacity(int(n_total), int(n_sets)))


def vor_batch_delaunay_capacity(n_total: int, n_sets: int) -> int:
    return int(library().vor_batch_delaunay_capacity(int(n_total), int(n_sets)))


def vor_batch_workspace_bytes(set_ptr_np, boxes_np, opts: VorOpts | None = None) -> int:
    """set_ptr_np: int64 [S+1] host array; boxes_np: int32 [S, 2] host array."""
    import numpy as np
    sp = np.ascontiguousarray(set_ptr_np, dtype=np.int64)
    bx = np.ascontiguousarray(boxes_np, dtype=np.int32)
    return int(library().vor_batch_workspace_bytes(
        ctypes.c_void_p(sp.ctypes.data), int(sp.shape[0] - 1), ctypes.c_void_p(bx.ctypes.data),
        ctypes.byref(opts) if opts is not None else None))


def vor_build_batch_async(d_sites_ptr: int, d_set_ptr: int, set_ptr_np, d_boxes: int, boxes_np,
                          opts: VorOpts, ws_ptr: int, ws_bytes: int, out: VorOut,
                          d_del_set_ptr: int, stream: int) -> int:
    P = ctypes.c_void_p
    return int(library().vor_build_batch_async(
        P(d_sites_ptr), P(d_set_ptr), P(set_ptr_np.ctypes.data), int(set_ptr_np.shape[0] - 1),
        P(d_boxes), P(boxes_np.ctypes.data), ctypes.byref(opts), P(ws_ptr), int(ws_bytes),
        ctypes.byref(out), P(d_del_set_ptr), P(stream)))


# ------------------------------------------------------------ convenience ----

@dataclass
class Diagram:
    """Result of one build (device tensors unless built with build_host)."""
    cell_ptr: object      # int64 [n+1]
    labels: object        # int32 [E]
    vx: object            # float64 [E]
    vy: object            # float64 [E]
    delaunay: object      # int32 [M, 2]
    stats: dict


class Workspace:
    """Device buffers for repeated builds of up to n sites (torch allocations)."""

    def __init__(self, n: int, box, opts: VorOpts, device=None):
        import torch
        self.n, self.box, self.opts = int(n), _box(box), opts
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        nb = vor_workspace_bytes(n, self.box, opts)
        if nb < 0:
            raise VorError(-1, "vor_workspace_bytes")
        self.ws = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
        self.ws_ptr = (self.ws.data_ptr() + 255) & ~255
        self.ws_bytes = nb
        ec, dc = vor_edge_capacity(n), vor_delaunay_capacity(n)
        self.cell_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
        self.labels = torch.empty(ec, dtype=torch.int32, device=dev)
        self.vx = torch.empty(ec, dtype=torch.float64, device=dev)
        self.vy = torch.empty(ec, dtype=torch.float64, device=dev)
        self.del_edge = torch.empty((dc, 2), dtype=torch.int32, device=dev)
        self.totals = torch.zeros(2, dtype=torch.int64, device=dev)
        self.out = VorOut(self.cell_ptr.data_ptr(), self.labels.data_ptr(), self.vx.data_ptr(),
                          self.vy.data_ptr(), self.del_edge.data_ptr(), self.totals.data_ptr(),
                          ec, dc)

    def launch(self, d_sites, stream=None) -> None:
        """Enqueue a build of the sites tensor (int32 [n,2], on the device)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = vor_build_async(d_sites.data_ptr(), d_sites.shape[0], self.box, self.opts,
                             self.ws_ptr, self.ws_bytes, self.out, s.cuda_stream)
        if rc != 0:
            raise VorError(rc, "vor_build_async")

    def finish(self, stream=None) -> Diagram:
        """Wait for the build, check its status and return views of the output."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        rc, st = vor_status(self.ws_ptr, s.cuda_stream)
        if rc != 0:
            raise VorError(rc, "vor_status")
        ne, nd = (int(v) for v in self.totals.cpu())
        return Diagram(self.cell_ptr, self.labels[:ne], self.vx[:ne], self.vy[:ne],
                       self.del_edge[:nd], st.as_dict())


def build(sites, box, **opts) -> Diagram:
    """Voronoi cells and Delaunay edges of ``sites`` (torch int32 [n,2] on the GPU).

    Keyword options are the fields of ``vor_opts`` (bucket_side,
    lanes_per_cell, target, exact_only, check_duplicates, collect_stats).
    """
    import torch
    if not (hasattr(sites, "is_cuda") and sites.is_cuda):
        raise TypeError("sites must be a CUDA tensor (int32 [n,2])")
    sites = sites.to(torch.int32).contiguous()
    ws = Workspace(sites.shape[0], box, vor_opts_default(**opts), device=sites.device)
    ws.launch(sites)
    return ws.finish()


def build_host(sites_np, box, **opts):
    """End-to-end form over host arrays (vor_build_host): returns numpy arrays."""
    import numpy as np
    import torch
    sites_np = np.ascontiguousarray(sites_np, dtype=np.int32)
    n = sites_np.shape[0]
    o = vor_opts_default(**opts)
    b = _box(box)
    nb = vor_workspace_bytes(n, b, o)
    if nb < 0:
        raise VorError(-1, "vor_workspace_bytes")
    dev = torch.device("cuda", torch.cuda.current_device())
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
    sb = vor_host_scratch_bytes(n)
    scratch = torch.empty(sb + 256, dtype=torch.uint8, device=dev)
    ec, dc = vor_edge_capacity(n), vor_delaunay_capacity(n)
    cell_ptr = np.empty(n + 1, dtype=np.int64)
    labels = np.empty(ec, dtype=np.int32)
    vx = np.empty(ec, dtype=np.float64)
    vy = np.empty(ec, dtype=np.float64)
    dl = np.empty((dc, 2), dtype=np.int32)
    ne, nd = ctypes.c_int64(), ctypes.c_int64()
    P = ctypes.c_void_p
    rc = vor_build_host(P(sites_np.ctypes.data), n, b, ctypes.byref(o),
                        P((ws.data_ptr() + 255) & ~255), nb, P((scratch.data_ptr() + 255) & ~255),
                        sb, P(cell_ptr.ctypes.data), P(labels.ctypes.data), P(vx.ctypes.data),
                        P(vy.ctypes.data), P(dl.ctypes.data), ec, dc, ctypes.byref(ne),
                        ctypes.byref(nd), P(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise VorError(rc, "vor_build_host")
    return Diagram(cell_ptr, labels[:ne.value], vx[:ne.value], vy[:ne.value], dl[:nd.value], {})


@dataclass
class BatchDiagram:
    """Result of a batch build: concatenated arrays, labels local to each set."""
    set_ptr: object       # int64 [S+1] (host)
    cell_ptr: object      # int64 [N+1]
    labels: object        # int32 [E]
    vx: object
    vy: object
    delaunay: object      # int32 [M, 2]
    del_set_ptr: object   # int64 [S+1]
    stats: dict

    def set(self, j: int) -> Diagram:
        """The diagram of set j (views; cell_ptr rebased to the set's first edge)."""
        a, b = int(self.set_ptr[j]), int(self.set_ptr[j + 1])
        cp = self.cell_ptr[a:b + 1]
        e0, e1 = int(cp[0]), int(cp[-1])
        d0, d1 = int(self.del_set_ptr[j]), int(self.del_set_ptr[j + 1])
        return Diagram(cp - e0, self.labels[e0:e1], self.vx[e0:e1], self.vy[e0:e1],
                       self.delaunay[d0:d1], {})


def vor_autotune_grid() -> list:
    """The library's default autotuner candidates (VorOpts)."""
    buf = (VorOpts * 64)()
    k = int(library().vor_autotune_grid(buf, 64))
    return [buf[i] for i in range(k)]


class BatchWorkspace:
    """Device buffers for repeated batch builds with fixed set offsets and boxes."""

    def __init__(self, set_ptr, boxes, opts: VorOpts, device=None, extra_opts=()):
        import numpy as np
        import torch
        self.set_ptr = np.ascontiguousarray(set_ptr, dtype=np.int64)
        self.boxes = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 2)
        self.n_sets = int(self.set_ptr.shape[0] - 1)
        if self.boxes.shape[0] != self.n_sets:
            raise ValueError("one box per set")
        self.n = int(self.set_ptr[-1])
        self.opts = opts
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        nb = max(vor_batch_workspace_bytes(self.set_ptr, self.boxes, o)
                 for o in (opts, *extra_opts))
        if nb < 0:
            raise VorError(-1, "vor_batch_workspace_bytes")
        self.ws = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
        self.ws_ptr = (self.ws.data_ptr() + 255) & ~255
        self.ws_bytes = nb
        self.d_set_ptr = torch.from_numpy(self.set_ptr).to(dev)
        self.d_boxes = torch.from_numpy(self.boxes).to(dev)
        ec = vor_batch_edge_capacity(self.n, self.n_sets)
        dc = vor_batch_delaunay_capacity(self.n, self.n_sets)
        self.cell_ptr = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
        self.labels = torch.empty(ec, dtype=torch.int32, device=dev)
        self.vx = torch.empty(ec, dtype=torch.float64, device=dev)
        self.vy = torch.empty(ec, dtype=torch.float64, device=dev)
        self.del_edge = torch.empty((dc, 2), dtype=torch.int32, device=dev)
        self.del_set_ptr = torch.zeros(self.n_sets + 1, dtype=torch.int64, device=dev)
        self.totals = torch.zeros(2, dtype=torch.int64, device=dev)
        self.out = VorOut(self.cell_ptr.data_ptr(), self.labels.data_ptr(), self.vx.data_ptr(),
                          self.vy.data_ptr(), self.del_edge.data_ptr(), self.totals.data_ptr(),
                          ec, dc)

    def launch(self, d_sites, stream=None) -> None:
        """Enqueue a build of the concatenated sites (int32 [N,2] on the device)."""
        import torch
        if d_sites.shape[0] != self.n:
            raise ValueError("sites do not match the set offsets")
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = vor_build_batch_async(d_sites.data_ptr(), self.d_set_ptr.data_ptr(), self.set_ptr,
                                   self.d_boxes.data_ptr(), self.boxes, self.opts, self.ws_ptr,
                                   self.ws_bytes, self.out, self.del_set_ptr.data_ptr(),
                                   s.cuda_stream)
        if rc != 0:
            raise VorError(rc, "vor_build_batch_async")

    def finish(self, stream=None) -> BatchDiagram:
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        rc, st = vor_status(self.ws_ptr, s.cuda_stream)
        if rc != 0:
            raise VorError(rc, "vor_status")
        ne, nd = (int(v) for v in self.totals.cpu())
        return BatchDiagram(self.set_ptr, self.cell_ptr, self.labels[:ne], self.vx[:ne],
                            self.vy[:ne], self.del_edge[:nd], self.del_set_ptr, st.as_dict())


def build_batch(sites, set_ptr, boxes, **opts) -> BatchDiagram:
    """Diagrams of many independent sets in one build.

    sites: torch int32 [N,2] on the GPU, the sets one after another;
    set_ptr: int64 [S+1] host offsets; boxes: int32 [S,2] host (w, h) per set.
    """
    import torch
    if not (hasattr(sites, "is_cuda") and sites.is_cuda):
        raise TypeError("sites must be a CUDA tensor (int32 [N,2])")
    sites = sites.to(torch.int32).contiguous()
    ws = BatchWorkspace(set_ptr, boxes, vor_opts_default(**opts), device=sites.device)
    ws.launch(sites)
    return ws.finish()


def autotune_batch(sites, set_ptr, boxes, candidates=None, reps: int = 2):
    """Time each candidate option set on this batch (vor_autotune_batch).

    Returns (best VorOpts, list of (VorOpts, mean ms)).  The batch may be a
    sample of the sets to be built later.
    """
    import numpy as np
    import torch
    cands = list(candidates) if candidates is not None else vor_autotune_grid()
    ws = BatchWorkspace(set_ptr, boxes, cands[0], device=sites.device, extra_opts=cands[1:])
    arr = (VorOpts * len(cands))(*cands)
    ms = (ctypes.c_float * len(cands))()
    best = ctypes.c_int32(-1)
    P = ctypes.c_void_p
    s = torch.cuda.current_stream()
    rc = library().vor_autotune_batch(
        P(sites.data_ptr()), P(ws.d_set_ptr.data_ptr()), P(ws.set_ptr.ctypes.data), ws.n_sets,
        P(ws.d_boxes.data_ptr()), P(ws.boxes.ctypes.data), arr, len(cands), int(reps),
        P(ws.ws_ptr), ws.ws_bytes, ctypes.byref(ws.out), P(ws.del_set_ptr.data_ptr()),
        P(s.cuda_stream), ctypes.byref(best), ms)
    if rc != 0:
        raise VorError(rc, "vor_autotune_batch")
    if best.value < 0:
        raise VorError(-6, "vor_autotune_batch: no candidate completed")
    return cands[best.value], [(c, float(ms[i])) for i, c in enumerate(cands)]


# ------------------------------------------------------------------ serving ----

def vor_server_config_default(**kw) -> VorServerConfig:
    """Server configuration with the library defaults; keyword arguments set
    fields (``opts`` takes a VorOpts)."""
    c = VorServerConfig()
    library().vor_server_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if v is None:
            continue
        if not hasattr(c, k):
            raise TypeError(f"unknown server option {k}")
        setattr(c, k, v if k == "opts" else int(v))
    return c


class Server:
    """The request server of the library (vor_server_*): continuous batching
    of point sets submitted from host memory.  Results are copied into numpy
    arrays by ``wait``/``poll`` and the ticket is released unless
    ``keep=True``."""

    def __init__(self, config: VorServerConfig | None = None, **kw):
        cfg = config if config is not None else vor_server_config_default(**kw)
        self._h = ctypes.c_void_p()
        rc = library().vor_server_create(ctypes.byref(cfg), ctypes.byref(self._h))
        if rc != 0:
            raise VorError(rc, "vor_server_create")
        self.config = cfg

    def submit(self, sites_np, box, timeout: float = 60.0) -> int:
        import numpy as np
        a = np.ascontiguousarray(sites_np, dtype=np.int32).reshape(-1, 2)
        t = ctypes.c_uint64()
        rc = library().vor_server_submit(self._h, ctypes.c_void_p(a.ctypes.data), a.shape[0],
                                         _box(box), float(timeout), ctypes.byref(t))
        if rc != 0:
            raise VorError(rc, "vor_server_submit")
        return int(t.value)

    @staticmethod
    def _result(r: VorRequestResult, arrays: bool = True) -> dict:
        import numpy as np
        out = {"status": int(r.status), "n": int(r.n), "wave_requests": int(r.wave_requests),
               "t_submit": r.t_submit, "t_start": r.t_start, "t_done": r.t_done,
               "n_edges": int(r.n_edges), "n_del": int(r.n_del)}
        if r.status == 0 and arrays:
            def arr(p, ct, count, shape=None):
                if count == 0:
                    return np.zeros(shape or (0,), dtype=np.dtype(ct))
                buf = (ct * count).from_address(p)
                a = np.frombuffer(buf, dtype=np.dtype(ct)).copy()
                return a.reshape(shape) if shape else a
            ne, nd = int(r.n_edges), int(r.n_del)
            out.update(cell_ptr=arr(r.cell_ptr, ctypes.c_int64, int(r.n) + 1),
                       labels=arr(r.edge_label, ctypes.c_int32, ne),
                       vx=arr(r.vx, ctypes.c_double, ne), vy=arr(r.vy, ctypes.c_double, ne),
                       delaunay=arr(r.del_edge, ctypes.c_int32, 2 * nd, (nd, 2)))
        return out

    def poll(self, ticket: int, keep: bool = False):
        """None while pending; else the result dict (status, arrays when ok)."""
        r = VorRequestResult()
        r.status = 99                    # untouched by the library for an unknown ticket
        rc = library().vor_server_poll(self._h, ticket, ctypes.byref(r))
        if r.status == 99:
            raise VorError(rc, "vor_server_poll: unknown ticket")
        if rc == PENDING:
            return None
        out = self._result(r)
        if not keep:
            self.release(ticket)
        return out

    def wait(self, ticket: int, timeout: float = 600.0, keep: bool = False,
             arrays: bool = True) -> dict:
        """The result dict once final (raises VorError on timeout); with
        arrays=False only the status, sizes and times."""
        r = VorRequestResult()
        r.status = 99
        rc = library().vor_server_wait(self._h, ticket, float(timeout), ctypes.byref(r))
        if r.status == 99:
            raise VorError(rc, "vor_server_wait: unknown ticket")
        if rc == E_TIMEOUT:
            raise VorError(rc, "vor_server_wait")
        out = self._result(r, arrays)
        if not keep:
            self.release(ticket)
        return out

    def cancel(self, ticket: int) -> None:
        rc = library().vor_server_cancel(self._h, ticket)
        if rc != 0:
            raise VorError(rc, "vor_server_cancel")

    def release(self, ticket: int) -> None:
        rc = library().vor_server_release(self._h, ticket)
        if rc != 0:
            raise VorError(rc, "vor_server_release")

    def stats(self) -> dict:
        st = VorServerStats()
        library().vor_server_statistics(self._h, ctypes.byref(st))
        return st.as_dict()

    def now(self) -> float:
        return float(library().vor_server_now(self._h))

    def close(self) -> None:
        if self._h:
            library().vor_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
