"""Exact CPU oracle of the projector algorithm (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: ``vor_oracle.c`` is compiled here with gcc and called through ctypes.

Functions
---------
``build_library()``   compile ``vor_oracle.c`` into ``oracle/_build/liboracle.so``
``cells(...)``        Voronoi cells (+ Delaunay edges, counters) of all or some sites
``endpoint(...)``     one ray endpoint T(p, theta) with its EquiDistList extremes
``si_rect(...)``      the integer rectangle S_I[y, r] of eq. (A.3)
``paper_beta(n)``     beta of Theorem 8.1(e) for a given n and epsilon

Every function follows the passage of the paper named in its docstring; the
C source carries the detailed citations.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vor_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

ST_NAMES = ("rays", "nodes", "endpoints", "comparisons", "vertices", "degenerate",
            "edges", "repeat_hits")

ERRORS = {-1: "invalid argument", -2: "site outside the open rectangle",
          -3: "duplicate site", -4: "box too large", -5: "out of memory",
          -9: "internal check failed"}

_lib = None
_lib_override = None


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, 'unknown')}")
        self.code = code


def build_library(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, pthreads)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib_override is not None:
        return _lib_override
    if _lib is not None:
        return _lib
    _lib = _bind(ctypes.CDLL(build_library()))
    return _lib


def _bind(lib):
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.orc_build.restype = P
    lib.orc_build.argtypes = [P, i64, i64, i64, ctypes.c_int, i64, i64, P, i64, ctypes.c_int,
                              ctypes.POINTER(ctypes.c_int)]
    lib.orc_result_sizes.argtypes = [P, P, P, P]
    lib.orc_result_copy.argtypes = [P, P, P, P, P, P]
    lib.orc_result_free.argtypes = [P]
    lib.orc_endpoint.restype = ctypes.c_int
    lib.orc_endpoint.argtypes = [P, i64, i64, i64, ctypes.c_int, i64, i64, i64, i64, i64, P, P, P]
    lib.orc_si.argtypes = [i64, i64, i64, i64, i64, i64, P]
    lib.orc_eta.restype = i64
    lib.orc_eta.argtypes = [i64, i64]
    return lib


class use_library:
    """Context manager: run the oracle functions against another build of the
    oracle source (the mutation tests compile copies with planted mistakes)."""

    def __init__(self, so_path: str):
        self.lib = _bind(ctypes.CDLL(so_path))

    def __enter__(self):
        global _lib_override
        _lib_override = self.lib
        return self

    def __exit__(self, *exc):
        global _lib_override
        _lib_override = None


def paper_beta(n: int, eps: float = 1e-6) -> int:
    """beta of Theorem 8.1(e): alpha_1 = (floor(sqrt(ln(n(1+2e^-400)/eps))) + OneTwo)^2,
    OneTwo making sqrt(alpha_1) odd, and beta = (sqrt(alpha_1) - 1) / 2."""
    f = int(math.floor(math.sqrt(math.log(n * (1 + 2 * math.exp(-400)) / eps))))
    one_two = 1 if f % 2 == 0 else 2
    return (f + one_two - 1) // 2


def paper_bucket_side(n: int, width: int) -> int:
    """Bucket side of Remark B.1(iv): m1 = m2 = floor(sqrt(n)) buckets per side,
    s = width / m1, rounded up to an integer so the grid covers X."""
    m1 = max(1, int(math.isqrt(n)))
    return -(-width // m1)


def _mode_args(mode, n, width, bucket_side, beta):
    if mode == "plain":
        return 0, 0, 0
    if mode == "bucketed":
        s = bucket_side if bucket_side else paper_bucket_side(n, width)
        b = beta if beta else paper_beta(n)
        return 1, s, b
    raise ValueError(mode)


def cells(xy, box, mode: str = "plain", sel=None, nthreads: int = 0,
          bucket_side: int | None = None, beta: int | None = None) -> dict:
    """Voronoi cells of the sites ``xy`` (int32 [n,2]) in X = [0,W] x [0,H].

    Returns a dict with, for the selected cells (all when ``sel`` is None):
      cell_ptr int64[m+1], labels int32[E] (canonical counter-clockwise order
      of outward normals starting at the smallest polar angle), vnum int64[E,3]
      (vertex i of a cell = (vnum[i,0]/vnum[i,2], vnum[i,1]/vnum[i,2]) exactly,
      the meeting point of edges i and i+1), delaunay int32[M,2] (pairs k < j
      ordered by k then j, from the selected cells), stats int64[m, 8].
    """
    lib = _load()
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    n = xy.shape[0]
    W, H = (box, box) if np.isscalar(box) else box
    m, s, b = _mode_args(mode, n, int(W), bucket_side, beta)
    if nthreads <= 0:
        nthreads = os.cpu_count() or 1
    selp = None
    nsel = 0
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        selp = sel.ctypes.data
        nsel = sel.shape[0]
    err = ctypes.c_int(0)
    h = lib.orc_build(xy.ctypes.data, n, int(W), int(H), m, s, b, selp, nsel, nthreads,
                      ctypes.byref(err))
    if not h:
        raise OracleError(err.value)
    try:
        if err.value != 0:
            raise OracleError(err.value)
        ns, ne, nd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lib.orc_result_sizes(h, ctypes.byref(ns), ctypes.byref(ne), ctypes.byref(nd))
        cell_ptr = np.zeros(ns.value + 1, dtype=np.int64)
        labels = np.zeros(max(ne.value, 1), dtype=np.int32)
        vnum = np.zeros((max(ne.value, 1), 3), dtype=np.int64)
        dl = np.zeros((max(nd.value, 1), 2), dtype=np.int32)
        stats = np.zeros((max(ns.value, 1), len(ST_NAMES)), dtype=np.int64)
        lib.orc_result_copy(h, cell_ptr.ctypes.data, labels.ctypes.data, vnum.ctypes.data,
                            dl.ctypes.data, stats.ctypes.data)
    finally:
        lib.orc_result_free(h)
    return {"cell_ptr": cell_ptr, "labels": labels[:ne.value], "vnum": vnum[:ne.value],
            "delaunay": dl[:nd.value], "stats": stats[:ns.value]}


def vertices_exact(res: dict, i: int) -> list:
    """Vertices of the i-th returned cell as exact Fractions."""
    a, b = res["cell_ptr"][i], res["cell_ptr"][i + 1]
    return [(Fraction(int(v[0]), int(v[2])), Fraction(int(v[1]), int(v[2])))
            for v in res["vnum"][a:b]]


def vertices_float(res: dict) -> tuple[np.ndarray, np.ndarray]:
    """float64 vertex coordinates (numerator / denominator; two roundings)."""
    v = res["vnum"]
    d = v[:, 2].astype(np.float64)
    return v[:, 0].astype(np.float64) / d, v[:, 1].astype(np.float64) / d


def endpoint(xy, box, k: int, theta, mode: str = "plain", bucket_side=None, beta=None):
    """The endpoint of the ray from site k in direction theta (eq. (2.1)).

    Returns (ccw_label, cw_label, n_tied_lines, t as Fraction, comparisons);
    the endpoint is p_k + t * theta.
    """
    lib = _load()
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    n = xy.shape[0]
    W, H = (box, box) if np.isscalar(box) else box
    m, s, b = _mode_args(mode, n, int(W), bucket_side, beta)
    out = np.zeros(3, dtype=np.int32)
    t4 = np.zeros(4, dtype=np.int64)
    cmp = ctypes.c_int64(0)
    rc = lib.orc_endpoint(xy.ctypes.data, n, int(W), int(H), m, s, b, int(k), int(theta[0]),
                          int(theta[1]), out.ctypes.data, t4.ctypes.data, ctypes.byref(cmp))
    if rc != 0:
        raise OracleError(rc)

    def join(hi, lo):
        return (int(hi) << 64) + (int(lo) & 0xFFFFFFFFFFFFFFFF)

    t = Fraction(join(t4[0], t4[1]), join(t4[2], t4[3]))
    return int(out[0]), int(out[1]), int(out[2]), t, cmp.value


def si_rect(y, r, s: int):
    """S_I[y, r] of eq. (A.3) for rational y = (yx, yy) and r (Fractions or ints).

    Returns (x_lo, x_hi, y_lo, y_hi)."""
    lib = _load()
    yx, yy, r = Fraction(y[0]), Fraction(y[1]), Fraction(r)
    den = math.lcm(yx.denominator, yy.denominator)
    out = np.zeros(4, dtype=np.int64)
    lib.orc_si(int(yx * den), int(yy * den), den, r.numerator, r.denominator, int(s),
               out.ctypes.data)
    return tuple(int(v) for v in out)


def eta(beta: int, s: int) -> int:
    """The integer probe distance of Method A.6: smallest eta >= 4 sqrt(2) (beta+1.01) s."""
    return int(_load().orc_eta(int(beta), int(s)))
