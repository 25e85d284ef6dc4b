"""Comparison of a GPU diagram with the oracle's (shared by the GPU tests).

Bit-exact: cell offsets, edge labels (the canonical counter-clockwise order)
and Delaunay pairs.  float64 vertices: |x_gpu - x| <= 1e-9 max(|x|, 1) per
coordinate, x the exact rational vertex of the oracle.
"""

from __future__ import annotations

import numpy as np

VERTEX_RTOL = 1e-9


def to_numpy(d):
    import torch

    def cv(t):
        return t.cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)

    return {"cell_ptr": cv(d.cell_ptr), "labels": cv(d.labels), "vx": cv(d.vx), "vy": cv(d.vy),
            "delaunay": cv(d.delaunay).reshape(-1, 2)}


def exact_vertices(r):
    v = r["vnum"]
    den = v[:, 2].astype(np.float64)
    return v[:, 0].astype(np.float64) / den, v[:, 1].astype(np.float64) / den


def assert_vertices_close(gx, gy, ox, oy):
    for g, o, name in ((gx, ox, "x"), (gy, oy, "y")):
        err = np.abs(g - o)
        tol = VERTEX_RTOL * np.maximum(np.abs(o), 1.0)
        bad = np.nonzero(err > tol)[0]
        assert bad.size == 0, f"vertex {name} mismatch at {bad[:5]}: {g[bad[:5]]} vs {o[bad[:5]]}"


def assert_full_parity(d, r):
    """Whole diagram: GPU result d (to_numpy form) vs oracle result r."""
    assert np.array_equal(d["cell_ptr"], r["cell_ptr"]), _first_cell_diff(d, r)
    assert np.array_equal(d["labels"], r["labels"]), _first_cell_diff(d, r)
    assert np.array_equal(d["delaunay"], r["delaunay"].reshape(-1, 2))
    ox, oy = exact_vertices(r)
    assert_vertices_close(d["vx"], d["vy"], ox, oy)


def assert_sampled_parity(d, r, sel):
    """Cells sel (oracle computed only those, in that order) vs the GPU's."""
    cp = d["cell_ptr"]
    ox, oy = exact_vertices(r)
    for i, k in enumerate(sel):
        a, b = cp[k], cp[k + 1]
        ra, rb = r["cell_ptr"][i], r["cell_ptr"][i + 1]
        assert np.array_equal(d["labels"][a:b], r["labels"][ra:rb]), (
            f"cell {k}: gpu {d['labels'][a:b]} oracle {r['labels'][ra:rb]}")
        assert_vertices_close(d["vx"][a:b], d["vy"][a:b], ox[ra:rb], oy[ra:rb])


def _first_cell_diff(d, r):
    n = min(len(d["cell_ptr"]), len(r["cell_ptr"])) - 1
    for k in range(n):
        a, b = d["cell_ptr"][k], d["cell_ptr"][k + 1]
        ra, rb = r["cell_ptr"][k], r["cell_ptr"][k + 1]
        if b - a != rb - ra or not np.array_equal(d["labels"][a:b], r["labels"][ra:rb]):
            return f"first differing cell {k}: gpu {d['labels'][a:b]} oracle {r['labels'][ra:rb]}"
    return "cells agree; totals differ"


def delaunay_symmetric_ok(d, n):
    """Properties that hold at any size: each Delaunay pair appears as a
    neighbour label in both cells, k < j, ordered by (k, j), E <= 3n - 6."""
    dl = d["delaunay"]
    if dl.shape[0] == 0:
        return True
    assert np.all(dl[:, 0] < dl[:, 1])
    key = dl[:, 0].astype(np.int64) * n + dl[:, 1]
    assert np.all(np.diff(key) > 0)
    if n >= 3:
        assert dl.shape[0] <= 3 * n - 6
    cp, lab = d["cell_ptr"], d["labels"]
    cell_of = np.repeat(np.arange(n), np.diff(cp))
    nbr = lab >= 0
    pairs = np.stack([np.minimum(cell_of[nbr], lab[nbr]), np.maximum(cell_of[nbr], lab[nbr])], 1)
    pk = pairs[:, 0].astype(np.int64) * n + pairs[:, 1]
    u, cnt = np.unique(pk, return_counts=True)
    assert np.all(cnt == 2), "every neighbour relation is listed by both cells"
    assert np.array_equal(u, key), "Delaunay pairs are exactly the neighbour pairs"
    return True


# ------------------------------------------------- stored oracle digests ----
#
# The oracle needs minutes to hours for the full-size clustered workloads, so
# tests/golden/make_digests.py runs it once (oracle only) and stores, per
# chunk of cells (or per set, or per request), a digest of the exact
# combinatorial output: the edge counts e_k, the edge labels in canonical
# order and the Delaunay pairs whose first index lies in the chunk.  A GPU
# test recomputes the same digest from the GPU output; equal digests mean
# bit-identical combinatorics.  The float64 vertices are then checked
# against the intersection of their two lines, computed exactly from the
# (verified) labels: vertex i of cell k is the point where the lines of
# edges i and i+1 meet (Section 5), u = p + N / D with integer N, D.

DIGEST_CHUNK = 1 << 16


def input_digest(xy) -> str:
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(xy, dtype=np.int32).tobytes()).hexdigest()


def cells_digest(cell_ptr, labels, delaunay, lo, hi, base=0) -> str:
    """Digest of cells [lo, hi) of a diagram (cell_ptr, labels, delaunay
    given for the whole diagram or set; `base` is subtracted from the cell
    offsets, so a set inside a batch digests like a diagram of its own)."""
    import hashlib
    cp = np.asarray(cell_ptr, dtype=np.int64)
    e = np.diff(cp[lo:hi + 1]).astype(np.int64)
    lab = np.asarray(labels, dtype=np.int32)[cp[lo] - base:cp[hi] - base]
    dl = np.asarray(delaunay, dtype=np.int32).reshape(-1, 2)
    a, b = np.searchsorted(dl[:, 0], [lo, hi], side="left")
    h = hashlib.sha256()
    h.update(np.int64(hi - lo).tobytes())
    h.update(e.tobytes())
    h.update(np.ascontiguousarray(lab).tobytes())
    h.update(np.ascontiguousarray(dl[a:b]).tobytes())
    return h.hexdigest()[:32]


def chunk_digests(cell_ptr, labels, delaunay, n, chunk=DIGEST_CHUNK) -> list:
    return [cells_digest(cell_ptr, labels, delaunay, lo, min(n, lo + chunk))
            for lo in range(0, n, chunk)]


def _lines(xy, box, k, lab):
    """Line 2 <nv, v - p> = c of label lab in the cell of site k (int64):
    a neighbour site j (nv = p_j - p, c = |nv|^2) or a side of X (nv the
    offset to p's reflection across the side, halved; c = 2 |nv|^2)."""
    W, H = (box, box) if np.isscalar(box) else box
    px = xy[k, 0].astype(np.int64)
    py = xy[k, 1].astype(np.int64)
    site = lab >= 0
    j = np.where(site, lab, 0)
    nx = np.where(site, xy[j, 0].astype(np.int64) - px, 0)
    ny = np.where(site, xy[j, 1].astype(np.int64) - py, 0)
    nx = np.where(lab == -2, W - px, np.where(lab == -4, -px, nx))
    ny = np.where(lab == -1, -py, np.where(lab == -3, H - py, ny))
    c = nx * nx + ny * ny
    c = np.where(site, c, 2 * c)
    return nx, ny, c


def assert_vertices_from_labels(xy, box, d):
    """The GPU's float64 vertices against the exact meeting point of each
    vertex's two lines (from the labels, which the digest has verified):
    |x_gpu - x| <= 1e-9 max(|x|, 1).  N and D are exact int64 (|N| < 2^62,
    |D| < 2^44) and so is the numerator p D + N; one rounding of it and one
    of the quotient keep x within 2^-52 |x|, far below the tolerance."""
    cp = np.asarray(d["cell_ptr"], dtype=np.int64)
    lab = np.asarray(d["labels"], dtype=np.int64)
    n = cp.shape[0] - 1
    e = np.diff(cp)
    k = np.repeat(np.arange(n), e)
    nxt = np.arange(lab.shape[0]) + 1
    nxt[cp[1:][e > 0] - 1] = cp[:-1][e > 0]
    xy = np.asarray(xy, dtype=np.int64)
    n1x, n1y, c1 = _lines(xy, box, k, lab)
    n2x, n2y, c2 = _lines(xy, box, k, lab[nxt])
    Nx = c1 * n2y - c2 * n1y
    Ny = c2 * n1x - c1 * n2x
    D = 2 * (n1x * n2y - n1y * n2x)
    assert np.all(D != 0), "consecutive edges on parallel lines"
    sg = np.where(D < 0, -1, 1)
    D, Nx, Ny = D * sg, Nx * sg, Ny * sg
    # the absolute vertex (p D + N) / D: its numerators lie in [0, W D]
    # (the vertex is in X), below 2^63, so the wrapping uint64 sum is exact
    u = np.uint64
    numx = xy[k, 0].astype(u) * D.astype(u) + Nx.astype(u)
    numy = xy[k, 1].astype(u) * D.astype(u) + Ny.astype(u)
    assert np.all(numx < u(1 << 63)) and np.all(numy < u(1 << 63)), "vertex outside X"
    ox = numx.astype(np.float64) / D.astype(np.float64)
    oy = numy.astype(np.float64) / D.astype(np.float64)
    assert_vertices_close(np.asarray(d["vx"]), np.asarray(d["vy"]), ox, oy)


def assert_shared_vertices_identical(d):
    """Each vertex is computed once, by the cell of the smallest site that
    shares it, and copied into the other cells: every vertex listed by
    several cells (the same three lines: three sites, or two sites and a
    side) carries bit-identical float64 coordinates in all of them."""
    cp = np.asarray(d["cell_ptr"], dtype=np.int64)
    lab = np.asarray(d["labels"], dtype=np.int64)
    n = cp.shape[0] - 1
    e = np.diff(cp)
    k = np.repeat(np.arange(n), e)
    nxt = np.arange(lab.shape[0]) + 1
    nxt[cp[1:][e > 0] - 1] = cp[:-1][e > 0]
    a, b = lab, lab[nxt]
    keep = (a >= 0) | (b >= 0)                       # at least one neighbour cell shares it
    t = np.sort(np.stack([k, a, b], 1)[keep], axis=1)
    vx = np.asarray(d["vx"])[keep]
    vy = np.asarray(d["vy"])[keep]
    order = np.lexsort((t[:, 2], t[:, 1], t[:, 0]))
    t, vx, vy = t[order], vx[order], vy[order]
    same = np.all(t[1:] == t[:-1], axis=1)
    assert same.sum() > 0, "no shared vertex found"
    bad = np.nonzero(same & ((vx[1:] != vx[:-1]) | (vy[1:] != vy[:-1])))[0]
    assert bad.size == 0, f"shared vertex differs between cells: {t[bad[:3]]}"
