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
