"""Independent exact reference computations used to pin the oracle.

Nothing here shares code with the oracle or the CUDA library.  Everything is
pure Python on ``fractions.Fraction``, written from the definitions:

* ``halfplane_cell``: the Voronoi cell of Definition 2.1 as X intersected with
  the half-planes {x : |x - p| <= |x - a|} (the "naive method" the paper's
  introduction and Section 2 describe), by successive exact polygon clipping.
* ``restricted_delaunay``: the Delaunay graph restricted to X (Section 6),
  computed in the dual way: for every pair of sites, the set of centres of
  circles through both sites with no site strictly inside is an interval of
  their bisector (the Voronoi edge of the whole plane); the pair is an edge
  when that interval, cut to X, has positive length.
"""

from __future__ import annotations

import math
from fractions import Fraction as F

SIDE_BOTTOM, SIDE_RIGHT, SIDE_TOP, SIDE_LEFT = -1, -2, -3, -4


def _constraints(xy, k, W, H):
    """Half-planes a.x <= b bounding the cell of site k, with their labels."""
    px, py = int(xy[k][0]), int(xy[k][1])
    cons = [((0, -1), 0, SIDE_BOTTOM), ((1, 0), W, SIDE_RIGHT),
            ((0, 1), H, SIDE_TOP), ((-1, 0), 0, SIDE_LEFT)]
    for j in range(len(xy)):
        if j == k:
            continue
        ax, ay = int(xy[j][0]), int(xy[j][1])
        # |x-p|^2 <= |x-a|^2  <=>  2 (a-p).x <= |a|^2 - |p|^2
        cons.append(((2 * (ax - px), 2 * (ay - py)), ax * ax + ay * ay - px * px - py * py, j))
    return cons


def _clip(poly, a, b):
    """Sutherland-Hodgman clip of a convex polygon by a.x <= b (exact)."""
    out = []
    m = len(poly)
    for i in range(m):
        P, Q = poly[i], poly[(i + 1) % m]
        fp = a[0] * P[0] + a[1] * P[1] - b
        fq = a[0] * Q[0] + a[1] * Q[1] - b
        if fp <= 0:
            out.append(P)
        if (fp < 0 < fq) or (fq < 0 < fp):
            s = fp / (fp - fq)
            out.append((P[0] + s * (Q[0] - P[0]), P[1] + s * (Q[1] - P[1])))
    # drop repeated points
    res = []
    for v in out:
        if not res or res[-1] != v:
            res.append(v)
    if len(res) > 1 and res[0] == res[-1]:
        res.pop()
    return res


def halfplane_cell(xy, k, W, H):
    """Exact cell of site k: (labels, vertices) in canonical form.

    labels: lines carrying an edge of positive length, ordered
    counter-clockwise by the polar angle of the edge's outward normal,
    starting from the smallest angle in [0, 2 pi).  vertices[i] is the end of
    edge i (the point shared with edge i+1).
    """
    cons = _constraints(xy, k, W, H)
    poly = [(F(0), F(0)), (F(W), F(0)), (F(W), F(H)), (F(0), F(H))]
    for a, b, _ in cons:
        poly = _clip(poly, a, b)
    # remove collinear vertices so every polygon edge has its own line
    changed = True
    while changed and len(poly) > 3:
        changed = False
        m = len(poly)
        for i in range(m):
            A, B, C = poly[i - 1], poly[i], poly[(i + 1) % m]
            if (B[0] - A[0]) * (C[1] - B[1]) - (B[1] - A[1]) * (C[0] - B[0]) == 0:
                poly.pop(i)
                changed = True
                break
    m = len(poly)
    edges = []
    for i in range(m):
        P, Q = poly[i], poly[(i + 1) % m]
        tight = [lab for a, b, lab in cons
                 if a[0] * P[0] + a[1] * P[1] == b and a[0] * Q[0] + a[1] * Q[1] == b]
        assert len(tight) == 1, (k, tight)
        a = next(c[0] for c in cons if c[2] == tight[0])
        ang = math.atan2(a[1], a[0])
        if ang < 0:
            ang += 2 * math.pi
        edges.append((ang, tight[0], Q))
    start = min(range(m), key=lambda i: edges[i][0])
    edges = edges[start:] + edges[:start]
    return [e[1] for e in edges], [e[2] for e in edges]


def restricted_delaunay(xy, W, H):
    """Delaunay edges (j, k), j < k, restricted to X, by the empty-circle rule."""
    n = len(xy)
    pts = [(int(x), int(y)) for x, y in xy]
    out = []
    for j in range(n):
        for k in range(j + 1, n):
            pj, pk = pts[j], pts[k]
            mx, my = F(pj[0] + pk[0], 2), F(pj[1] + pk[1], 2)
            dx, dy = -(pk[1] - pj[1]), pk[0] - pj[0]      # bisector direction
            lo, hi = None, None                            # admissible t interval
            empty = True
            for a in range(n):
                if a == j or a == k:
                    continue
                pa = pts[a]
                # |c-a|^2 - |c-pj|^2 >= 0 with c = m + t d:
                # (|m-a|^2 - |m-pj|^2) + 2 t <d, pj - a> >= 0
                c0 = ((mx - pa[0]) ** 2 + (my - pa[1]) ** 2) - ((mx - pj[0]) ** 2 + (my - pj[1]) ** 2)
                c1 = 2 * (dx * (pj[0] - pa[0]) + dy * (pj[1] - pa[1]))
                if c1 == 0:
                    if c0 < 0:
                        empty = False
                        break
                    continue
                t0 = -c0 / c1
                if c1 > 0:
                    lo = t0 if lo is None else max(lo, t0)
                else:
                    hi = t0 if hi is None else min(hi, t0)
            if not empty:
                continue
            # restrict c(t) to X: 0 <= mx + t dx <= W, 0 <= my + t dy <= H
            for m0, d0, top in ((mx, dx, W), (my, dy, H)):
                if d0 == 0:
                    if not (0 <= m0 <= top):
                        empty = False
                    continue
                ta, tb = (0 - m0) / d0, (top - m0) / d0
                if ta > tb:
                    ta, tb = tb, ta
                lo = ta if lo is None else max(lo, ta)
                hi = tb if hi is None else min(hi, tb)
            if empty and lo is not None and hi is not None and lo < hi:
                out.append((j, k))
    return out


def polygon_area(verts):
    s = F(0)
    m = len(verts)
    for i in range(m):
        x0, y0 = verts[i]
        x1, y1 = verts[(i + 1) % m]
        s += x0 * y1 - x1 * y0
    return s / 2
