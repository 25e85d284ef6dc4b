"""Seeded synthetic point-site generators.

This module holds no arithmetic of the projector method.  It only draws
integer point sites (and request streams) from fixed seeds, with the shapes
and distributions of the workloads the method is measured on:

* uniform sites in a square world X = [0, W] x [0, H] (Section 8, part (e) of
  the paper analyses exactly this case),
* a Gaussian-mixture ("clustered") distribution that stresses the uniform
  bucketing of Method A.5,
* batches of independent point sets of log-uniform size,
* a Poisson stream of requests for the serving loop.

Every random number comes from SplitMix64 evaluated on a counter
(``mix(seed + i * GOLDEN)``), so a value depends only on (seed, stream, i) and
never on the order in which arrays are drawn.  Coordinates are drawn from
[1, W-1] x [1, H-1] so every site is strictly inside X, which the paper
assumes (Section 2, before Definition 2.1); the library rejects sites on the
boundary of X.

Both the oracle-side tests and the GPU path take their inputs from here; the
oracle and the CUDA path never exchange data.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64",
    "uniform_sites",
    "gaussian_mixture_sites",
    "enforce_general_position",
    "batch_sets",
    "poisson_requests",
    "lattice_sites",
    "WORLD",
    "SEED_BASE",
]

WORLD = 1 << 20          # side of the square world X used by every workload
SEED_BASE = 1212_1095     # base seed; each workload adds its own index

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Counter-based SplitMix64: returns ``count`` uint64 words.

    Word i is the SplitMix64 output for state ``seed*2^32 + stream`` advanced
    ``start + i + 1`` times.  (Steele, Lea, Flood, "Fast splittable
    pseudorandom number generators", OOPSLA 2014.)
    """
    with np.errstate(over="ignore"):
        base = np.uint64((int(seed) * (1 << 32) + int(stream)) & 0xFFFFFFFFFFFFFFFF)
        i = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        z = base + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _uniform_int(words: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Map uint64 words to integers in [lo, hi] (multiply-shift on the top 32 bits)."""
    span = np.uint64(hi - lo + 1)
    assert int(span) <= (1 << 32)
    top = words >> np.uint64(32)
    return (lo + ((top * span) >> np.uint64(32))).astype(np.int64)


def _unit_open(words: np.ndarray) -> np.ndarray:
    """Map uint64 words to doubles in the open interval (0, 1)."""
    return ((words >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / (1 << 53))


def _dedup_keep_order(xy: np.ndarray) -> np.ndarray:
    key = xy[:, 0].astype(np.int64) * (1 << 21) + xy[:, 1].astype(np.int64)
    _, first = np.unique(key, return_index=True)
    first.sort()
    return xy[first]


def _fill_unique(n: int, draw, box: int) -> np.ndarray:
    """Draw batches with ``draw(count, start)`` until n distinct sites exist.

    Duplicates are removed keeping the first occurrence; the generator then
    tops up from the continuation of the same counter stream.
    """
    out = np.zeros((0, 2), dtype=np.int64)
    start = 0
    want = n
    while True:
        batch = draw(want + 16 + want // 64, start)
        start += batch.shape[0]
        out = _dedup_keep_order(np.concatenate([out, batch]))
        if out.shape[0] >= n:
            return out[:n].astype(np.int32)
        want = n - out.shape[0]


def uniform_sites(n: int, seed: int = SEED_BASE, box: int = WORLD) -> np.ndarray:
    """n distinct sites, coordinates uniform on the integer grid [1, box-1]^2."""

    def draw(count, start):
        wx = splitmix64(seed, 1, count, start)
        wy = splitmix64(seed, 2, count, start)
        return np.stack([_uniform_int(wx, 1, box - 1), _uniform_int(wy, 1, box - 1)], axis=1)

    return _fill_unique(n, draw, box)


def gaussian_mixture_sites(n: int, seed: int = SEED_BASE, box: int = WORLD,
                           components: int = 64, sigma: float = 4096.0) -> np.ndarray:
    """n distinct sites from an isotropic Gaussian mixture.

    Centres are uniform in the world, every component has standard deviation
    ``sigma``, and the mixture weights are Dirichlet(1) (normalised Exp(1)
    draws).  Samples are rounded to the nearest integer; samples that fall
    outside [1, box-1]^2 are redrawn (rejection), so no pile-up forms at the
    boundary.  Duplicates are removed and the set is topped up to exactly n.
    """
    cw = splitmix64(seed, 10, 3 * components)
    centres = np.stack([_unit_open(cw[:components]) * box,
                        _unit_open(cw[components:2 * components]) * box], axis=1)
    g = -np.log(_unit_open(cw[2 * components:]))
    weights = g / g.sum()
    cdf = np.cumsum(weights)
    cdf[-1] = 1.0

    def draw(count, start):
        pts = []
        got = 0
        s = start
        while got < count:
            m = count - got + 64
            wc = _unit_open(splitmix64(seed, 11, m, s))
            u1 = _unit_open(splitmix64(seed, 12, m, s))
            u2 = _unit_open(splitmix64(seed, 13, m, s))
            s += m
            comp = np.searchsorted(cdf, wc, side="right")
            comp = np.minimum(comp, components - 1)
            r = np.sqrt(-2.0 * np.log(u1)) * sigma
            x = np.rint(centres[comp, 0] + r * np.cos(2 * np.pi * u2))
            y = np.rint(centres[comp, 1] + r * np.sin(2 * np.pi * u2))
            ok = (x >= 1) & (x <= box - 1) & (y >= 1) & (y <= box - 1)
            p = np.stack([x[ok], y[ok]], axis=1).astype(np.int64)
            pts.append(p)
            got += p.shape[0]
        out = np.concatenate(pts)[:count]
        return out

    # The counter offset of each top-up round must not overlap the previous
    # one; scale it so rejection redraws never reuse words.
    def draw_scaled(count, start):
        return draw(count, start * 4)

    return _fill_unique(n, draw_scaled, box)


def _incircle_exact(a, b, c, d) -> int:
    """Sign-exact incircle determinant of four integer points (Python ints)."""
    adx, ady = a[0] - d[0], a[1] - d[1]
    bdx, bdy = b[0] - d[0], b[1] - d[1]
    cdx, cdy = c[0] - d[0], c[1] - d[1]
    return ((adx * adx + ady * ady) * (bdx * cdy - cdx * bdy)
            + (bdx * bdx + bdy * bdy) * (cdx * ady - adx * cdy)
            + (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady))


def _cocircular_quads(xy: np.ndarray) -> list[tuple[int, int, int, int]]:
    """Quadruples of sites that lie exactly on one empty circle.

    Candidate quadruples are the pairs of adjacent triangles of a Delaunay
    triangulation computed by ``scipy.spatial.Delaunay``; four co-circular
    sites on an empty circle always form such a pair.  A floating-point filter
    with a generous bound discards clearly non-zero determinants and the rest
    are evaluated exactly with Python integers.
    """
    from scipy.spatial import Delaunay  # used only to enumerate candidates

    pts = xy.astype(np.float64)
    tri = Delaunay(pts)
    simp = tri.simplices
    nb = tri.neighbors
    quads = []
    t_idx, e_idx = np.nonzero(nb >= 0)
    keep = t_idx < nb[t_idx, e_idx]
    t_idx, e_idx = t_idx[keep], e_idx[keep]
    other = nb[t_idx, e_idx]
    a = simp[t_idx, 0]
    b = simp[t_idx, 1]
    c = simp[t_idx, 2]
    # the vertex of the neighbouring triangle that is not shared
    os = simp[other]
    shared = np.stack([simp[t_idx, (e_idx + 1) % 3], simp[t_idx, (e_idx + 2) % 3]], axis=1)
    mask = (os != shared[:, :1]) & (os != shared[:, 1:2])
    d = os[np.arange(os.shape[0]), np.argmax(mask, axis=1)]
    P = xy.astype(np.float64)
    A, B, C, Dd = P[a], P[b], P[c], P[d]
    adx, ady = A[:, 0] - Dd[:, 0], A[:, 1] - Dd[:, 1]
    bdx, bdy = B[:, 0] - Dd[:, 0], B[:, 1] - Dd[:, 1]
    cdx, cdy = C[:, 0] - Dd[:, 0], C[:, 1] - Dd[:, 1]
    t1 = (adx * adx + ady * ady) * (bdx * cdy - cdx * bdy)
    t2 = (bdx * bdx + bdy * bdy) * (cdx * ady - adx * cdy)
    t3 = (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady)
    det = t1 + t2 + t3
    perm = (np.abs(adx * adx + ady * ady) * (np.abs(bdx * cdy) + np.abs(cdx * bdy))
            + np.abs(bdx * bdx + bdy * bdy) * (np.abs(cdx * ady) + np.abs(adx * cdy))
            + np.abs(cdx * cdx + cdy * cdy) * (np.abs(adx * bdy) + np.abs(bdx * ady)))
    suspect = np.nonzero(np.abs(det) <= 1e-9 * perm + 1.0)[0]
    for q in suspect:
        ia, ib, ic, id_ = int(a[q]), int(b[q]), int(c[q]), int(d[q])
        pa, pb, pc, pd = (tuple(int(v) for v in xy[i]) for i in (ia, ib, ic, id_))
        if _incircle_exact(pa, pb, pc, pd) == 0:
            quads.append((ia, ib, ic, id_))
    return quads


def enforce_general_position(xy: np.ndarray, seed: int, box: int = WORLD,
                             max_rounds: int = 50) -> np.ndarray:
    """Redraw sites until no four of them lie on one empty circle (exact test).

    One site of every co-circular quadruple is replaced by a fresh uniform
    draw (distinct from all others) and the test is repeated.
    """
    xy = xy.copy()
    start = 0
    for _ in range(max_rounds):
        quads = _cocircular_quads(xy)
        if not quads:
            return xy
        taken = set((int(x) << 21) | int(y) for x, y in xy)
        for q in quads:
            i = q[3]
            while True:
                wx = splitmix64(seed, 90, 1, start)
                wy = splitmix64(seed, 91, 1, start)
                start += 1
                nx = int(_uniform_int(wx, 1, box - 1)[0])
                ny = int(_uniform_int(wy, 1, box - 1)[0])
                if ((nx << 21) | ny) not in taken:
                    break
            taken.add((nx << 21) | ny)
            xy[i] = (nx, ny)
    raise RuntimeError("general position not reached")


def lattice_sites(k: int, spacing: int, offset: int) -> np.ndarray:
    """k x k lattice: sites at (offset + i*spacing, offset + j*spacing)."""
    i, j = np.meshgrid(np.arange(k), np.arange(k), indexing="ij")
    return np.stack([offset + i.ravel() * spacing, offset + j.ravel() * spacing], axis=1).astype(np.int32)


def batch_sets(n_sets: int = 4096, seed: int = SEED_BASE + 4, lo: int = 16, hi: int = 65536,
               box: int = WORLD):
    """Independent point sets of log-uniform size in [lo, hi].

    Even-numbered sets are uniform, odd-numbered sets are Gaussian mixtures
    (64 components, sigma 2^12, Dirichlet(1) weights).  Returns
    (sites int32[S,2] concatenated, set_ptr int64[n_sets+1]).
    """
    w = _unit_open(splitmix64(seed, 20, n_sets))
    sizes = np.floor(np.exp(np.log(lo) + w * (np.log(hi) - np.log(lo)))).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    parts = []
    for s in range(n_sets):
        if s % 2 == 0:
            parts.append(uniform_sites(int(sizes[s]), seed=seed * 8192 + s, box=box))
        else:
            parts.append(gaussian_mixture_sites(int(sizes[s]), seed=seed * 8192 + s, box=box))
    ptr = np.zeros(n_sets + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(sizes)
    return np.concatenate(parts).astype(np.int32), ptr


def poisson_requests(n_req: int, rate_per_s: float, seed: int = SEED_BASE + 5,
                     lo: int = 100, hi: int = 1_000_000):
    """A Poisson stream: arrival times (s), sizes (log-uniform), kind (0 uniform, 1 clustered)."""
    gaps = -np.log(_unit_open(splitmix64(seed, 30, n_req))) / rate_per_s
    arrivals = np.cumsum(gaps)
    w = _unit_open(splitmix64(seed, 31, n_req))
    sizes = np.floor(np.exp(np.log(lo) + w * (np.log(hi) - np.log(lo)))).astype(np.int64)
    kind = (splitmix64(seed, 32, n_req) >> np.uint64(63)).astype(np.int64)
    return arrivals, np.clip(sizes, lo, hi), kind


# ------------------------------------------------------------------ workloads

def _cache_dir():
    import os
    import tempfile
    d = os.path.join(tempfile.gettempdir(), "vor_synth_cache")
    os.makedirs(d, exist_ok=True)
    return d


def workload(name: str, cache: bool = True) -> np.ndarray:
    """The named site sets of the benchmark and the parity tests.

    ``uniform_1k``  n = 1,000 uniform sites, no four on an empty circle
    ``uniform_1m``  n = 1,048,576 uniform sites, no four on an empty circle
    ``gauss_4m``    n = 4,194,304 sites of the 64-component Gaussian mixture
                    (sigma = 2^12, Dirichlet(1) weights); co-circular sites allowed
    All live in the world X = [0, 2^20]^2.
    """
    import os
    spec = {
        "uniform_1k": (1000, "u", True, SEED_BASE + 1),
        "uniform_1m": (1 << 20, "u", True, SEED_BASE + 2),
        "gauss_4m": (1 << 22, "g", False, SEED_BASE + 3),
    }
    n, kind, gp, seed = spec[name]
    path = os.path.join(_cache_dir(), f"{name}_{seed}.npy") if cache else None
    if path and os.path.exists(path):
        xy = np.load(path)
        if xy.shape == (n, 2):
            return xy
    xy = uniform_sites(n, seed=seed) if kind == "u" else gaussian_mixture_sites(n, seed=seed)
    if gp:
        xy = enforce_general_position(xy, seed=seed)
    if path:
        tmp = path + f".{os.getpid()}.npy"
        np.save(tmp, xy)
        os.replace(tmp, path)
    return xy


def batch_workload(cache: bool = True):
    """The batched workload: 4,096 sets of log-uniform size in [16, 65,536],
    even sets uniform, odd sets Gaussian mixtures, all in [0, 2^20]^2.
    Returns (sites int32[N,2], set_ptr int64[4097])."""
    import os
    seed = SEED_BASE + 4
    path = os.path.join(_cache_dir(), f"batch_4096_{seed}.npz") if cache else None
    if path and os.path.exists(path):
        d = np.load(path)
        return d["xy"], d["ptr"]
    xy, ptr = batch_sets(n_sets=4096, seed=seed)
    if path:
        tmp = path + f".{os.getpid()}.npz"
        np.savez(tmp, xy=xy, ptr=ptr)
        os.replace(tmp, path)
    return xy, ptr


def serve_pools(cache: bool = True):
    """Site pools of the serving workload: 2^21 uniform and 2^21 Gaussian
    mixture sites in [0, 2^20]^2, in random order, so that a contiguous
    slice of a pool is a random sample of its distribution."""
    import os
    seed = SEED_BASE + 6
    path = os.path.join(_cache_dir(), f"serve_pools_{seed}.npz") if cache else None
    if path and os.path.exists(path):
        d = np.load(path)
        return d["uniform"], d["clustered"]
    u = uniform_sites(1 << 21, seed=seed)
    g = gaussian_mixture_sites(1 << 21, seed=seed + 1)
    if path:
        tmp = path + f".{os.getpid()}.npz"
        np.savez(tmp, uniform=u, clustered=g)
        os.replace(tmp, path)
    return u, g


def serve_request(j: int, size: int, kind: int, pools, seed: int = SEED_BASE + 7) -> np.ndarray:
    """Request j of the serving workload: `size` sites, a contiguous slice of
    the uniform (kind 0) or clustered (kind 1) pool at a seeded offset."""
    pool = pools[int(kind)]
    span = pool.shape[0] - int(size)
    off = int(splitmix64(seed, 40, 1, j)[0] % np.uint64(span + 1))
    return pool[off:off + int(size)]
