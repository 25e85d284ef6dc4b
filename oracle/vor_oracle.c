/*
 * vor_oracle.c -- plain, slow, exact CPU oracle of the projector algorithm.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * What it computes (D. Reem, "The projector algorithm: a simple parallel
 * algorithm for computing Voronoi diagrams and Delaunay graphs"):
 *
 *   - the Voronoi cell R_k of Definition 2.1 of every integer site p_k inside
 *     the rectangle X = [0,W] x [0,H], as the ordered list of lines that carry
 *     a positive-length edge of R_k (a neighbour site j >= 0, or a side of X:
 *     -1 bottom, -2 right, -3 top, -4 left) and the vertices between
 *     consecutive edges (Section 5);
 *   - the Delaunay graph restricted to X (Section 6).
 *
 * It does so by running Algorithm 1 (Section 4) literally for each cell,
 * with EdgeQueue kept as a LIFO list, and it finds each ray endpoint
 * T(p, theta) of eq. (2.1) either
 *   - "plain":    Method 4.1 in the single pass of Remark A.2 (every site is
 *                 compared once with the moving point y), starting from the
 *                 boundary point of eq. (A.1)/(A.2), or
 *   - "bucketed": Method A.6 over the buckets of Method A.5, with the
 *                 rectangular list of sites (with deletion), the probe
 *                 y = p + eta*theta, the square S_I[y, 2 beta s] and the
 *                 shell-by-shell scan of Remark A.7(ii).
 * Ties at an endpoint (the ray meets a vertex) are resolved as Remark A.4
 * prescribes: among the equidistant sites the two with extreme angles carry
 * the cell's edges.  All decisions use exact integer arithmetic (64- and
 * 128-bit); no floating point decides anything.
 *
 * Readings of points the paper leaves open (each one is listed in the design
 * notes of the repository):
 *   1. Projector corners: integer directions (2,-1), (0,1), (-2,-1) instead
 *      of the irrational unit vectors of Section 4; every projector yields the
 *      same cell.
 *   2. Directions are kept as unnormalised integer vectors; theta_3 of
 *      Algorithm 1 is u - p (or p - u, or a line direction) scaled by the
 *      common denominator, which does not change the ray.
 *   3. EdgeQueue is LIFO ("the highest (first) subedge").
 *   4. Remark A.4 lets either extreme site represent a vertex endpoint; the
 *      oracle keeps both and uses, for a subedge {theta_1, theta_2} taken
 *      counter-clockwise, the extreme that faces the subwedge: the most
 *      counter-clockwise one at theta_1 and the most clockwise one at theta_2.
 *   5. The cell is closed (Definition 2.1): "in the wedge" and "inside the
 *      cell" both accept equality.
 *   6. A side of X is represented by the reflection of p across it (a
 *      "mirror site"): the bisector of p and its mirror is exactly that side,
 *      so eq. (A.1) is the bisector formula.
 *   7. Method A.6 with exact rational points: the probe lies on the ray at a
 *      distance between eta and sqrt(2)*eta (eta an integer upper bound of
 *      4 sqrt(2) (beta + 1.01) s), and every S_I[y, d(p,y)] window is the
 *      exact integer rectangle of eq. (A.3) for an integer upper bound of the
 *      centre's coordinates and of d(p,y).  A larger window only adds
 *      comparisons (Lemma SitesInLargeSquare holds for any superset).
 *
 * Geometry in coordinates relative to p: a line is { v : 2<n, v> = c } with
 *   site a:   n = a - p,            c = |n|^2        (the bisector of p and a)
 *   side:     n = (mirror - p) / 2, c = 2 |n|^2      (the side itself)
 * so a ray p + t*theta meets the line at t = c / (2 <n, theta>) when
 * <n, theta> > 0.  |n| < 2^20 and c < 2^41, and every direction component is
 * below 2^62, so every product below fits in a signed 128-bit integer.
 */

#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

typedef __int128 i128;
typedef int64_t i64;

#define ORC_OK 0
#define ORC_E_ARG (-1)
#define ORC_E_OUTSIDE (-2)
#define ORC_E_DUPLICATE (-3)
#define ORC_E_BOX (-4)
#define ORC_E_NOMEM (-5)
#define ORC_E_INTERNAL (-9)

#define SIDE_BOTTOM (-1)
#define SIDE_RIGHT (-2)
#define SIDE_TOP (-3)
#define SIDE_LEFT (-4)

#define MODE_PLAIN 0
#define MODE_BUCKETED 1

/* per-cell counters */
enum {
    ST_RAYS = 0,        /* rays shot: the 3 projector corners + one per split   */
    ST_NODES,           /* nodes of the algorithm tree (start node + subedges)  */
    ST_ENDPOINTS,       /* endpoint computations (two per subedge, Alg. 1)      */
    ST_COMPARISONS,     /* distance comparisons d(y,a) vs d(y,p)                */
    ST_VERTICES,        /* vertices stored by Algorithm 1                       */
    ST_DEGENERATE,      /* vertices of the cell lying on more than two lines    */
    ST_EDGES,           /* e_k                                                  */
    ST_REPEAT_HITS,     /* rays violating Lemma IntermediateRay (must stay 0)   */
    ST_N
};

typedef struct { i64 x, y; } dir_t;
typedef struct { i64 nx, ny, c; int32_t label; } line_t;
typedef struct { i128 tn, td; } tpar_t;               /* t = tn / td, td > 0 */
typedef struct { int32_t ccw, cw; tpar_t t; int32_t ties; } endpoint_t;

typedef struct {
    const int32_t *xy;
    i64 n, W, H;
    int mode;
    /* Method A.5 buckets */
    i64 s, m1, m2;
    i64 *bstart, *bsite;
    i64 eta, beta;
} world_t;

typedef struct { i64 ray_a, ray_b; int wedge; } subedge_t;
typedef struct { dir_t th; int wedge; int initial; int done; int32_t label; int32_t tie; } ray_t;
typedef struct { int32_t l1, l2; i64 nx, ny, d; } vstore_t;

typedef struct {
    int32_t *stamp;       /* deletion marks of the rectangular list (bucketed) */
    int32_t gen;
    subedge_t *stack; i64 stack_cap;
    ray_t *rays; i64 rays_cap;
    int32_t *edges; i64 edges_n, edges_cap;
    vstore_t *verts; i64 verts_n, verts_cap;
    int32_t *ties; i64 ties_cap;
    i64 *shell; i64 shell_cap;
} work_t;

/* ------------------------------------------------------------------ */
/* small exact helpers                                                 */
/* ------------------------------------------------------------------ */

static i128 dot(const line_t *L, dir_t th) { return (i128)L->nx * th.x + (i128)L->ny * th.y; }
static i128 crossd(dir_t a, dir_t b) { return (i128)a.x * b.y - (i128)a.y * b.x; }

static i128 floordiv128(i128 a, i128 b) {   /* b > 0 */
    i128 q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

static i128 ceildiv128(i128 a, i128 b) {    /* b > 0 */
    return -floordiv128(-a, b);
}

static i64 isqrt_ceil(i128 v) {              /* smallest r >= 0 with r*r >= v */
    if (v <= 0) return 0;
    i64 r = (i64)sqrtl((long double)v);
    while ((i128)r * r < v) r++;
    while (r > 0 && (i128)(r - 1) * (r - 1) >= v) r--;
    return r;
}

static line_t line_of(const world_t *w, i64 px, i64 py, int32_t label) {
    line_t L;
    L.label = label;
    if (label >= 0) {
        L.nx = (i64)w->xy[2 * label] - px;
        L.ny = (i64)w->xy[2 * label + 1] - py;
        L.c = L.nx * L.nx + L.ny * L.ny;
    } else {
        switch (label) {
        case SIDE_BOTTOM: L.nx = 0; L.ny = -py; break;
        case SIDE_RIGHT:  L.nx = w->W - px; L.ny = 0; break;
        case SIDE_TOP:    L.nx = 0; L.ny = w->H - py; break;
        default:          L.nx = -px; L.ny = 0; break;
        }
        L.c = 2 * (L.nx * L.nx + L.ny * L.ny);
    }
    return L;
}

/* y = p + t*theta is strictly closer to the line's site than to p, i.e. y is
 * strictly beyond the line:  2 t <n, theta> > c. */
static int beyond(const line_t *L, dir_t th, tpar_t t) {
    return 2 * t.tn * dot(L, th) > (i128)L->c * t.td;
}

/* y = p + t*theta lies on the line (d(y,a) = d(y,p)) and the ray crosses it. */
static int on_line(const line_t *L, dir_t th, tpar_t t) {
    i128 d = dot(L, th);
    return d > 0 && 2 * t.tn * d == (i128)L->c * t.td;
}

static tpar_t hit_t(const line_t *L, dir_t th) {
    tpar_t t; t.tn = L->c; t.td = 2 * dot(L, th); return t;
}

static int tless(tpar_t a, tpar_t b) { return a.tn * b.td < b.tn * a.td; }

/* a is strictly more counter-clockwise than b (both normals lie in one open
 * half-plane, so the cross product orders them). */
static int more_ccw(const line_t *a, const line_t *b) {
    return (i128)b->nx * a->ny - (i128)b->ny * a->nx > 0;
}

#define GROW(ptr, cap, need, type)                                            \
    do {                                                                      \
        if ((need) > (cap)) {                                                 \
            i64 nc_ = (cap) ? 2 * (cap) : 64;                                 \
            while (nc_ < (need)) nc_ *= 2;                                    \
            type *np_ = (type *)realloc((ptr), (size_t)nc_ * sizeof(type));   \
            if (!np_) return ORC_E_NOMEM;                                     \
            (ptr) = np_; (cap) = nc_;                                         \
        }                                                                     \
    } while (0)

/* Remark A.4: from the equidistant lines keep the two extreme ones. */
static void extremes(const world_t *w, i64 px, i64 py, const int32_t *ties, i64 nt,
                     endpoint_t *e) {
    line_t best_ccw = line_of(w, px, py, ties[0]);
    line_t best_cw = best_ccw;
    for (i64 i = 1; i < nt; i++) {
        line_t L = line_of(w, px, py, ties[i]);
        if (more_ccw(&L, &best_ccw)) best_ccw = L;
        if (more_ccw(&best_cw, &L)) best_cw = L;
    }
    e->ccw = best_ccw.label;
    e->cw = best_cw.label;
    e->ties = (int32_t)nt;
}

/* ------------------------------------------------------------------ */
/* Endpoint, plain: Method 4.1 in the single pass of Remark A.2         */
/* ------------------------------------------------------------------ */

static int endpoint_plain(const world_t *w, work_t *wk, i64 k, dir_t th, endpoint_t *out,
                          i64 *cmp) {
    const i64 px = w->xy[2 * k], py = w->xy[2 * k + 1];
    /* Step 1: y := the point where the ray leaves X, eq. (A.1)/(A.2): the
     * first side with <N_j, theta> > 0 met by the ray. */
    tpar_t t; t.tn = 0; t.td = 0;
    int32_t lab = 0;
    for (int32_t s = -1; s >= -4; s--) {
        line_t L = line_of(w, px, py, s);
        if (dot(&L, th) <= 0) continue;
        tpar_t ts = hit_t(&L, th);
        if (t.td == 0 || tless(ts, t)) { t = ts; lab = s; }
    }
    if (t.td == 0) return ORC_E_INTERNAL;
    /* Steps 2-6, single pass: whenever y is closer to a site a than to p,
     * move y to the intersection of the ray with the bisector of p and a. */
    for (i64 j = 0; j < w->n; j++) {
        if (j == k) continue;
        line_t L = line_of(w, px, py, (int32_t)j);
        (*cmp)++;
        if (beyond(&L, th, t)) { t = hit_t(&L, th); lab = (int32_t)j; }
    }
    /* Remark A.4: the sites equidistant from the final y (and sides through
     * y) form EquiDistList. */
    i64 nt = 0;
    GROW(wk->ties, wk->ties_cap, 8, int32_t);
    for (int32_t s = -1; s >= -4; s--) {
        line_t L = line_of(w, px, py, s);
        if (on_line(&L, th, t)) wk->ties[nt++] = s;
    }
    for (i64 j = 0; j < w->n; j++) {
        if (j == k) continue;
        line_t L = line_of(w, px, py, (int32_t)j);
        (*cmp)++;
        if (beyond(&L, th, t)) return ORC_E_INTERNAL;   /* y must be in the cell */
        if (on_line(&L, th, t)) {
            GROW(wk->ties, wk->ties_cap, nt + 1, int32_t);
            wk->ties[nt++] = (int32_t)j;
        }
    }
    if (nt == 0) return ORC_E_INTERNAL;
    (void)lab;
    out->t = t;
    extremes(w, px, py, wk->ties, nt, out);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Endpoint, bucketed: Method A.6                                       */
/* ------------------------------------------------------------------ */

/* Bucket index range of the integer rectangle S_I[y, r] (eq. (A.3)) for the
 * point y = p + theta * tn / td and any r with r <= rup, clamped to the grid
 * (buckets outside the grid are the empty shell of Method A.5). */
typedef struct { i64 x0, x1, y0, y1; } brect_t;

static brect_t window_of(const world_t *w, i64 px, i64 py, dir_t th, tpar_t t, i64 rup) {
    /* integer bounds of y's coordinates */
    i128 ax = (i128)th.x * t.tn, ay = (i128)th.y * t.tn;
    i128 ylo_x = px + floordiv128(ax, t.td), yhi_x = px + ceildiv128(ax, t.td);
    i128 ylo_y = py + floordiv128(ay, t.td), yhi_y = py + ceildiv128(ay, t.td);
    brect_t b;
    b.x0 = (i64)floordiv128(ylo_x - rup, w->s);
    b.x1 = (i64)floordiv128(yhi_x + rup, w->s);
    b.y0 = (i64)floordiv128(ylo_y - rup, w->s);
    b.y1 = (i64)floordiv128(yhi_y + rup, w->s);
    if (b.x0 < 0) b.x0 = 0;
    if (b.y0 < 0) b.y0 = 0;
    if (b.x1 > w->m1 - 1) b.x1 = w->m1 - 1;
    if (b.y1 > w->m2 - 1) b.y1 = w->m2 - 1;
    return b;
}

/* integer upper bound of d(p, y) for y = p + theta * tn / td */
static i64 dist_up(dir_t th, tpar_t t) {
    i128 ax = (i128)(th.x < 0 ? -th.x : th.x) * t.tn, ay = (i128)(th.y < 0 ? -th.y : th.y) * t.tn;
    i128 cx = ceildiv128(ax, t.td), cy = ceildiv128(ay, t.td);
    return isqrt_ceil(cx * cx + cy * cy);
}

static brect_t brect_and(brect_t a, brect_t b) {
    brect_t r;
    r.x0 = a.x0 > b.x0 ? a.x0 : b.x0; r.x1 = a.x1 < b.x1 ? a.x1 : b.x1;
    r.y0 = a.y0 > b.y0 ? a.y0 : b.y0; r.y1 = a.y1 < b.y1 ? a.y1 : b.y1;
    return r;
}

/* Remark A.7(ii): the buckets of the rectangle r in shells around (cx, cy).
 * Fills wk->shell with bucket ids; returns the count (or an error). */
static i64 shell_order(const world_t *w, work_t *wk, brect_t r, i64 cx, i64 cy) {
    if (r.x0 > r.x1 || r.y0 > r.y1) return 0;
    i64 cnt = (r.x1 - r.x0 + 1) * (r.y1 - r.y0 + 1);
    GROW(wk->shell, wk->shell_cap, cnt, i64);
    i64 rmax = 0;
    i64 d;
    d = cx - r.x0; if (d > rmax) rmax = d;
    d = r.x1 - cx; if (d > rmax) rmax = d;
    d = cy - r.y0; if (d > rmax) rmax = d;
    d = r.y1 - cy; if (d > rmax) rmax = d;
    i64 m = 0;
    for (i64 sh = 0; sh <= rmax && m < cnt; sh++) {
        for (i64 by = cy - sh; by <= cy + sh; by++) {
            if (by < r.y0 || by > r.y1) continue;
            int edge_row = (by == cy - sh || by == cy + sh);
            for (i64 bx = cx - sh; bx <= cx + sh; bx += (edge_row || sh == 0) ? 1 : 2 * sh) {
                if (bx >= r.x0 && bx <= r.x1) wk->shell[m++] = by * w->m1 + bx;
            }
        }
    }
    return m;
}

static i64 bucket_coord(const world_t *w, i64 px, dir_t th, i64 thc, tpar_t t) {
    (void)th;
    i128 a = (i128)thc * t.tn;
    i128 y = px + floordiv128(a, t.td);
    i64 b = (i64)floordiv128(y, w->s);
    if (b < 0) b = 0;
    return b;
}

static int endpoint_bucketed(const world_t *w, work_t *wk, i64 k, dir_t th, endpoint_t *out,
                             i64 *cmp) {
    const i64 px = w->xy[2 * k], py = w->xy[2 * k + 1];
    /* y_X: the point where the ray leaves X (Remark A.1, eq. (A.1)/(A.2)) */
    tpar_t tX; tX.tn = 0; tX.td = 0;
    int32_t labX = 0;
    for (int32_t s = -1; s >= -4; s--) {
        line_t L = line_of(w, px, py, s);
        if (dot(&L, th) <= 0) continue;
        tpar_t ts = hit_t(&L, th);
        if (tX.td == 0 || tless(ts, tX)) { tX = ts; labX = s; }
    }
    if (tX.td == 0) return ORC_E_INTERNAL;

    /* Step 1: the probe y = p + eta * theta / |theta|_inf */
    i64 thinf = th.x < 0 ? -th.x : th.x;
    i64 ay_ = th.y < 0 ? -th.y : th.y;
    if (ay_ > thinf) thinf = ay_;
    tpar_t t; t.tn = w->eta; t.td = thinf;
    int outside = 0;
    int32_t lab = labX;
    /* Steps 2-3: if y is not in X, y := y_X */
    if (!tless(t, tX) && !(t.tn * tX.td == tX.tn * t.td)) {
        t = tX;
    } else {
        /* Step 4: compare with every site in S_I[y, 2 beta s] */
        brect_t r = window_of(w, px, py, th, t, 2 * w->beta * w->s);
        i64 cx = bucket_coord(w, px, th, th.x, t), cy = bucket_coord(w, py, th, th.y, t);
        if (cx > w->m1 - 1) cx = w->m1 - 1;
        if (cy > w->m2 - 1) cy = w->m2 - 1;
        i64 nb = shell_order(w, wk, r, cx, cy);
        if (nb < 0) return (int)nb;
        for (i64 q = 0; q < nb && !outside; q++) {
            i64 b = wk->shell[q];
            for (i64 i = w->bstart[b]; i < w->bstart[b + 1]; i++) {
                i64 j = w->bsite[i];
                if (j == k) continue;
                line_t L = line_of(w, px, py, (int32_t)j);
                (*cmp)++;
                if (beyond(&L, th, t)) { outside = 1; lab = (int32_t)j; break; }
            }
        }
        if (!outside) t = tX;
    }
    /* Step 5: the rectangular list of sites: S_I[y~, d(p, y~)] */
    brect_t rect = window_of(w, px, py, th, t, dist_up(th, t));
    wk->gen++;
    if (wk->gen == 0x7fffffff) { memset(wk->stamp, 0, (size_t)w->n * sizeof(int32_t)); wk->gen = 1; }
    /* Step 6 */
    if (outside) {
        /* Steps 9-11: move y to the bisector of p and CloseNeighbor */
        line_t L = line_of(w, px, py, lab);
        t = hit_t(&L, th);
    } else {
        lab = labX;
    }
    /* Step 7 loop */
    int32_t *eq = NULL; i64 neq = 0, eqcap = 0;
    for (;;) {
        brect_t r = brect_and(window_of(w, px, py, th, t, dist_up(th, t)), rect);
        i64 cx = bucket_coord(w, px, th, th.x, t), cy = bucket_coord(w, py, th, th.y, t);
        if (cx > w->m1 - 1) cx = w->m1 - 1;
        if (cy > w->m2 - 1) cy = w->m2 - 1;
        i64 nb = shell_order(w, wk, r, cx, cy);
        if (nb < 0) { free(eq); return (int)nb; }
        int moved = 0;
        neq = 0;
        for (i64 q = 0; q < nb && !moved; q++) {
            i64 b = wk->shell[q];
            for (i64 i = w->bstart[b]; i < w->bstart[b + 1]; i++) {
                i64 j = w->bsite[i];
                if (j == k || wk->stamp[j] == wk->gen) continue;
                wk->stamp[j] = wk->gen;          /* removed from the rectangular list */
                line_t L = line_of(w, px, py, (int32_t)j);
                (*cmp)++;
                if (beyond(&L, th, t)) {         /* Step 9: CloseNeighbor := a */
                    t = hit_t(&L, th);           /* Steps 10-11 */
                    lab = (int32_t)j;
                    moved = 1;
                    break;
                }
                if (on_line(&L, th, t)) {
                    if (neq + 1 > eqcap) {
                        eqcap = eqcap ? 2 * eqcap : 8;
                        int32_t *ne = (int32_t *)realloc(eq, (size_t)eqcap * sizeof(int32_t));
                        if (!ne) { free(eq); return ORC_E_NOMEM; }
                        eq = ne;
                    }
                    eq[neq++] = (int32_t)j;
                }
            }
        }
        if (!moved) break;                       /* Step 8: y is the endpoint */
    }
    /* EquiDistList (Remark A.4): the line y was last moved to, the sites found
     * equidistant in the last pass, and the sides through y. */
    i64 nt = 0;
    GROW(wk->ties, wk->ties_cap, neq + 5, int32_t);
    for (int32_t s = -1; s >= -4; s--) {
        line_t L = line_of(w, px, py, s);
        if (on_line(&L, th, t)) wk->ties[nt++] = s;
    }
    if (lab >= 0) wk->ties[nt++] = lab;
    for (i64 i = 0; i < neq; i++) if (eq[i] != lab) wk->ties[nt++] = eq[i];
    free(eq);
    if (nt == 0) return ORC_E_INTERNAL;
    out->t = t;
    extremes(w, px, py, wk->ties, nt, out);
    return ORC_OK;
}

static int endpoint(const world_t *w, work_t *wk, i64 k, dir_t th, endpoint_t *out, i64 *cmp) {
    return w->mode == MODE_BUCKETED ? endpoint_bucketed(w, wk, k, th, out, cmp)
                                    : endpoint_plain(w, wk, k, th, out, cmp);
}

/* ------------------------------------------------------------------ */
/* "u is inside the cell" (Algorithm 1): u = p + N/D                    */
/* ------------------------------------------------------------------ */

/* Line L is strictly violated by u:  2 <n, N> / D > c. Returns +1 when
 * violated, 0 when u lies on L, -1 when u is strictly inside. */
static int vs_point(const line_t *L, i64 Nx, i64 Ny, i64 D) {
    i128 lhs = 2 * ((i128)L->nx * Nx + (i128)L->ny * Ny);
    i128 rhs = (i128)L->c * D;
    if (D < 0) { lhs = -lhs; rhs = -rhs; }
    return lhs > rhs ? 1 : (lhs == rhs ? 0 : -1);
}

/* Visit every line that can matter at u: all sites (plain) or the sites of
 * S_I[u, d(p,u)] (bucketed, Lemma SitesInLargeSquare), plus the 4 sides.
 * Returns 1 if u is in the cell, 0 if not; counts the lines through u other
 * than skip1/skip2 in *through. */
static int point_in_cell(const world_t *w, work_t *wk, i64 k, i64 Nx, i64 Ny, i64 D,
                         int32_t skip1, int32_t skip2, i64 *through, i64 *cmp, int stop_early) {
    const i64 px = w->xy[2 * k], py = w->xy[2 * k + 1];
    int inside = 1;
    *through = 0;
    for (int32_t s = -1; s >= -4; s--) {
        line_t L = line_of(w, px, py, s);
        int v = vs_point(&L, Nx, Ny, D);
        if (v > 0) { inside = 0; if (stop_early) return 0; }
        if (v == 0 && s != skip1 && s != skip2) (*through)++;
    }
    if (w->mode == MODE_PLAIN) {
        for (i64 j = 0; j < w->n; j++) {
            if (j == k) continue;
            line_t L = line_of(w, px, py, (int32_t)j);
            (*cmp)++;
            int v = vs_point(&L, Nx, Ny, D);
            if (v > 0) { inside = 0; if (stop_early) return 0; }
            if (v == 0 && j != skip1 && j != skip2) (*through)++;
        }
        return inside;
    }
    /* bucketed: the point u as p + theta * tn / td with theta = N, t = 1/D */
    dir_t th; th.x = Nx; th.y = Ny;
    tpar_t t; t.tn = 1; t.td = D;
    if (D < 0) { th.x = -Nx; th.y = -Ny; t.td = -D; }
    brect_t r = window_of(w, px, py, th, t, dist_up(th, t));
    for (i64 by = r.y0; by <= r.y1; by++) {
        for (i64 bx = r.x0; bx <= r.x1; bx++) {
            i64 b = by * w->m1 + bx;
            for (i64 i = w->bstart[b]; i < w->bstart[b + 1]; i++) {
                i64 j = w->bsite[i];
                if (j == k) continue;
                line_t L = line_of(w, px, py, (int32_t)j);
                (*cmp)++;
                int v = vs_point(&L, Nx, Ny, D);
                if (v > 0) { inside = 0; if (stop_early) return 0; }
                if (v == 0 && j != skip1 && j != skip2) (*through)++;
            }
        }
    }
    (void)wk;
    return inside;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 for one cell                                             */
/* ------------------------------------------------------------------ */

/* Intersection u of two lines: u - p = N / D with
 *   N = (c1 n2y - c2 n1y, c2 n1x - c1 n2x),  D = 2 (n1x n2y - n1y n2x). */
static void intersect(const line_t *a, const line_t *b, i64 *Nx, i64 *Ny, i64 *D) {
    *Nx = a->c * b->ny - b->c * a->ny;
    *Ny = b->c * a->nx - a->c * b->nx;
    *D = 2 * (a->nx * b->ny - a->ny * b->nx);
}

static int half_of(i64 x, i64 y) { return (y > 0 || (y == 0 && x > 0)) ? 0 : 1; }

static int angle_less(const line_t *a, const line_t *b) {
    int ha = half_of(a->nx, a->ny), hb = half_of(b->nx, b->ny);
    if (ha != hb) return ha < hb;
    return (i128)a->nx * b->ny - (i128)a->ny * b->nx > 0;
}

static int add_edge(work_t *wk, int32_t lab) {
    for (i64 i = 0; i < wk->edges_n; i++) if (wk->edges[i] == lab) return ORC_OK;
    GROW(wk->edges, wk->edges_cap, wk->edges_n + 1, int32_t);
    wk->edges[wk->edges_n++] = lab;
    return ORC_OK;
}

typedef struct {
    int32_t *labels;   /* e_k labels, canonical order          */
    i64 *vnum;         /* 3 * e_k: (x numerator, y numerator, denominator) */
    i64 e;
    i64 st[ST_N];
} cellres_t;

static int in_wedge(dir_t a, dir_t b, dir_t v) { return crossd(a, v) >= 0 && crossd(v, b) >= 0; }

static int cell_run(const world_t *w, work_t *wk, i64 k, cellres_t *res) {
    const i64 px = w->xy[2 * k], py = w->xy[2 * k + 1];
    memset(res->st, 0, sizeof(res->st));
    i64 *st = res->st;
    i64 cmp = 0;
    wk->edges_n = 0;
    wk->verts_n = 0;

    /* The projector: corners psi_1, psi_2, psi_3 and its three edges. */
    const dir_t psi[3] = {{2, -1}, {0, 1}, {-2, -1}};
    i64 nrays = 0;
    GROW(wk->rays, wk->rays_cap, 3, ray_t);
    for (int i = 0; i < 3; i++) {
        wk->rays[i].th = psi[i]; wk->rays[i].wedge = -1; wk->rays[i].initial = 1;
        wk->rays[i].done = 0; wk->rays[i].label = 0; wk->rays[i].tie = 0;
    }
    nrays = 3;
    i64 sp = 0;
    GROW(wk->stack, wk->stack_cap, 3, subedge_t);
    /* EdgeQueue: {psi1,psi2} on top, then {psi2,psi3}, then {psi3,psi1} */
    wk->stack[sp].ray_a = 2; wk->stack[sp].ray_b = 0; wk->stack[sp].wedge = 2; sp++;
    wk->stack[sp].ray_a = 1; wk->stack[sp].ray_b = 2; wk->stack[sp].wedge = 1; sp++;
    wk->stack[sp].ray_a = 0; wk->stack[sp].ray_b = 1; wk->stack[sp].wedge = 0; sp++;
    st[ST_NODES] = 1;   /* the start node of the algorithm tree */

    while (sp > 0) {
        subedge_t se = wk->stack[--sp];
        st[ST_NODES]++;
        /* Lemma e_k: the tree of a cell has at most 2 e_k nodes, and a cell
         * has at most n - 1 + 4 edges; more nodes means a broken invariant. */
        if (st[ST_NODES] > 2 * (w->n + 4) + 8) return ORC_E_INTERNAL;
        dir_t t1 = wk->rays[se.ray_a].th, t2 = wk->rays[se.ray_b].th;
        endpoint_t e1, e2;
        int rc = endpoint(w, wk, k, t1, &e1, &cmp); if (rc) return rc;
        rc = endpoint(w, wk, k, t2, &e2, &cmp); if (rc) return rc;
        st[ST_ENDPOINTS] += 2;
        ray_t *ra = &wk->rays[se.ray_a], *rb = &wk->rays[se.ray_b];
        if (!ra->done) { ra->done = 1; ra->label = e1.ccw; ra->tie = e1.ties > 1; }
        if (!rb->done) { rb->done = 1; rb->label = e2.cw; rb->tie = e2.ties > 1; }
        int32_t L1 = e1.ccw, L2 = e2.cw;
        rc = add_edge(wk, L1); if (rc) return rc;
        rc = add_edge(wk, L2); if (rc) return rc;
        if (L1 == L2) continue;                       /* same line: no vertex here */
        line_t l1 = line_of(w, px, py, L1), l2 = line_of(w, px, py, L2);
        i64 Nx, Ny, D;
        intersect(&l1, &l2, &Nx, &Ny, &D);
        dir_t t3;
        if (D == 0) {
            /* parallel lines: theta_3 := the direction of the lines, turned into the wedge */
            t3.x = -l1.ny; t3.y = l1.nx;
            if (!in_wedge(t1, t2, t3)) { t3.x = -t3.x; t3.y = -t3.y; }
        } else {
            i64 sg = D > 0 ? 1 : -1;
            dir_t N; N.x = Nx; N.y = Ny;
            int inw = sg * crossd(t1, N) >= 0 && sg * crossd(N, t2) >= 0;  /* lambda >= 0 */
            if (inw) {
                i64 through;
                if (point_in_cell(w, wk, k, Nx, Ny, D, L1, L2, &through, &cmp, 1)) {
                    GROW(wk->verts, wk->verts_cap, wk->verts_n + 1, vstore_t);
                    vstore_t *v = &wk->verts[wk->verts_n++];
                    v->l1 = L1; v->l2 = L2; v->nx = Nx; v->ny = Ny; v->d = D;
                    continue;                           /* u is a vertex: store it */
                }
                t3.x = sg * Nx; t3.y = sg * Ny;         /* theta_3 := u - p */
            } else {
                t3.x = -sg * Nx; t3.y = -sg * Ny;       /* theta_3 := p - u */
            }
        }
        /* divide the subedge: {theta_1, theta_3} and {theta_3, theta_2} */
        GROW(wk->rays, wk->rays_cap, nrays + 1, ray_t);
        wk->rays[nrays].th = t3; wk->rays[nrays].wedge = se.wedge; wk->rays[nrays].initial = 0;
        wk->rays[nrays].done = 0; wk->rays[nrays].label = 0; wk->rays[nrays].tie = 0;
        GROW(wk->stack, wk->stack_cap, sp + 2, subedge_t);
        wk->stack[sp].ray_a = nrays; wk->stack[sp].ray_b = se.ray_b; wk->stack[sp].wedge = se.wedge; sp++;
        wk->stack[sp].ray_a = se.ray_a; wk->stack[sp].ray_b = nrays; wk->stack[sp].wedge = se.wedge; sp++;
        nrays++;
    }
    st[ST_RAYS] = nrays;
    st[ST_VERTICES] = wk->verts_n;

    /* Lemma IntermediateRay: within one initial wedge an intermediate ray hits
     * an edge that no other ray of that wedge hits (checked where no tie
     * makes "the edge" ambiguous). */
    for (i64 i = 3; i < nrays; i++) {
        ray_t *ri = &wk->rays[i];
        if (ri->tie || !ri->done) continue;
        int wdg = ri->wedge;
        int c0 = wdg, c1 = (wdg + 1) % 3;   /* boundary corners of the wedge */
        for (i64 j = 0; j < nrays; j++) {
            if (j == i) continue;
            ray_t *rj = &wk->rays[j];
            if (rj->tie || !rj->done) continue;
            int same_wedge = rj->initial ? (j == c0 || j == c1) : (rj->wedge == wdg);
            if (same_wedge && rj->label == ri->label) { st[ST_REPEAT_HITS]++; break; }
        }
    }

    /* Canonical form: edges in counter-clockwise order of their outward
     * normals, starting from the smallest polar angle in [0, 2 pi). */
    i64 e = wk->edges_n;
    line_t *ls = (line_t *)malloc((size_t)(e > 0 ? e : 1) * sizeof(line_t));
    if (!ls) return ORC_E_NOMEM;
    for (i64 i = 0; i < e; i++) ls[i] = line_of(w, px, py, wk->edges[i]);
    for (i64 i = 1; i < e; i++) {               /* insertion sort: e is small */
        line_t key = ls[i];
        i64 j = i - 1;
        while (j >= 0 && angle_less(&key, &ls[j])) { ls[j + 1] = ls[j]; j--; }
        ls[j + 1] = key;
    }
    res->labels = (int32_t *)malloc((size_t)(e > 0 ? e : 1) * sizeof(int32_t));
    res->vnum = (i64 *)malloc((size_t)(e > 0 ? e : 1) * 3 * sizeof(i64));
    if (!res->labels || !res->vnum) { free(ls); return ORC_E_NOMEM; }
    res->e = e;
    int rc = ORC_OK;
    for (i64 i = 0; i < e; i++) {
        res->labels[i] = ls[i].label;
        line_t *a = &ls[i], *b = &ls[(i + 1) % e];
        i64 Nx, Ny, D;
        intersect(a, b, &Nx, &Ny, &D);
        if (D == 0) { rc = ORC_E_INTERNAL; break; }
        /* every vertex lies in the cell, and more than two lines through it
         * make it degenerate */
        i64 through;
        if (!point_in_cell(w, wk, k, Nx, Ny, D, a->label, b->label, &through, &cmp, 0)) {
            rc = ORC_E_INTERNAL; break;
        }
        if (through > 0) st[ST_DEGENERATE]++;
        /* absolute coordinates: (p D + N) / D, the numerators lie in [0, W|D|] */
        uint64_t ux = (uint64_t)px * (uint64_t)D + (uint64_t)Nx;
        uint64_t uy = (uint64_t)py * (uint64_t)D + (uint64_t)Ny;
        res->vnum[3 * i] = (i64)ux;
        res->vnum[3 * i + 1] = (i64)uy;
        res->vnum[3 * i + 2] = D;
    }
    /* every vertex stored by Algorithm 1 is a vertex of the canonical polygon */
    for (i64 v = 0; v < wk->verts_n && rc == ORC_OK; v++) {
        vstore_t *sv = &wk->verts[v];
        int found = 0;
        for (i64 i = 0; i < e && !found; i++) {
            i64 Dv = res->vnum[3 * i + 2];
            i128 ax = (i128)res->vnum[3 * i] * sv->d, bx = ((i128)px * sv->d + sv->nx) * Dv;
            i128 ay = (i128)res->vnum[3 * i + 1] * sv->d, by = ((i128)py * sv->d + sv->ny) * Dv;
            if (ax == bx && ay == by) found = 1;
        }
        if (!found) rc = ORC_E_INTERNAL;
    }
    free(ls);
    st[ST_EDGES] = e;
    st[ST_COMPARISONS] = cmp;
    return rc;
}

/* ------------------------------------------------------------------ */
/* world set-up, validation, Method A.5 buckets                         */
/* ------------------------------------------------------------------ */

static int cmp_xy(const void *a, const void *b) {
    const int32_t *p = (const int32_t *)a, *q = (const int32_t *)b;
    if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
    if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
    return 0;
}

/* strict interior (Section 2) and distinct sites: lexicographic sort, then
 * adjacent comparison (Appendix 2, duplicate removal). */
static int validate(const int32_t *xy, i64 n, i64 W, i64 H) {
    if (n < 1) return ORC_E_ARG;
    if (W < 2 || H < 2 || W > (1 << 20) || H > (1 << 20)) return ORC_E_BOX;
    for (i64 i = 0; i < n; i++) {
        if (xy[2 * i] <= 0 || xy[2 * i] >= W || xy[2 * i + 1] <= 0 || xy[2 * i + 1] >= H)
            return ORC_E_OUTSIDE;
    }
    int32_t *c = (int32_t *)malloc((size_t)n * 2 * sizeof(int32_t));
    if (!c) return ORC_E_NOMEM;
    memcpy(c, xy, (size_t)n * 2 * sizeof(int32_t));
    qsort(c, (size_t)n, 2 * sizeof(int32_t), cmp_xy);
    int rc = ORC_OK;
    for (i64 i = 1; i < n; i++) if (c[2 * i] == c[2 * i - 2] && c[2 * i + 1] == c[2 * i - 1]) { rc = ORC_E_DUPLICATE; break; }
    free(c);
    return rc;
}

/* eta: the smallest integer with eta >= 4 sqrt(2) (beta + 1.01) s, i.e.
 * 10^4 eta^2 >= 32 (100 beta + 101)^2 s^2. */
static i64 eta_of(i64 beta, i64 s) {
    i128 v = (i128)32 * (100 * beta + 101) * (100 * beta + 101) * s * s;
    i64 e = (i64)ceill(sqrtl((long double)v / 10000.0L));
    while ((i128)10000 * e * e < v) e++;
    while (e > 0 && (i128)10000 * (e - 1) * (e - 1) >= v) e--;
    return e;
}

static int world_init(world_t *w, const int32_t *xy, i64 n, i64 W, i64 H, int mode, i64 s, i64 beta) {
    memset(w, 0, sizeof(*w));
    w->xy = xy; w->n = n; w->W = W; w->H = H; w->mode = mode;
    if (mode != MODE_BUCKETED) return ORC_OK;
    if (s < 1 || beta < 1) return ORC_E_ARG;
    w->s = s; w->beta = beta;
    w->m1 = (W + s - 1) / s; w->m2 = (H + s - 1) / s;
    w->eta = eta_of(beta, s);
    i64 m = w->m1 * w->m2;
    w->bstart = (i64 *)calloc((size_t)m + 1, sizeof(i64));
    w->bsite = (i64 *)malloc((size_t)n * sizeof(i64));
    if (!w->bstart || !w->bsite) return ORC_E_NOMEM;
    for (i64 i = 0; i < n; i++) {
        i64 b = (xy[2 * i + 1] / s) * w->m1 + xy[2 * i] / s;
        w->bstart[b + 1]++;
    }
    for (i64 b = 0; b < m; b++) w->bstart[b + 1] += w->bstart[b];
    i64 *fill = (i64 *)malloc((size_t)m * sizeof(i64));
    if (!fill) return ORC_E_NOMEM;
    memcpy(fill, w->bstart, (size_t)m * sizeof(i64));
    for (i64 i = 0; i < n; i++) {
        i64 b = (xy[2 * i + 1] / s) * w->m1 + xy[2 * i] / s;
        w->bsite[fill[b]++] = i;
    }
    free(fill);
    return ORC_OK;
}

static void world_free(world_t *w) { free(w->bstart); free(w->bsite); }

static int work_init(work_t *wk, const world_t *w) {
    memset(wk, 0, sizeof(*wk));
    if (w->mode == MODE_BUCKETED) {
        wk->stamp = (int32_t *)calloc((size_t)w->n, sizeof(int32_t));
        if (!wk->stamp) return ORC_E_NOMEM;
    }
    return ORC_OK;
}

static void work_free(work_t *wk) {
    free(wk->stamp); free(wk->stack); free(wk->rays); free(wk->edges);
    free(wk->verts); free(wk->ties); free(wk->shell);
}

/* ------------------------------------------------------------------ */
/* exported: whole diagram (or a list of cells), multithreaded          */
/* ------------------------------------------------------------------ */

typedef struct {
    i64 n_sel;
    i64 *sel;            /* selected cells (NULL: all) */
    cellres_t *cells;
    i64 n_edges, n_del;
    int err;
} orc_result;

typedef struct {
    const world_t *w;
    orc_result *r;
    i64 next;
    pthread_mutex_t mu;
    int err;
} job_t;

static void *worker(void *arg) {
    job_t *job = (job_t *)arg;
    work_t wk;
    int rc = work_init(&wk, job->w);
    for (;;) {
        pthread_mutex_lock(&job->mu);
        i64 i = job->next;
        if (i < job->r->n_sel && job->err == ORC_OK && rc == ORC_OK) job->next += 16;
        else i = job->r->n_sel;
        pthread_mutex_unlock(&job->mu);
        if (rc != ORC_OK || i >= job->r->n_sel) break;
        i64 hi = i + 16 < job->r->n_sel ? i + 16 : job->r->n_sel;
        for (; i < hi; i++) {
            i64 k = job->r->sel ? job->r->sel[i] : i;
            int crc = cell_run(job->w, &wk, k, &job->r->cells[i]);
            if (crc != ORC_OK) { rc = crc; break; }
        }
    }
    if (rc != ORC_OK) {
        pthread_mutex_lock(&job->mu);
        if (job->err == ORC_OK) job->err = rc;
        pthread_mutex_unlock(&job->mu);
    }
    work_free(&wk);
    return NULL;
}

/* Build the cells listed in sel[0..n_sel) (sel == NULL: all n cells).
 * mode 0 = plain (Method 4.1), 1 = bucketed (Method A.6, bucket side s, beta).
 * Returns an opaque result; *err receives the status. */
void *orc_build(const int32_t *xy, i64 n, i64 W, i64 H, int mode, i64 s, i64 beta,
                const i64 *sel, i64 n_sel, int nthreads, int *err) {
    int rc = validate(xy, n, W, H);
    if (rc) { *err = rc; return NULL; }
    world_t w;
    rc = world_init(&w, xy, n, W, H, mode, s, beta);
    if (rc) { world_free(&w); *err = rc; return NULL; }
    orc_result *r = (orc_result *)calloc(1, sizeof(orc_result));
    if (!r) { world_free(&w); *err = ORC_E_NOMEM; return NULL; }
    r->n_sel = sel ? n_sel : n;
    if (sel) {
        r->sel = (i64 *)malloc((size_t)(n_sel > 0 ? n_sel : 1) * sizeof(i64));
        if (!r->sel) { free(r); world_free(&w); *err = ORC_E_NOMEM; return NULL; }
        for (i64 i = 0; i < n_sel; i++) {
            if (sel[i] < 0 || sel[i] >= n) { free(r->sel); free(r); world_free(&w); *err = ORC_E_ARG; return NULL; }
            r->sel[i] = sel[i];
        }
    }
    r->cells = (cellres_t *)calloc((size_t)(r->n_sel > 0 ? r->n_sel : 1), sizeof(cellres_t));
    if (!r->cells) { free(r->sel); free(r); world_free(&w); *err = ORC_E_NOMEM; return NULL; }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    job_t job;
    job.w = &w; job.r = r; job.next = 0; job.err = ORC_OK;
    pthread_mutex_init(&job.mu, NULL);
    pthread_t th[256];
    int started = 0;
    for (int t = 1; t < nthreads; t++) {
        if (pthread_create(&th[t], NULL, worker, &job) == 0) started++;
        else break;
    }
    worker(&job);
    for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&job.mu);
    world_free(&w);
    r->err = job.err;
    *err = job.err;
    i64 ne = 0, nd = 0;
    for (i64 i = 0; i < r->n_sel; i++) {
        ne += r->cells[i].e;
        i64 k = r->sel ? r->sel[i] : i;
        for (i64 q = 0; q < r->cells[i].e; q++) if (r->cells[i].labels[q] > k) nd++;
    }
    r->n_edges = ne;
    r->n_del = nd;
    return r;
}

void orc_result_sizes(void *h, i64 *n_sel, i64 *n_edges, i64 *n_del) {
    orc_result *r = (orc_result *)h;
    *n_sel = r->n_sel; *n_edges = r->n_edges; *n_del = r->n_del;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return x < y ? -1 : (x > y);
}

/* Copy the result out: cell_ptr[n_sel+1], labels[n_edges], vnum[3*n_edges],
 * del[2*n_del] (pairs (k, j), k < j, ordered by k then j), stats[ST_N*n_sel]. */
void orc_result_copy(void *h, i64 *cell_ptr, int32_t *labels, i64 *vnum, int32_t *del,
                     i64 *stats) {
    orc_result *r = (orc_result *)h;
    i64 pe = 0, pd = 0;
    cell_ptr[0] = 0;
    for (i64 i = 0; i < r->n_sel; i++) {
        cellres_t *c = &r->cells[i];
        i64 k = r->sel ? r->sel[i] : i;
        memcpy(labels + pe, c->labels, (size_t)c->e * sizeof(int32_t));
        memcpy(vnum + 3 * pe, c->vnum, (size_t)c->e * 3 * sizeof(i64));
        i64 d0 = pd;
        for (i64 q = 0; q < c->e; q++) {
            if (c->labels[q] > k) { del[2 * pd + 1] = c->labels[q]; pd++; }
        }
        int32_t *tmp = (int32_t *)malloc((size_t)(pd - d0 + 1) * sizeof(int32_t));
        if (tmp) {
            for (i64 q = d0; q < pd; q++) tmp[q - d0] = del[2 * q + 1];
            qsort(tmp, (size_t)(pd - d0), sizeof(int32_t), cmp_i32);
            for (i64 q = d0; q < pd; q++) { del[2 * q] = (int32_t)k; del[2 * q + 1] = tmp[q - d0]; }
            free(tmp);
        }
        memcpy(stats + ST_N * i, c->st, ST_N * sizeof(i64));
        pe += c->e;
        cell_ptr[i + 1] = pe;
    }
}

void orc_result_free(void *h) {
    orc_result *r = (orc_result *)h;
    if (!r) return;
    for (i64 i = 0; i < r->n_sel; i++) { free(r->cells[i].labels); free(r->cells[i].vnum); }
    free(r->cells); free(r->sel); free(r);
}

/* ------------------------------------------------------------------ */
/* exported probes used by the pins                                     */
/* ------------------------------------------------------------------ */

/* The endpoint T(p_k, theta) (eq. (2.1)) with EquiDistList extremes.
 * out[0] = ccw label, out[1] = cw label, out[2] = number of tied lines;
 * t = tn / td returned as (hi, lo) 64-bit halves of each 128-bit value. */
int orc_endpoint(const int32_t *xy, i64 n, i64 W, i64 H, int mode, i64 s, i64 beta, i64 k,
                 i64 thx, i64 thy, int32_t *out, i64 *t4, i64 *cmp) {
    int rc = validate(xy, n, W, H);
    if (rc) return rc;
    if (k < 0 || k >= n || (thx == 0 && thy == 0)) return ORC_E_ARG;
    world_t w;
    rc = world_init(&w, xy, n, W, H, mode, s, beta);
    if (rc) { world_free(&w); return rc; }
    work_t wk;
    rc = work_init(&wk, &w);
    if (rc) { world_free(&w); return rc; }
    dir_t th; th.x = thx; th.y = thy;
    endpoint_t e;
    *cmp = 0;
    rc = endpoint(&w, &wk, k, th, &e, cmp);
    if (rc == ORC_OK) {
        out[0] = e.ccw; out[1] = e.cw; out[2] = e.ties;
        t4[0] = (i64)(e.t.tn >> 64); t4[1] = (i64)(uint64_t)e.t.tn;
        t4[2] = (i64)(e.t.td >> 64); t4[3] = (i64)(uint64_t)e.t.td;
    }
    work_free(&wk);
    world_free(&w);
    return rc;
}

/* The integer rectangle S_I[y, r] of eq. (A.3) for a rational centre
 * y = (yx/yd, yy/yd) and radius r = rn/rd (all denominators > 0):
 * out = [s floor((y1-r)/s), s (floor((y1+r)/s)+1), same for y2]. */
void orc_si(i64 yx, i64 yy, i64 yd, i64 rn, i64 rd, i64 s, i64 *out) {
    /* (y - r)/s = (y rd - rn yd) / (yd rd s) */
    i128 den = (i128)yd * rd * s;
    i128 lo_x = (i128)yx * rd - (i128)rn * yd, hi_x = (i128)yx * rd + (i128)rn * yd;
    i128 lo_y = (i128)yy * rd - (i128)rn * yd, hi_y = (i128)yy * rd + (i128)rn * yd;
    out[0] = (i64)(s * floordiv128(lo_x, den));
    out[1] = (i64)(s * (floordiv128(hi_x, den) + 1));
    out[2] = (i64)(s * floordiv128(lo_y, den));
    out[3] = (i64)(s * (floordiv128(hi_y, den) + 1));
}

/* eta of Method A.6 (exposed for the pins) */
i64 orc_eta(i64 beta, i64 s) { return eta_of(beta, s); }
