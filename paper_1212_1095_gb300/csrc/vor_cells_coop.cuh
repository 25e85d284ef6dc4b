// vor_cells_coop.cuh -- the cooperative large-cell tier: one block of CO_NW
// warps per cell, the cell's subwedges spread over the warps.
//
// Algorithm 1 splits the cell's boundary into subedges that are handled
// independently once their endpoints are known: the three initial wedges of
// the projector, and every subwedge a split creates (the paper's remark on
// the parallel case in Appendix 2: each subwedge can be processed by another
// processing unit).  Here the pending subedges of a cell form a queue in
// block-shared memory, processed in rounds: in a round every warp takes
// pending subedges one at a time, shoots the subedge's ray with its 32 lanes
// over the candidate table (FP32 filter, exact 128-bit fallback, Remark A.4
// extremes for ties), and either records the edges it found (the subedge
// lies on one line, or the vertex u of its two lines is in the cell) or
// appends the two subedges of the split to the queue for the next round.
//
// The edges found are marked per candidate (an edge can be met by several
// subedges), then sorted by the polar angle of their outward normals: for a
// convex polygon around p this is the counter-clockwise order, and sorting
// from the smallest angle in [0, 2 pi) is exactly the library's canonical
// order.  Consecutive edges meet at the vertices.
//
// Candidates and certificate are those of the warp-per-cell tiers: the sites
// within rho of p (with the sites of the polygon the warp tier handed on),
// then the vertex-disc ("flower") certificate, whose bucket rows are now
// spread over all warps of the block.
//
// Two modes share the code.  Mode S keeps a cell's arrays in shared memory
// with fixed capacities; a cell that exceeds them is handed to mode G, which
// keeps them in a global-memory slice per block with room for every site of
// the cell's set (n_j sites, n_j + 4 lines, 2 (n_j + 8) + 16 pending
// subedges), so no valid input exceeds it: every edge line is a candidate,
// and Algorithm 1 creates at most two subedges per ray.
#pragma once

#include "vor_cells.cuh"

namespace vor {

constexpr int CO_NW = 8;                  // warps per block
constexpr int CO_T = 32 * CO_NW;
constexpr int CO_CS = 1536;               // mode S: candidates
constexpr int CO_QS = 1024;               // mode S: pending subedges (ring)

// a pending subedge: its corner directions (left, right, counter-clockwise
// from left to right) and the lines met there: the counter-clockwise
// extreme at the left corner, the clockwise extreme at the right corner
struct CoopQ {
    long long lx, ly, rx, ry;
    int l1, l2;
};

// The arrays of one cell (shared memory in mode S, a global slice in mode G).
// The member names are those the certificate helpers of vor_cells.cuh read.
struct CoopView {
    float4 *cand;            // [cap] nx, ny, 1/c, (|nx|+|ny|)/c
    int *lab;                // [cap] site index in the set, or side -1..-4
    unsigned char *is_edge;  // [cap] the candidate's line carries an edge
    int *emit;               // [pow2 >= cap] the edges (candidate indices), sorted ccw
    float *vx, *vy, *vr;     // [cap] vertices relative to p, padded vertex-disc radii
    CoopQ *q;                // [qcap] pending subedges (ring); also scratch
    int cap, qcap, ecap;     // ecap: length of emit (a power of two >= cap)
};

struct CoopCtl {
    int ncand, flag, ne, qhead, qtail, qtake, err;
    Hit init[3];
    float red[CO_NW];
    int ired[CO_NW];
};

enum { CO_OK = 0, CO_CAP = 1, CO_INTERNAL = 2 };

// Bytes of one mode-G slice for sets of at most nmax sites.
__host__ __device__ inline long long coop_slice_caps(long long nmax, long long &cap, long long &qcap,
                                                     long long &ecap) {
    cap = nmax + 8;
    qcap = 2 * cap + 16;
    ecap = 1;
    while (ecap < cap) ecap <<= 1;
    auto al = [](long long x) { return (x + 255) & ~255ll; };
    return al(cap * 16) + al(cap * 4) + al(cap) + al(ecap * 4) + 3 * al(cap * 4) +
           al(qcap * (long long)sizeof(CoopQ));
}

__device__ inline CoopView coop_view_at(char *base, long long cap, long long qcap, long long ecap) {
    auto al = [](long long x) { return (x + 255) & ~255ll; };
    CoopView V;
    long long at = 0;
    V.cand = (float4 *)(base + at); at += al(cap * 16);
    V.lab = (int *)(base + at); at += al(cap * 4);
    V.is_edge = (unsigned char *)(base + at); at += al(cap);
    V.emit = (int *)(base + at); at += al(ecap * 4);
    V.vx = (float *)(base + at); at += al(cap * 4);
    V.vy = (float *)(base + at); at += al(cap * 4);
    V.vr = (float *)(base + at); at += al(cap * 4);
    V.q = (CoopQ *)(base + at);
    V.cap = (int)cap;
    V.qcap = (int)qcap;
    V.ecap = (int)ecap;
    return V;
}

// Mode S layout in dynamic shared memory.
struct __align__(16) CoopSmem {
    float4 cand[CO_CS];
    CoopQ q[CO_QS];
    int lab[CO_CS];
    int emit[2048];
    float vx[CO_CS], vy[CO_CS], vr[CO_CS];
    unsigned char is_edge[CO_CS];
};
static_assert(CO_CS <= 2048, "emit holds a power of two >= CO_CS");

__device__ __forceinline__ float block_max(float v, CoopCtl &K) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = group_max<32>(v, 0xffffffffu);
    __syncthreads();
    if (lane == 0) K.red[w] = v;
    __syncthreads();
    float r = K.red[0];
#pragma unroll
    for (int q = 1; q < CO_NW; q++) r = fmaxf(r, K.red[q]);
    return r;
}

// One ray of one warp: the filter pass over the C candidates and the
// decision (the ray of direction (tx, ty); for a vertex test, the ray
// towards u = p + N / D of lines la, lb).  Returns true when u is inside the
// cell (vertex test only); else h holds the endpoint's extreme lines.
__device__ bool coop_shoot(const CoopView &V, int C, int qt, i64 tx, i64 ty, int la, int lb, i64 Nx,
                           i64 Ny, i64 D, int exact_only, Hit &h, Counters &cnt) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float fx = (float)tx, fy = (float)ty;
    const float eth = fmaxf(fabsf(fx), fabsf(fy)) * VOR_TOL_SCALE;
    Filt f{-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX, -1};
    for (int c = lane; c < C; c += 32) {
        const float4 q = V.cand[c];
        const float den = fmaf(q.x, fx, q.y * fy);
        const float tol = q.w * eth;
        const float U = fmaf(den, q.z, tol);
        const float L = fmaf(den, q.z, -tol);
        if (U > f.u1) { f.u2 = f.u1; f.u1 = U; f.i1 = c; f.ls = L; }
        else f.u2 = fmaxf(f.u2, U);
        if (c != la && c != lb) f.ux = fmaxf(f.ux, U);
    }
    filt_reduce<32>(f, FULL);
    cnt.evals += C;
    h = Hit{-1, -1};
    if (qt == Q_UTEST) {
        cnt.vtests++;
        const i64 aD = D > 0 ? D : -D;
        const float kuf = (float)(aD / 2);
        const float klo = kuf * (1.f - 0x1p-21f), khi = kuf * (1.f + 0x1p-21f);
        if (!exact_only && f.ux < klo) return true;
        if (!exact_only && f.ls > f.u2 && f.ls > khi && f.i1 != la && f.i1 != lb) {
            h = Hit{f.i1, f.i1};
            return false;
        }
        cnt.exact++;
        int viol = 0;
        for (int c = lane; c < C && !viol; c += 32) {
            if (c == la || c == lb) continue;
            if (!exact_only) {
                const float4 q = V.cand[c];
                const float den = fmaf(q.x, fx, q.y * fy);
                if (fmaf(den, q.z, q.w * eth) < klo) continue;
            }
            int nx, ny;
            i64 cc;
            cand_int(V, c, nx, ny, cc);
            const i128 lhs = 2 * dot128(nx, ny, Nx, Ny) * (i128)(D > 0 ? 1 : -1);
            if (lhs > (i128)cc * aD) viol = 1;
        }
        viol = group_or<32>(viol, FULL);
        if (!viol) return true;
        h = exact_argmax<32>(V, C, tx, ty, fx, fy, eth, !exact_only, f.ls, lane, FULL);
        return false;
    }
    cnt.rays++;
    if (!exact_only && f.ls > f.u2 && f.ls > 0.f) {
        h = Hit{f.i1, f.i1};
    } else {
        cnt.exact++;
        h = exact_argmax<32>(V, C, tx, ty, fx, fy, eth, !exact_only, f.ls, lane, FULL);
    }
    return false;
}

// candidate a's outward normal strictly before b's in the counter-clockwise
// order from angle 0 (ties, which only equal lines have, by index); -1 is
// +infinity (padding)
__device__ __forceinline__ bool coop_edge_less(const CoopView &V, int a, int b) {
    if (a < 0) return false;
    if (b < 0) return true;
    const float4 qa = V.cand[a], qb = V.cand[b];
    const int ax = __float2int_rn(qa.x), ay = __float2int_rn(qa.y);
    const int bx = __float2int_rn(qb.x), by = __float2int_rn(qb.y);
    if (angle_less(ax, ay, bx, by)) return true;
    if (angle_less(bx, by, ax, ay)) return false;
    return a < b;
}

// Algorithm 1 over the C candidates with all warps of the block; the edges
// end in V.emit[0..ne) sorted counter-clockwise.  Returns CO_OK with K.ne
// set, CO_CAP when a mode-S capacity is exceeded, CO_INTERNAL on a failed
// consistency check.
__device__ int coop_projector(const CoopView &V, CoopCtl &K, int C, int exact_only, Counters &cnt) {
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int c = tid; c < C; c += CO_T) V.is_edge[c] = 0;
    if (tid == 0) { K.err = 0; K.qhead = 0; K.qtail = 0; K.qtake = 0; }
    if (w < 3) {
        // the three projector corners (integer directions; Section 4)
        const i64 tx = w == 0 ? 2 : (w == 1 ? 0 : -2), ty = w == 1 ? 1 : -1;
        Hit h;
        coop_shoot(V, C, Q_SHOOT, tx, ty, -1, -1, 0, 0, 0, exact_only, h, cnt);
        if (lane == 0) K.init[w] = h;
    }
    __syncthreads();
    if (tid == 0) {
        if (K.init[0].ccw < 0 || K.init[1].ccw < 0 || K.init[2].ccw < 0) {
            K.err = CO_INTERNAL;
        } else {
            V.q[0] = CoopQ{2, -1, 0, 1, K.init[0].ccw, K.init[1].cw};
            V.q[1] = CoopQ{0, 1, -2, -1, K.init[1].ccw, K.init[2].cw};
            V.q[2] = CoopQ{-2, -1, 2, -1, K.init[2].ccw, K.init[0].cw};
            K.qtail = 3;
        }
    }
    __syncthreads();
    const int guard = 4 * C + 64;            // rounds; a round handles at least one subedge
    for (int round = 0;; round++) {
        const int h0 = K.qhead, t0 = K.qtail;
        if (h0 == t0 || K.err) break;
        if (round > guard) { if (tid == 0) K.err = CO_INTERNAL; break; }
        for (;;) {
            int idx = 0;
            if (lane == 0) idx = atomicAdd(&K.qtake, 1);
            idx = __shfl_sync(0xffffffffu, idx, 0) + h0;
            if (idx >= t0) break;
            const CoopQ e = V.q[idx % V.qcap];
            if (e.l1 == e.l2) {                           // one line: an edge, no vertex
                if (lane == 0) V.is_edge[e.l1] = 1;
                continue;
            }
            int n1x, n1y, n2x, n2y;
            i64 c1, c2, Nx, Ny, D, tx, ty;
            cand_int(V, e.l1, n1x, n1y, c1);
            cand_int(V, e.l2, n2x, n2y, c2);
            intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
            int qt = Q_SHOOT, la = e.l1, lb = e.l2;
            if (D == 0) {                                  // parallel lines
                tx = -(i64)n1y;
                ty = (i64)n1x;
                if (!(cross128(e.lx, e.ly, tx, ty) >= 0 && cross128(tx, ty, e.rx, e.ry) >= 0)) {
                    tx = -tx;
                    ty = -ty;
                }
                la = lb = -1;
            } else {
                const int sg = D > 0 ? 1 : -1;
                const bool inw = sg * cross_sign(e.lx, e.ly, Nx, Ny) >= 0 &&
                                 sg * cross_sign(Nx, Ny, e.rx, e.ry) >= 0;   // lambda >= 0
                tx = sg * Nx;
                ty = sg * Ny;
                if (inw) {
                    qt = Q_UTEST;                          // the ray towards u
                } else {
                    tx = -tx;                              // theta_3 := p - u
                    ty = -ty;
                    la = lb = -1;
                }
            }
            Hit h;
            const bool inside = coop_shoot(V, C, qt, tx, ty, la, lb, Nx, Ny, D, exact_only, h, cnt);
            if (lane != 0) continue;
            if (inside) {                                  // u is a vertex: L1, L2 carry edges
                V.is_edge[e.l1] = 1;
                V.is_edge[e.l2] = 1;
                continue;
            }
            if (h.ccw < 0) { K.err = CO_INTERNAL; continue; }
            const int s = atomicAdd(&K.qtail, 2);          // divide the subedge at theta_3
            if (s + 2 - h0 > V.qcap) { atomicMax(&K.err, CO_CAP); continue; }
            V.q[s % V.qcap] = CoopQ{e.lx, e.ly, tx, ty, e.l1, h.cw};
            V.q[(s + 1) % V.qcap] = CoopQ{tx, ty, e.rx, e.ry, h.ccw, e.l2};
        }
        __syncthreads();
        if (tid == 0) { K.qhead = t0; K.qtake = 0; }
        __syncthreads();
    }
    __syncthreads();                                       // K.err as the last round left it
    if (K.err) return K.err;
    // the edges, then sorted counter-clockwise (bitonic network over ecap2)
    if (tid == 0) K.ne = 0;
    __syncthreads();
    for (int c = tid; c < C; c += CO_T) {
        if (V.is_edge[c]) V.emit[atomicAdd(&K.ne, 1)] = c;
    }
    __syncthreads();
    const int ne = K.ne;
    int P2 = 1;
    while (P2 < ne) P2 <<= 1;
    for (int i = ne + tid; i < P2; i += CO_T) V.emit[i] = -1;
    __syncthreads();
    for (int k = 2; k <= P2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P2; i += CO_T) {
                const int l = i ^ j;
                if (l > i) {
                    const int a = V.emit[i], b = V.emit[l];
                    const bool up = (i & k) == 0;
                    if (up ? coop_edge_less(V, b, a) : coop_edge_less(V, a, b)) {
                        V.emit[i] = b;
                        V.emit[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    return ne >= 3 ? CO_OK : CO_INTERNAL;
}

// The polygon's vertices (edges V.emit[0..e), counter-clockwise) into
// V.vx/V.vy/V.vr; returns max |v - p|^2 (block-wide), K.flag = 2 when two
// consecutive edges are parallel.
__device__ float coop_vertices(const CoopView &V, CoopCtl &K, int e) {
    float R2 = 0.f;
    for (int q = threadIdx.x; q < e; q += CO_T) {
        const int a = V.emit[q], b = V.emit[q + 1 < e ? q + 1 : 0];
        int n1x, n1y, n2x, n2y;
        i64 c1, c2, Nx, Ny, D;
        cand_int(V, a, n1x, n1y, c1);
        cand_int(V, b, n2x, n2y, c2);
        intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
        if (D == 0) { K.flag = 2; continue; }
        const float rd = 1.f / (float)D;
        const float vx = (float)Nx * rd, vy = (float)Ny * rd;
        V.vx[q] = vx;
        V.vy[q] = vy;
        const float r2 = fmaf(vx, vx, vy * vy);
        V.vr[q] = sqrtf(r2) * (1.f + 0x1p-10f) + 2.f;   // padded as in polygon_vertices
        R2 = fmaxf(R2, r2);
    }
    return block_max(R2, K);
}

// scan_rows of vor_cells.cuh spread over the block: the rows are
// row_of(k) for k in [kb, ke), warp w taking k = kb + 32 w + lane,
// kb + 32 (w + NW) + lane, ...; row_of returns -1 for no row
template <int NSPAN, int ILP, class RowOf, class RowSpans, class Visit>
__device__ __forceinline__ void coop_scan_rows(const CellGrid &g, const int2 *__restrict__ sxy, int kb,
                                               int ke, RowOf row_of, RowSpans row_spans, Visit visit) {
    const unsigned FULL = 0xffffffffu;
    const int w = threadIdx.x >> 5, gl = threadIdx.x & 31;
    for (int r0 = kb + 32 * w; r0 < ke; r0 += 32 * CO_NW) {
        const int row = r0 + gl < ke ? row_of(r0 + gl) : -1;
        int x0[NSPAN], x1[NSPAN];
        int ns = 0;
        if (row >= 0) ns = row_spans(row, x0, x1);
        int nmax = ns;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nmax = max(nmax, __shfl_xor_sync(FULL, nmax, off));
        const int *rb = g.bs + (size_t)(row >= 0 ? row : 0) * g.m1;
#pragma unroll
        for (int k = 0; k < NSPAN; k++) {
            if (k >= nmax) break;
            int a = 0, len = 0;
            if (k < ns) {
                a = rb[x0[k]];
                len = rb[x1[k] + 1] - a;
            }
            int incl = len;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, off);
                if (gl >= off) incl += y;
            }
            const int total = __shfl_sync(FULL, incl, 31);
            const int excl = incl - len;
            for (int k0 = 0; k0 < total; k0 += ILP * 32) {
                int pk[ILP];
                int2 sk[ILP];
#pragma unroll
                for (int u = 0; u < ILP; u++) {
                    const int kk = k0 + u * 32 + gl;
                    int j = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int ex = __shfl_sync(FULL, excl, j + step);
                        if (ex <= kk) j += step;
                    }
                    pk[u] = __shfl_sync(FULL, a, j) + kk - __shfl_sync(FULL, excl, j);
                    sk[u] = kk < total ? sxy[pk[u]] : make_int2(0, 0);
                }
#pragma unroll
                for (int u = 0; u < ILP; u++)
                    if (k0 + u * 32 + gl < total) visit(pk[u], sk[u]);
            }
        }
    }
}

// Append every site a != p with |a - p|^2 <= r2 to the candidates (the
// first disc); K.flag = 1 when the table would overflow.
__device__ void coop_scan_disc(const CellParams &P, const CellGrid &g, const CoopView &V, CoopCtl &K,
                               const int2 p, const int self, const i64 r2, Counters &cnt) {
    const int s = g.s;
    const int r = (int)ceilf(sqrtf((float)r2)) + 1;
    const int by0 = p.y - r <= 0 ? 0 : (p.y - r) / s;
    const int by1 = min(g.m2 - 1, (p.y + r) / s);
    const int cap = V.cap;
    auto visit = [&](int pos, int2 q) {
        if (pos == self) return;
        const int nx = q.x - p.x, ny = q.y - p.y;
        if ((i64)nx * nx + (i64)ny * ny > r2) return;
        const int at = atomicAdd(&K.ncand, 1);
        if (at < cap) {
            const float fnx = (float)nx, fny = (float)ny, rc = 1.f / fmaf(fnx, fnx, fny * fny);
            V.cand[at] = make_float4(fnx, fny, rc, (float)(abs(nx) + abs(ny)) * rc);
            V.lab[at] = P.sid[pos] - g.site_base;
        } else {
            K.flag = 1;
        }
    };
    auto row_of = [&](int k) { return by0 + k; };
    auto span = [&](int row, int *x0, int *x1) -> int {
        return disc_row_span(g, row, p.x, p.y, r2, x0[0], x1[0]) && x0[0] <= x1[0] ? 1 : 0;
    };
    coop_scan_rows<1, 2>(g, P.sxy, 0, by1 - by0 + 1, row_of, span, visit);
}

// The bucket rows in order of distance from p's row: k = 0, 1, 2, 3, ... is
// row prow, prow + 1, prow - 1, prow + 2, ...
__device__ __forceinline__ int sweep_row(const CellGrid &g, int prow, int k) {
    const int h = (k + 1) >> 1;
    const int row = (k & 1) ? prow + h : prow - h;
    return row >= 0 && row < g.m2 ? row : -1;
}

// One step of the certificate sweep: the rows sweep_row(k) for k in
// [k0, k0 + len).  The sites with r2lo < |a - p|^2 <= r2hi that cut the
// polygon of e vertices (reading only the parts of each row that meet a
// vertex disc) are appended to the candidates; once the table is full
// (K.flag) the step adds nothing more and is repeated, over fewer rows,
// after the next projector run.
__device__ void coop_sweep_step(const CellParams &P, const CellGrid &g, const CoopView &V, CoopCtl &K,
                                const int2 p, const int self, const i64 r2lo, const i64 r2hi,
                                const int e, const int prow, const int k0, const int len,
                                Counters &cnt) {
    const int cap = V.cap;
    auto visit = [&](int pos, int2 q) {
        if (pos == self) return;
        const int nx = q.x - p.x, ny = q.y - p.y;
        const i64 cc = (i64)nx * nx + (i64)ny * ny;
        if (cc <= r2lo || cc > r2hi) return;
        cnt.annulus++;
        if (K.flag || !cuts_polygon(V, e, nx, ny, cc)) return;
        const int at = atomicAdd(&K.ncand, 1);
        if (at < cap) {
            const float fnx = (float)nx, fny = (float)ny, rc = 1.f / fmaf(fnx, fnx, fny * fny);
            V.cand[at] = make_float4(fnx, fny, rc, (float)(abs(nx) + abs(ny)) * rc);
            V.lab[at] = P.sid[pos] - g.site_base;
        } else {
            K.flag = 1;
        }
    };
    auto row_of = [&](int k) { return sweep_row(g, prow, k); };
    auto spans = [&](int row, int *x0, int *x1) -> int {
        return flower_row_spans(g, V, e, p, r2lo, r2hi, row, x0, x1);
    };
    coop_scan_rows<5, 2>(g, P.sxy, k0, k0 + len, row_of, spans, visit);
}

// Keep only the candidates whose lines carry an edge of the polygon (edge q
// becomes candidate q; the other half-planes contain this polygon and every
// later one), through the queue as scratch.
__device__ void coop_prune(const CoopView &V, int e) {
    float4 *tc = reinterpret_cast<float4 *>(V.q);
    int *tl = reinterpret_cast<int *>(tc + e);
    for (int q = threadIdx.x; q < e; q += CO_T) {
        tc[q] = V.cand[V.emit[q]];
        tl[q] = V.lab[V.emit[q]];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < e; q += CO_T) {
        V.cand[q] = tc[q];
        V.lab[q] = tl[q];
        V.emit[q] = q;
    }
    __syncthreads();
}

// One cell with the whole block.  Returns CELL_OK (output written),
// CELL_DEFER (a mode-S capacity was exceeded) or CELL_FAIL (internal).
__device__ int coop_cell(const CellParams &P, const CoopView &V, CoopCtl &K, int i, Counters &cnt) {
    const int tid = threadIdx.x;
    const int2 p = P.sxy[i];
    const int k = P.sid[i];
    const CellGrid g = cell_grid(P, i);
    const int kl = k - g.site_base;
    const i64 cxf = max(p.x, g.W - p.x), cyf = max(p.y, g.H - p.y);
    const i64 far2 = cxf * cxf + cyf * cyf;            // no site is farther than a corner

    // ---- 1. the sites within rho (about P.target of them by the local density)
    const int s = g.s;
    const int bx = p.x / s, by = p.y / s;
    int c9 = 0, nb9 = 0;
    {
        const int x0 = max(bx - 1, 0), x1 = min(bx + 1, g.m1 - 1);
        for (int row = max(by - 1, 0); row <= min(by + 1, g.m2 - 1); row++) {
            c9 += g.bs[row * g.m1 + x1 + 1] - g.bs[row * g.m1 + x0];
            nb9 += x1 - x0 + 1;
        }
    }
    const float area = (float)nb9 * (float)s * (float)s;
    i64 rho2 = (i64)((float)P.target * area / (3.14159265f * (float)max(c9 - 1, 1)));
    rho2 = max(min(rho2, (i64)(16.f * (float)s * (float)s)), (i64)4);
    for (int attempt = 0;; attempt++) {
        if (tid == 0) { K.ncand = 0; K.flag = 0; }
        __syncthreads();
        coop_scan_disc(P, g, V, K, p, i, rho2, cnt);
        __syncthreads();
        if (!K.flag) break;
        if (attempt >= 24 || rho2 <= 4) return CELL_DEFER;
        rho2 /= 4;                                     // too dense: a smaller disc
    }
    int C = K.ncand;
    if (C + 4 > V.cap) return CELL_DEFER;
    if (P.seed_poly) {
        // the polygon an earlier tier left (ecount = -e, its lines in the
        // slot): its sites outside the disc join the candidates (extra
        // candidates never change the cell; these start it near its edges)
        const int e1 = -P.ecount[k];
        if (e1 >= 3 && e1 <= SLOT_CAP) {
            __syncthreads();                           // every thread has read the count
            if (tid < e1) {
                const int lab = P.slot[(size_t)k * SLOT_CAP + tid];
                if (lab >= 0 && lab < set_of(P.sets, P.sset, i).n && lab != kl) {
                    const int2 a = __ldg(P.sites + g.site_base + lab);
                    const int nx = a.x - p.x, ny = a.y - p.y;
                    if ((i64)nx * nx + (i64)ny * ny > rho2) {   // else the disc listed it
                        const int at = atomicAdd(&K.ncand, 1);
                        if (at < V.cap - 4) {
                            const float fnx = (float)nx, fny = (float)ny, rc = 1.f / fmaf(fnx, fnx, fny * fny);
                            V.cand[at] = make_float4(fnx, fny, rc, (float)(abs(nx) + abs(ny)) * rc);
                            V.lab[at] = lab;
                        }
                    }
                }
            }
            __syncthreads();
            C = min(K.ncand, V.cap - 4);
        }
    }
    if (tid == 0) {
        const int sx[4] = {0, g.W - p.x, 0, -p.x};
        const int sy[4] = {-p.y, 0, g.H - p.y, 0};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float cf = (float)(2 * ((i64)sx[q] * sx[q] + (i64)sy[q] * sy[q]));
            const float rc = 1.f / cf;
            V.cand[C + q] = make_float4((float)sx[q], (float)sy[q], rc,
                                        (float)(abs(sx[q]) + abs(sy[q])) * rc);
            V.lab[C + q] = -1 - q;
        }
    }
    C += 4;
    if (tid == 0) cnt.cands += C;
    __syncthreads();

    // ---- 2. Algorithm 1 --------------------------------------------------------
    int rc = coop_projector(V, K, C, P.exact_only, cnt);
    if (rc != CO_OK) return rc == CO_CAP ? CELL_DEFER : CELL_FAIL;
    int e = K.ne;

    // ---- 3. vertex-disc certificate, outward sweeps of bucket rows -----------
    // Invariant: every site within rho of p is a candidate or cuts no polygon
    // from here on (polygons only shrink, and so do their vertex discs).  A
    // round stops when 2R <= rho (Lemmas Byy'Syy' and SitesInLargeSquare) or
    // rho covers the box; else it sweeps the rows outward from p's row over
    // the annulus rho < |a - p| <= min(2R, 2 rho), adding the sites that cut
    // the current polygon, and reruns the projector whenever cutters
    // accumulate (or the table fills: the step is then repeated over fewer
    // rows), which shrinks the polygon, its vertex discs and the annulus
    // still to sweep.  After the sweep every site within the annulus's final
    // outer radius has been seen: rho grows to it.
    const int prow = p.y / s;
    for (int round = 0;; round++) {
        if (tid == 0) K.flag = 0;
        __syncthreads();
        float R2 = coop_vertices(V, K, e);
        if (K.flag == 2) return CELL_FAIL;
        i64 need = (i64)(4.f * (R2 * (1.f + 0x1p-12f) + 1.f)) + 1;   // > (2R)^2
        if (need <= rho2 || rho2 >= far2) break;
        if (round >= 64) return CELL_FAIL;
        coop_prune(V, e);
        C = e;
        if (tid == 0) cnt.widen++;
        // the next annulus reaches at most twice as far: the nearest cutters
        // first (they shrink the polygon and its vertex discs the most)
        i64 r2hi = min(min(need, rho2 < ((i64)1 << 60) / 4 ? 4 * rho2 + 4 : rho2), far2);
        int ran = C;                                   // candidates the last projector run saw
        int repeats = 0;
        int len = CO_T;                                // rows per step: fewer after a full table
        for (int k0 = 0;;) {
            const int rmax = (int)(sqrtf((float)r2hi) / (float)s) + 2;   // rows beyond cannot meet
            const bool last = k0 + len > 2 * rmax + 1;
            if (tid == 0) { K.ncand = C; K.flag = 0; }
            __syncthreads();
            coop_sweep_step(P, g, V, K, p, i, rho2, r2hi, e, prow, k0, len, cnt);
            __syncthreads();
            const bool full = K.flag != 0;
            C = min(K.ncand, V.cap);
            if (full || C - ran >= 64 || last) {
                if (C > ran) {
                    if (tid == 0) { cnt.reruns++; cnt.cands += C - ran; }
                    rc = coop_projector(V, K, C, P.exact_only, cnt);
                    if (rc != CO_OK) return rc == CO_CAP ? CELL_DEFER : CELL_FAIL;
                    e = K.ne;
                    if (tid == 0) K.flag = 0;
                    __syncthreads();
                    R2 = coop_vertices(V, K, e);
                    if (K.flag == 2) return CELL_FAIL;
                    need = (i64)(4.f * (R2 * (1.f + 0x1p-12f) + 1.f)) + 1;
                    r2hi = min(r2hi, need);
                    coop_prune(V, e);
                    C = ran = e;
                }
                if (full) {                            // the step again, with room, over fewer rows
                    if (++repeats > 64) return CELL_DEFER;
                    len = max(len / 2, 8);
                    continue;
                }
            }
            repeats = 0;
            if (last) break;
            k0 += len;
            len = min(len * 2, CO_T);
        }
        rho2 = r2hi;
    }

    // ---- 4. output: the sorted order starts at the smallest normal angle ------
    int *dst;
    int off = -1;
    if (e <= SLOT_CAP) {
        dst = P.slot + (size_t)k * SLOT_CAP;
    } else {
        if (tid == 0) K.qtake = atomicAdd(&P.hdr->spill_top, e);
        __syncthreads();
        off = K.qtake;
        if (off + e > P.spill_cap) return CELL_FAIL;
        dst = P.spill + off;
    }
    int dcnt = 0;
    for (int q = tid; q < e; q += CO_T) {
        const int lab = V.lab[V.emit[q]];
        dst[q] = lab;
        dcnt += lab > kl ? 1 : 0;
    }
    dcnt = group_sum<32>(dcnt, 0xffffffffu);
    if ((threadIdx.x & 31) == 0) K.ired[threadIdx.x >> 5] = dcnt;
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int q = 0; q < CO_NW; q++) tot += K.ired[q];
        P.ecount[k] = e;
        P.dcount[k] = tot;
        P.loc[k] = off;
        if ((unsigned long long)e > cnt.maxe) cnt.maxe = e;
    }
    __syncthreads();
    return CELL_OK;
}

// Persistent: each block takes cells of P.cell_list from *P.next_cell.
// Mode S (GMODE false): arrays in dynamic shared memory; cells that exceed
// them go to P.deferred.  Mode G: block b uses slice b of the arena.
template <bool GMODE>
__global__ void __launch_bounds__(CO_T, 2) coop_cells_kernel(CellParams P, char *arena, long long slice,
                                                             long long cap, long long qcap,
                                                             long long ecap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ CoopCtl K;
    __shared__ int s_t;
    if (P.hdr->err) return;
    CoopView V;
    if (GMODE) {
        V = coop_view_at(arena + (long long)blockIdx.x * slice, cap, qcap, ecap);
    } else {
        CoopSmem &S = *reinterpret_cast<CoopSmem *>(smem_raw);
        V.cand = S.cand; V.lab = S.lab; V.is_edge = S.is_edge; V.emit = S.emit;
        V.vx = S.vx; V.vy = S.vy; V.vr = S.vr; V.q = S.q;
        V.cap = CO_CS; V.qcap = CO_QS; V.ecap = 2048;
    }
    const int total = *P.list_count;
    Counters cnt{};
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(P.next_cell, 1);
        __syncthreads();
        const int t = s_t;
        __syncthreads();
        if (t >= total) break;
        const int i = P.cell_list[t];
        const int rc = coop_cell(P, V, K, i, cnt);
        if (rc != CELL_OK && threadIdx.x == 0) {
            // mode G holds every site of the set: nothing is deferred from it
            if (!GMODE && rc == CELL_DEFER && P.deferred) {
                const int q = atomicAdd(P.deferred_count, 1);
                P.deferred[q] = i;
                cnt.deferred++;
            } else {
                atomicOr(&P.hdr->err, ERRB_INTERNAL);
            }
        }
        __syncthreads();
    }
    if (P.collect_stats && (threadIdx.x & 31) == 0) {
        unsigned long long *st = P.hdr->stats;
        atomicAdd(&st[STAT_RAYS], cnt.rays);
        atomicAdd(&st[STAT_VTESTS], cnt.vtests);
        atomicAdd(&st[STAT_EVALS], cnt.evals);
        atomicAdd(&st[STAT_EXACT], cnt.exact);
        atomicAdd(&st[STAT_ANNULUS], cnt.annulus);
        atomicAdd(&st[STAT_RERUNS], cnt.reruns);
        atomicAdd(&st[STAT_DEFERRED], cnt.deferred);
        atomicAdd(&st[STAT_CANDIDATES], cnt.cands);
        atomicMax(&st[STAT_MAXE], cnt.maxe);
        atomicAdd(&st[STAT_WIDEN], cnt.widen);
    }
}

}  // namespace vor
