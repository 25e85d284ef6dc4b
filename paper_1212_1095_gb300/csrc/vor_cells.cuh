// vor_cells.cuh -- the per-cell projector kernel (ray shooting).
//
// A group of G lanes of one warp computes one Voronoi cell with Algorithm 1
// of the paper; a warp holds 32/G groups, each on its own cell.
//
//  1. Candidates.  The sites within distance rho of p (found through the
//     buckets of Method A.5 that meet the square [p - rho, p + rho]) are
//     staged in shared memory, with the four sides of X written as lines (the
//     reflection of p across a side has that side as its bisector with p, so
//     eq. (A.1) is a bisector hit like any other).
//  2. Projector.  The three projector corners are shot, then the subedges are
//     processed depth-first, left child first, so subwedges are visited
//     counter-clockwise and the cell's edges come out in that order.  The
//     loop is a state machine that issues exactly one ray per iteration from
//     a single call site, so the groups of a warp stay converged while they
//     scan their candidates.  A ray's endpoint T(p, theta) (eq. (2.1)) is the
//     candidate line with the largest key K = <n, theta> / c: lanes split the
//     candidates, evaluate an FP32 filter with a certified error bound and
//     reduce with warp shuffles; only rays whose winner the bound cannot
//     separate (near ties, and exact ties where the ray meets a vertex,
//     Remark A.4) are re-decided exactly in 128-bit integers, again split
//     over the lanes.  The test "u is inside the cell" of Algorithm 1 is the
//     ray towards u: u is inside iff no line other than L1, L2 is met first.
//  3. Certificate.  R = the largest distance from p to a vertex of the
//     polygon.  A site farther than 2R cannot cut it (for x in the polygon,
//     |x - a| >= |a - p| - |x - p| > R >= |x - p|; the argument of Lemmas
//     Byy'Syy' and SitesInLargeSquare).  All sites within rho were
//     candidates; while 2R > rho, rho grows (at most doubling), the new sites
//     are tested against the polygon's vertices, the ones that cut it join
//     the candidates and the projector runs again.
//  4. Output.  The edge labels are rotated to start at the smallest normal
//     angle and written to a fixed slot per cell (or a spill area).
//
// Two uses of this code.  With several lanes per cell (lanes_per_cell > 1)
// it is the first pass over all cells (small capacities, bounded
// certificate work), deferring the rare cells that exceed its limits.  With
// one warp per cell and larger capacities it is the warp tier: it takes the
// cells the thread-per-cell passes leave, certifies them with the vertex
// discs of the polygon (flower) over growing annuli, and hands the cells
// that exceed it, or whose next annulus lies over a cluster's core, to the
// block tier (vor_cells_coop.cuh).  Its first candidates include the sites
// of the polygon the last pass left in the cell's slot, and it leaves its
// own polygon there for the block tier.  For a single diagram the warp tier
// runs a cell's subedges on four groups of 8 lanes (projector_par).
#pragma once

#include <cfloat>
#include <cmath>
#include <cstddef>

#include "vor_device.cuh"
#include "vor_internal.h"

namespace vor {

template <int CMAX, int SMAX, int EMAX>
struct __align__(16) GroupSmem {
    float4 cand[CMAX];           // nx, ny, 1/c, (|nx|+|ny|)/c
    int lab[CMAX];               // site index (>= 0) or side (-1..-4)
    long long sx[SMAX], sy[SMAX];// subedge stack: right corners
    short scw[SMAX], sccw[SMAX]; // their clockwise / counter-clockwise lines
    short emit[EMAX];            // edges, counter-clockwise
    float vx[EMAX], vy[EMAX];    // approximate vertices relative to p
    float vr[EMAX];              // |v - p|, padded (vertex-disc radii of the certificate)
    short tmp[EMAX];             // scratch of the candidate compaction
    int ncand;                   // candidate count while appending
    int flag;
    int hist[32];                // certificate: cutters per distance bin of the annulus
    // the parallel projector only (last, so that a launch without it can
    // leave them out of its shared memory: group_smem_bytes)
    long long slx[SMAX], sly[SMAX];// left corners of the stacked subedges
    unsigned char is_edge[CMAX]; // the candidate's line carries an edge
    int sp, nedge, perr;         // stack top, edges, error
    int ini[6];                  // the corner rays' extreme lines
};

// Shared memory of one group: the whole struct with the parallel projector,
// else up to its first field (one group per block only: the struct's size
// is the stride between groups).
template <int CMAX, int SMAX, int EMAX>
inline int group_smem_bytes(bool par) {
    using SM = GroupSmem<CMAX, SMAX, EMAX>;
    return par ? (int)sizeof(SM) : (int)((offsetof(SM, slx) + 15) & ~(size_t)15);
}

struct Hit { int ccw, cw; };

struct Counters {
    unsigned long long rays, vtests, evals, exact, annulus, reruns, deferred, cands, maxe, widen;
};

enum { CELL_OK = 0, CELL_DEFER = 1, CELL_FAIL = 2 };

// The warp tier hands a cell on to the block tier when its next certificate
// annulus may hold more sites than this while they are a small part (under
// 1/16) of its set: a cluster's core in a large set.  Measured on the
// clustered 4M set: the cells moved are the slowest of the warp tier's wave,
// and the large-cell stage shortens by a third (thresholds of 4 k to 32 k
// sites tried, 8 k the best); in small sets the warp tier finishes such
// cells sooner than the block tier.
constexpr int M_DEFER_SITES = 8192;

// Float filter: the computed key k of a candidate satisfies
//   |k - K| <= 7.1 u (|nx||tx| + |ny||ty|) / c,  u = 2^-24
// (theta rounded to float u, the dot product 2u, c = nx^2 + ny^2 by one FMA
// 2u and its rounded reciprocal u, the product u).  The kernel uses
// tol = (|nx|+|ny|)/c * max(|tx|,|ty|) * 2^-19 (= 32 u), a margin of more
// than 4x, which also absorbs the rounding of k + tol and k - tol.
#define VOR_TOL_SCALE 0x1p-19f

struct Filt { float u1, ls, u2, ux; int i1; };

template <int G>
__device__ __forceinline__ void filt_reduce(Filt &f, unsigned gmask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        float ou1 = __shfl_xor_sync(gmask, f.u1, off, G);
        float ols = __shfl_xor_sync(gmask, f.ls, off, G);
        float ou2 = __shfl_xor_sync(gmask, f.u2, off, G);
        float oux = __shfl_xor_sync(gmask, f.ux, off, G);
        int oi1 = __shfl_xor_sync(gmask, f.i1, off, G);
        bool take = (ou1 > f.u1) || (ou1 == f.u1 && oi1 < f.i1);
        float lo = take ? f.u1 : ou1;
        f.u2 = fmaxf(fmaxf(f.u2, ou2), lo);
        if (take) { f.u1 = ou1; f.i1 = oi1; f.ls = ols; }
        f.ux = fmaxf(f.ux, oux);
    }
}

template <class SM>
__device__ __forceinline__ void cand_int(const SM &S, int c, int &nx, int &ny, i64 &cc) {
    float4 q = S.cand[c];
    nx = __float2int_rn(q.x);
    ny = __float2int_rn(q.y);
    cc = line_c(nx, ny, S.lab[c] < 0);
}

// a strictly more counter-clockwise than b (normals in one open half-plane)
template <class SM>
__device__ __forceinline__ bool more_ccw(const SM &S, int a, int b) {
    int ax, ay, bx, by;
    i64 ca, cb;
    cand_int(S, a, ax, ay, ca);
    cand_int(S, b, bx, by, cb);
    return (i64)bx * ay - (i64)by * ax > 0;
}

// merge (best, ccw, cw) with (ob, occ, ocw) for direction (tx, ty), exactly
template <class SM>
__device__ __forceinline__ void exact_merge(const SM &S, i64 tx, i64 ty, int &best, int &ccw,
                                            int &cw, int ob, int occ, int ocw) {
    if (ob < 0) return;
    if (best < 0) { best = ob; ccw = occ; cw = ocw; return; }
    int ax, ay, bx, by;
    i64 ca, cb;
    cand_int(S, best, ax, ay, ca);
    cand_int(S, ob, bx, by, cb);
    i128 da = dot128(ax, ay, tx, ty), db = dot128(bx, by, tx, ty);
    i128 lhs = db * (i128)ca, rhs = da * (i128)cb;   // key(ob) vs key(best)
    if (lhs > rhs) { best = ob; ccw = occ; cw = ocw; }
    else if (lhs == rhs) {
        if (more_ccw(S, occ, ccw)) ccw = occ;
        if (more_ccw(S, cw, ocw)) cw = ocw;
    }
}

// Exact endpoint of direction (tx, ty) over the candidates whose filter upper
// bound reaches thr (all candidates when use_thr is false).
template <int G, class SM>
__device__ Hit exact_argmax(const SM &S, int C, i64 tx, i64 ty, float fx, float fy, float eth,
                            bool use_thr, float thr, int gl, unsigned gmask) {
    int best = -1, ccw = -1, cw = -1;
    for (int c = gl; c < C; c += G) {
        float4 q = S.cand[c];
        if (use_thr) {
            float den = fmaf(q.x, fx, q.y * fy);
            float U = fmaf(den, q.z, q.w * eth);
            if (!(U >= thr)) continue;
        }
        int nx = __float2int_rn(q.x), ny = __float2int_rn(q.y);
        if (dot128(nx, ny, tx, ty) <= 0) continue;
        exact_merge(S, tx, ty, best, ccw, cw, c, c, c);
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        int ob = __shfl_xor_sync(gmask, best, off, G);
        int oc = __shfl_xor_sync(gmask, ccw, off, G);
        int ow = __shfl_xor_sync(gmask, cw, off, G);
        exact_merge(S, tx, ty, best, ccw, cw, ob, oc, ow);
    }
    return Hit{ccw, cw};
}

// Sign of cross(a, b) = ax by - ay bx for 64-bit integer vectors: a float
// evaluation with a bound on its error, the exact 128-bit value when the
// bound cannot decide.
__device__ __forceinline__ int cross_sign(i64 ax, i64 ay, i64 bx, i64 by) {
    const float p = (float)ax * (float)by, q = (float)ay * (float)bx;
    const float v = p - q, bound = (fabsf(p) + fabsf(q)) * 0x1p-20f;
    if (v > bound) return 1;
    if (v < -bound) return -1;
    const i128 e = cross128(ax, ay, bx, by);
    return e > 0 ? 1 : (e < 0 ? -1 : 0);
}

enum { Q_SHOOT = 0, Q_UTEST = 1 };

// Algorithm 1 over the C staged candidates.  Returns the number of edges (in
// S.emit, counter-clockwise from the edge met by psi_1), or -1 when a
// capacity is exceeded.  Not inlined: the warp tier calls it twice (the
// first polygon and the reruns of the certificate), and one copy of its code
// instead of two keeps the tier's hot loop in the instruction cache (the
// top stall of the tier with 21 warps per SM at different points of it;
// measured: the batch's tiers 33.3 -> 24.5 ms).
template <int G, int CMAX, int SMAX, int EMAX, int RMAX>
__device__ __noinline__ int projector(GroupSmem<CMAX, SMAX, EMAX> &S, const int C, const int gl,
                         const unsigned gmask, const int exact_only, Counters &cnt) {
    int phase = 0;                  // 0..2: the projector corners; 3: the subedges
    Hit init[3];
    i64 lx = 0, ly = 0;             // left corner of the current subwedge
    int llab = -1;                  // its line (the counter-clockwise extreme)
    int sp = 0, ne = 0, rays = 3, first = -1, last = -1;
    for (int guard = 0; guard < 4 * RMAX + 8; guard++) {
        // ---- choose the next ray (control only, no candidate scans) ----
        int qt = Q_SHOOT;
        i64 tx = 0, ty = 0, Nx = 0, Ny = 0, D = 0;
        int la = -1, lb = -1;
        if (phase < 3) {
            tx = phase == 0 ? 2 : (phase == 1 ? 0 : -2);
            ty = phase == 1 ? 1 : -1;
        } else {
            bool have = false;
            while (sp > 0) {
                const int top = sp - 1;
                const i64 rx = S.sx[top], ry = S.sy[top];
                const int rcw = S.scw[top];
                if (llab == rcw) {                         // same line: no vertex here
                    if (llab != last) {
                        if (ne >= EMAX) return -1;
                        if (gl == 0) S.emit[ne] = (short)llab;
                        if (first < 0) first = llab;
                        last = llab;
                        ne++;
                    }
                    lx = rx; ly = ry; llab = S.sccw[top];
                    sp--;
                    continue;
                }
                int n1x, n1y, n2x, n2y;
                i64 c1, c2;
                cand_int(S, llab, n1x, n1y, c1);
                cand_int(S, rcw, n2x, n2y, c2);
                intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
                la = llab;
                lb = rcw;
                if (D == 0) {                              // parallel lines
                    tx = -(i64)n1y;
                    ty = (i64)n1x;
                    if (!(cross128(lx, ly, tx, ty) >= 0 && cross128(tx, ty, rx, ry) >= 0)) {
                        tx = -tx;
                        ty = -ty;
                    }
                    la = lb = -1;
                } else {
                    const int sg = D > 0 ? 1 : -1;
                    const bool inw = sg * cross_sign(lx, ly, Nx, Ny) >= 0 &&
                                     sg * cross_sign(Nx, Ny, rx, ry) >= 0;   // lambda >= 0
                    tx = sg * Nx;
                    ty = sg * Ny;
                    if (inw) {
                        qt = Q_UTEST;                      // ray towards u
                    } else {
                        tx = -tx;                          // theta_3 := p - u
                        ty = -ty;
                        la = lb = -1;
                    }
                }
                have = true;
                break;
            }
            if (!have) break;                              // EdgeQueue is empty
        }
        // ---- one filter pass over the candidates (the only call site) ----
        const float fx = (float)tx, fy = (float)ty;
        const float eth = fmaxf(fabsf(fx), fabsf(fy)) * VOR_TOL_SCALE;
        Filt f{-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX, -1};
        // unrolled twice: a lane's next candidate loads while this one is
        // compared (measured: the batch's tiers 26.5 -> 23.4 ms)
#pragma unroll 2
        for (int c = gl; c < C; c += G) {
            const float4 q = S.cand[c];
            const float den = fmaf(q.x, fx, q.y * fy);
            const float tol = q.w * eth;
            const float U = fmaf(den, q.z, tol);
            const float L = fmaf(den, q.z, -tol);
            if (U > f.u1) { f.u2 = f.u1; f.u1 = U; f.i1 = c; f.ls = L; }
            else f.u2 = fmaxf(f.u2, U);
            if (c != la && c != lb) f.ux = fmaxf(f.ux, U);
        }
        filt_reduce<G>(f, gmask);
        cnt.evals += C;
        // ---- decide ----
        Hit h{-1, -1};
        bool inside = false;
        if (qt == Q_UTEST) {
            cnt.vtests++;
            const i64 aD = D > 0 ? D : -D;
            const float kuf = (float)(aD / 2);             // key of u: |D|/2, an integer
            const float klo = kuf * (1.f - 0x1p-21f), khi = kuf * (1.f + 0x1p-21f);
            if (!exact_only && f.ux < klo) {
                inside = true;
            } else if (!exact_only && f.ls > f.u2 && f.ls > khi && f.i1 != la && f.i1 != lb) {
                h = Hit{f.i1, f.i1};
            } else {
                cnt.exact++;
                // exact: u violates line c iff 2 <n_c, N> sgn(D) > c |D|
                int viol = 0;
                for (int c = gl; c < C && !viol; c += G) {
                    if (c == la || c == lb) continue;
                    if (!exact_only) {
                        const float4 q = S.cand[c];
                        const float den = fmaf(q.x, fx, q.y * fy);
                        if (fmaf(den, q.z, q.w * eth) < klo) continue;
                    }
                    int nx, ny;
                    i64 cc;
                    cand_int(S, c, nx, ny, cc);
                    const i128 lhs = 2 * dot128(nx, ny, Nx, Ny) * (i128)(D > 0 ? 1 : -1);
                    if (lhs > (i128)cc * aD) viol = 1;
                }
                viol = group_or<G>(viol, gmask);
                if (!viol) inside = true;
                else h = exact_argmax<G>(S, C, tx, ty, fx, fy, eth, !exact_only, f.ls, gl, gmask);
            }
        } else {
            cnt.rays++;
            if (!exact_only && f.ls > f.u2 && f.ls > 0.f) {
                h = Hit{f.i1, f.i1};
            } else {
                cnt.exact++;
                h = exact_argmax<G>(S, C, tx, ty, fx, fy, eth, !exact_only, f.ls, gl, gmask);
            }
        }
        // ---- update the subedge state ----
        if (phase < 3) {
            init[phase] = h;
            if (h.ccw < 0) return -1;
            if (++phase == 3) {
                lx = 2; ly = -1; llab = init[0].ccw;
                if (gl == 0) {
                    S.sx[0] = 2;  S.sy[0] = -1; S.scw[0] = (short)init[0].cw; S.sccw[0] = (short)init[0].ccw;
                    S.sx[1] = -2; S.sy[1] = -1; S.scw[1] = (short)init[2].cw; S.sccw[1] = (short)init[2].ccw;
                    S.sx[2] = 0;  S.sy[2] = 1;  S.scw[2] = (short)init[1].cw; S.sccw[2] = (short)init[1].ccw;
                }
                sp = 3;
            }
        } else if (inside) {                               // u is a vertex: L1, L2 are edges
            const int top = sp - 1;
            if (la != last) {
                if (ne >= EMAX) return -1;
                if (gl == 0) S.emit[ne] = (short)la;
                if (first < 0) first = la;
                last = la;
                ne++;
            }
            if (lb != last) {
                if (ne >= EMAX) return -1;
                if (gl == 0) S.emit[ne] = (short)lb;
                if (first < 0) first = lb;
                last = lb;
                ne++;
            }
            lx = S.sx[top]; ly = S.sy[top]; llab = S.sccw[top];
            sp--;
        } else {                                           // divide the subedge at theta_3
            if (sp >= SMAX || ++rays > RMAX || h.ccw < 0) return -1;
            if (gl == 0) {
                S.sx[sp] = tx; S.sy[sp] = ty; S.scw[sp] = (short)h.cw; S.sccw[sp] = (short)h.ccw;
            }
            sp++;
        }
        group_sync<G>(gmask);
    }
    group_sync<G>(gmask);
    if (phase < 3 || sp > 0) return -1;
    if (ne > 1 && last == first) ne--;                     // the walk closes on its first edge
    return ne;
}

// One ray shot by a group of GL lanes (the filter pass over the C candidates,
// the reduction within the group and the decision; exact fallbacks as in
// projector).  Returns true when u is inside the cell (vertex test only);
// else h holds the endpoint's extreme lines.
template <int GL, class SM>
__device__ bool group_shoot(const SM &S, int C, int qt, i64 tx, i64 ty, int la, int lb, i64 Nx, i64 Ny,
                            i64 D, int exact_only, int gl, unsigned gmask, Hit &h, Counters &cnt) {
    const float fx = (float)tx, fy = (float)ty;
    const float eth = fmaxf(fabsf(fx), fabsf(fy)) * VOR_TOL_SCALE;
    Filt f{-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX, -1};
#pragma unroll 2
    for (int c = gl; c < C; c += GL) {
        const float4 q = S.cand[c];
        const float den = fmaf(q.x, fx, q.y * fy);
        const float tol = q.w * eth;
        const float U = fmaf(den, q.z, tol);
        const float L = fmaf(den, q.z, -tol);
        if (U > f.u1) { f.u2 = f.u1; f.u1 = U; f.i1 = c; f.ls = L; }
        else f.u2 = fmaxf(f.u2, U);
        if (c != la && c != lb) f.ux = fmaxf(f.ux, U);
    }
    filt_reduce<GL>(f, gmask);
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
        for (int c = gl; c < C && !viol; c += GL) {
            if (c == la || c == lb) continue;
            if (!exact_only) {
                const float4 q = S.cand[c];
                const float den = fmaf(q.x, fx, q.y * fy);
                if (fmaf(den, q.z, q.w * eth) < klo) continue;
            }
            int nx, ny;
            i64 cc;
            cand_int(S, c, nx, ny, cc);
            const i128 lhs = 2 * dot128(nx, ny, Nx, Ny) * (i128)(D > 0 ? 1 : -1);
            if (lhs > (i128)cc * aD) viol = 1;
        }
        viol = group_or<GL>(viol, gmask);
        if (!viol) return true;
        h = exact_argmax<GL>(S, C, tx, ty, fx, fy, eth, !exact_only, f.ls, gl, gmask);
        return false;
    }
    cnt.rays++;
    if (!exact_only && f.ls > f.u2 && f.ls > 0.f) {
        h = Hit{f.i1, f.i1};
    } else {
        cnt.exact++;
        h = exact_argmax<GL>(S, C, tx, ty, fx, fy, eth, !exact_only, f.ls, gl, gmask);
    }
    return false;
}

// candidate a's outward normal strictly before b's counter-clockwise from
// angle 0 (equal lines, which distinct sites cannot give, by index)
template <class SM>
__device__ __forceinline__ bool normal_less(const SM &S, int a, int b) {
    int ax, ay, bx, by;
    i64 ca, cb;
    cand_int(S, a, ax, ay, ca);
    cand_int(S, b, bx, by, cb);
    if (angle_less(ax, ay, bx, by)) return true;
    if (angle_less(bx, by, ax, ay)) return false;
    return a < b;
}

// Algorithm 1 for one warp with NG groups of 32 / NG lanes, each group
// taking its own subedge (Appendix 2, the parallel case: the subwedges are
// handled independently once their corners are known).  The three corner
// rays go to groups 0..2; then in every step each group pops one pending
// subedge (the subwedge between its corner directions, with the lines met
// there) and either marks the edges it finds (one line on the whole
// subedge, or the vertex of its two lines inside the cell) or pushes the two
// subedges of the split.  The edges, marked per candidate, are then sorted by
// the angle of their outward normals: the counter-clockwise order of a
// convex polygon around p, starting at the smallest angle (the canonical
// order).  Returns the number of edges (in S.emit), or -1 when a capacity is
// exceeded.  The counters of all groups end in lane 0's.
template <int NG, int CMAX, int SMAX, int EMAX, int RMAX>
__device__ __noinline__ int projector_par(GroupSmem<CMAX, SMAX, EMAX> &S, const int C, const int lane,
                             const int exact_only, Counters &cnt) {
    static_assert(NG >= 3 && 32 % NG == 0, "three corner rays, whole groups");
    constexpr int GL = 32 / NG;
    const unsigned FULL = 0xffffffffu;
    const int grp = lane / GL, gl = lane % GL;
    const unsigned gmask = (GL == 32) ? FULL : (((1u << GL) - 1u) << (grp * GL));
    const Counters c0 = cnt;
    for (int c = lane; c < C; c += 32) S.is_edge[c] = 0;
    if (grp < 3) {
        const i64 tx = grp == 0 ? 2 : (grp == 1 ? 0 : -2), ty = grp == 1 ? 1 : -1;
        Hit h;
        group_shoot<GL>(S, C, Q_SHOOT, tx, ty, -1, -1, 0, 0, 0, exact_only, gl, gmask, h, cnt);
        if (gl == 0) { S.ini[2 * grp] = h.ccw; S.ini[2 * grp + 1] = h.cw; }
    }
    __syncwarp();
    if (lane == 0) {
        S.perr = (S.ini[0] < 0 || S.ini[2] < 0 || S.ini[4] < 0) ? 1 : 0;
        // subwedges (left corner, right corner) counter-clockwise, with the
        // counter-clockwise extreme line at the left corner, the clockwise
        // extreme at the right one
        const long long cx[3] = {2, 0, -2}, cy[3] = {-1, 1, -1};
        for (int k = 0; k < 3; k++) {
            const int kn = k == 2 ? 0 : k + 1;
            S.slx[k] = cx[k]; S.sly[k] = cy[k];
            S.sx[k] = cx[kn]; S.sy[k] = cy[kn];
            S.sccw[k] = (short)S.ini[2 * k];
            S.scw[k] = (short)S.ini[2 * kn + 1];
        }
        S.sp = 3;
    }
    __syncwarp();
    int rays = 3;
    for (int step = 0; !S.perr; step++) {
        const int sp0 = S.sp;
        if (sp0 == 0) break;
        const int take = min(sp0, NG);
        rays += take;
        if (rays > RMAX + 3 * NG) { if (lane == 0) S.perr = 1; break; }
        __syncwarp();
        if (lane == 0) S.sp = sp0 - take;                 // the popped entries, then pushes on top
        int k = -1;
        i64 elx = 0, ely = 0, erx = 0, ery = 0;
        int l1 = -1, l2 = -1;
        if (grp < take) {
            k = sp0 - 1 - grp;
            elx = S.slx[k]; ely = S.sly[k]; erx = S.sx[k]; ery = S.sy[k];
            l1 = S.sccw[k]; l2 = S.scw[k];
        }
        __syncwarp();
        if (k >= 0 && l1 == l2) {                        // one line: an edge, no vertex
            if (gl == 0) S.is_edge[l1] = 1;
        } else if (k >= 0) {
            int n1x, n1y, n2x, n2y;
            i64 c1, c2, Nx, Ny, D, tx, ty;
            cand_int(S, l1, n1x, n1y, c1);
            cand_int(S, l2, n2x, n2y, c2);
            intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
            int qt = Q_SHOOT, la = l1, lb = l2;
            if (D == 0) {                                  // parallel lines
                tx = -(i64)n1y;
                ty = (i64)n1x;
                if (!(cross128(elx, ely, tx, ty) >= 0 && cross128(tx, ty, erx, ery) >= 0)) {
                    tx = -tx;
                    ty = -ty;
                }
                la = lb = -1;
            } else {
                const int sg = D > 0 ? 1 : -1;
                const bool inw = sg * cross_sign(elx, ely, Nx, Ny) >= 0 &&
                                 sg * cross_sign(Nx, Ny, erx, ery) >= 0;   // lambda >= 0
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
            const bool inside = group_shoot<GL>(S, C, qt, tx, ty, la, lb, Nx, Ny, D, exact_only, gl,
                                                gmask, h, cnt);
            if (gl == 0) {
                if (inside) {                              // u is a vertex: L1, L2 carry edges
                    S.is_edge[l1] = 1;
                    S.is_edge[l2] = 1;
                } else if (h.ccw < 0) {
                    S.perr = 1;
                } else {                                   // divide the subedge at theta_3
                    const int at = atomicAdd(&S.sp, 2);
                    if (at + 2 > SMAX) {
                        S.perr = 1;
                    } else {
                        S.slx[at] = elx; S.sly[at] = ely; S.sx[at] = tx; S.sy[at] = ty;
                        S.sccw[at] = (short)l1; S.scw[at] = (short)h.cw;
                        S.slx[at + 1] = tx; S.sly[at + 1] = ty; S.sx[at + 1] = erx; S.sy[at + 1] = ery;
                        S.sccw[at + 1] = (short)h.ccw; S.scw[at + 1] = (short)l2;
                    }
                }
            }
        }
        __syncwarp();
    }
    __syncwarp();
    // the counters of the group leaders into lane 0
    {
        unsigned long long d[4] = {cnt.rays - c0.rays, cnt.vtests - c0.vtests, cnt.evals - c0.evals,
                                   cnt.exact - c0.exact};
#pragma unroll
        for (int z = 0; z < 4; z++) {
            if (gl != 0) d[z] = 0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) d[z] += __shfl_xor_sync(FULL, d[z], off);
        }
        cnt.rays = c0.rays + d[0];
        cnt.vtests = c0.vtests + d[1];
        cnt.evals = c0.evals + d[2];
        cnt.exact = c0.exact + d[3];
    }
    if (S.perr) return -1;
    // the marked edges, sorted counter-clockwise by rank
    if (lane == 0) S.nedge = 0;
    __syncwarp();
    for (int c = lane; c < C; c += 32) {
        if (S.is_edge[c]) {
            const int at = atomicAdd(&S.nedge, 1);
            if (at < EMAX) S.tmp[at] = (short)c;
        }
    }
    __syncwarp();
    const int ne = S.nedge;
    if (ne > EMAX) return -1;
    for (int q = lane; q < ne; q += 32) {
        const int a = S.tmp[q];
        int r = 0;
        for (int j = 0; j < ne; j++) r += normal_less(S, S.tmp[j], a) ? 1 : 0;
        S.emit[r] = (short)a;
    }
    __syncwarp();
    return ne;
}

// The warp tier (one warp per cell) of a single diagram runs the subedges of
// a cell on four groups of 8 lanes: few cells per warp, so a cell's latency
// sets the tier's length (uniform 1M: 0.083 -> 0.059 ms).  A batch's warp
// tier holds many cells per warp and is throughput-bound; there the
// sequential walk with 32 lanes per ray is faster (4,096 sets: 35.4 vs
// 38.0 ms), as it is for the first-pass group kernels.
constexpr int M_PAR_GROUPS = 4;
template <int G, int CMAX, int SMAX, int EMAX, int RMAX, bool USE_PAR>
__device__ __forceinline__ int run_projector(GroupSmem<CMAX, SMAX, EMAX> &S, const int C, const int gl,
                                             const unsigned gmask, const int exact_only, Counters &cnt) {
    if constexpr (G == 32 && USE_PAR)
        return projector_par<M_PAR_GROUPS, CMAX, SMAX, EMAX, RMAX>(S, C, gl, exact_only, cnt);
    else
        return projector<G, CMAX, SMAX, EMAX, RMAX>(S, C, gl, gmask, exact_only, cnt);
}

// Walk the sites of the bucket rows by0..by1 with the G lanes of a group.
// row_spans(row, x0, x1) writes up to NSPAN disjoint bucket ranges of a row
// to visit (in ascending order) and returns how many.  Each lane reads the
// site ranges of one row; for every span slot a prefix sum of the range
// lengths over the group lets the lanes take consecutive sites of the
// concatenated ranges, ILP per lane per step with their loads in flight, so
// rows of unequal length keep every lane busy and the loads overlap.
// visit(pos, site) runs once per site position.  Returns the sites visited.
template <int G, int NSPAN, int ILP, class RowSpans, class Visit>
__device__ __forceinline__ int scan_rows(const CellGrid &g, const int2 *__restrict__ sxy, int by0,
                                         int by1, int gl, unsigned gmask, RowSpans row_spans,
                                         Visit visit) {
    int seen = 0;
    for (int r0 = by0; r0 <= by1; r0 += G) {
        const int row = r0 + gl;
        int x0[NSPAN], x1[NSPAN];
        int ns = 0;
        if (row <= by1) ns = row_spans(row, x0, x1);
        int nmax = ns;
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) nmax = max(nmax, __shfl_xor_sync(gmask, nmax, off, G));
        const int *rb = g.bs + (size_t)(row <= by1 ? row : by0) * g.m1;
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
            for (int off = 1; off < G; off <<= 1) {
                const int y = __shfl_up_sync(gmask, incl, off, G);
                if (gl >= off) incl += y;
            }
            const int total = __shfl_sync(gmask, incl, G - 1, G);
            const int excl = incl - len;
            seen += total;
            for (int k0 = 0; k0 < total; k0 += ILP * G) {
                int pk[ILP];
                int2 sk[ILP];
#pragma unroll
                for (int u = 0; u < ILP; u++) {
                    const int kk = k0 + u * G + gl;
                    int j = 0;               // the last lane whose range starts at or before kk
#pragma unroll
                    for (int step = G / 2; step > 0; step >>= 1) {
                        const int ex = __shfl_sync(gmask, excl, j + step, G);
                        if (ex <= kk) j += step;
                    }
                    pk[u] = __shfl_sync(gmask, a, j, G) + kk - __shfl_sync(gmask, excl, j, G);
                    sk[u] = kk < total ? sxy[pk[u]] : make_int2(0, 0);
                }
#pragma unroll
                for (int u = 0; u < ILP; u++)
                    if (k0 + u * G + gl < total) visit(pk[u], sk[u]);
            }
        }
    }
    return seen;
}

// Buckets of a row (band [row s, row s + s] in y) that meet the disc of
// squared radius r2 around (cx, cy): the chord's x-range, widened by one unit.
__device__ __forceinline__ bool disc_row_span(const CellGrid &g, int row, int cx, int cy, i64 r2,
                                              int &x0, int &x1) {
    const i64 ylo = (i64)row * g.s, yhi = ylo + g.s;
    const i64 dy = cy < ylo ? ylo - cy : (cy > yhi ? cy - yhi : 0);
    if (dy * dy > r2) return false;
    const float h = sqrtf((float)(r2 - dy * dy)) + 1.f;   // error < 0.25 + rounding
    x0 = max(0, (int)floorf(((float)cx - h) / (float)g.s));
    x1 = min(g.m1 - 1, (int)floorf(((float)cx + h) / (float)g.s));
    return true;
}

// The parts of a row that can hold a site cutting the polygon (vertices
// S.vx/S.vy relative to p, padded radii S.vr) within the annulus
// r2lo < |a - p|^2 <= r2hi, as up to 4 disjoint ascending bucket ranges:
// the union of the vertex discs' chords (merged into at most 4 intervals; a
// fifth is folded into its nearest neighbour, which only widens the range),
// clipped to the outer disc's chord, less the part of the inner disc's
// chord that lies inside the inner disc over the whole band.  Every range
// is a superset of what it must cover; sites are tested exactly afterwards.
template <class SM>
__device__ int flower_row_spans(const CellGrid &g, const SM &S, int e, int2 p, i64 r2lo, i64 r2hi,
                                int row, int *x0, int *x1) {
    constexpr int K = 4;
    const float s = (float)g.s;
    const i64 ylo = (i64)row * g.s, yhi = ylo + g.s;
    const i64 dy = p.y < ylo ? ylo - p.y : (p.y > yhi ? p.y - yhi : 0);
    if (dy * dy > r2hi) return 0;
    const float ho = sqrtf((float)(r2hi - dy * dy)) + 1.f;
    const float olo = (float)p.x - ho, ohi = (float)p.x + ho;
    float lo[K], hi[K];
    int nk = 0;
    const float fylo = (float)ylo, fyhi = (float)yhi;
    for (int v = 0; v < e; v++) {
        const float vxa = (float)p.x + S.vx[v], vya = (float)p.y + S.vy[v], rv = S.vr[v];
        const float dv = fmaxf(0.f, fmaxf(fylo - vya, vya - fyhi));
        if (dv > rv) continue;
        const float h = sqrtf(fmaxf(rv * rv - dv * dv, 0.f)) + 1.f;
        float a = fmaxf(vxa - h, olo), b = fminf(vxa + h, ohi);
        if (a > b) continue;
        // merge into an overlapping interval, else append, else fold into
        // the nearest one
        int hit = -1;
        float best = FLT_MAX;
        int near = 0;
#pragma unroll
        for (int j = 0; j < K; j++) {
            if (j < nk) {
                if (hit < 0 && a <= hi[j] && lo[j] <= b) hit = j;
                const float gap = fmaxf(lo[j] - b, a - hi[j]);
                if (gap < best) { best = gap; near = j; }
            }
        }
        if (hit < 0 && nk < K) {
#pragma unroll
            for (int j = 0; j < K; j++) if (j == nk) { lo[j] = a; hi[j] = b; }
            nk++;
            continue;
        }
        const int j0 = hit >= 0 ? hit : near;
#pragma unroll
        for (int j = 0; j < K; j++)
            if (j == j0) { lo[j] = fminf(lo[j], a); hi[j] = fmaxf(hi[j], b); }
    }
    if (nk == 0) return 0;
    // sort (insertion, K small), then merge overlapping intervals: the
    // pieces below must come out disjoint and ascending, or a site would be
    // read (and added) twice
#pragma unroll
    for (int x = 1; x < K; x++) {
#pragma unroll
        for (int y = x; y > 0; y--) {
            if (y < nk && lo[y] < lo[y - 1]) {
                const float tl = lo[y], th = hi[y];
                lo[y] = lo[y - 1]; hi[y] = hi[y - 1];
                lo[y - 1] = tl; hi[y - 1] = th;
            }
        }
    }
    {
        int m = 1;                                       // merged intervals so far
#pragma unroll
        for (int j = 1; j < K; j++) {
            if (j < nk) {
                float last_hi = hi[0];
#pragma unroll
                for (int q = 1; q < K; q++) if (q == m - 1) last_hi = hi[q];
                if (lo[j] <= last_hi) {
#pragma unroll
                    for (int q = 0; q < K; q++) if (q == m - 1) hi[q] = fmaxf(hi[q], hi[j]);
                } else {
                    const float a = lo[j], b = hi[j];
#pragma unroll
                    for (int q = 1; q < K; q++) if (q == m) { lo[q] = a; hi[q] = b; }
                    m++;
                }
            }
        }
        nk = m;
    }
    // the inner disc over the whole band: |dy| is at most dyf there
    const i64 dyf = max(llabs(ylo - p.y), llabs(yhi - p.y));
    float ilo = 1.f, ihi = 0.f;                          // empty
    if (dyf * dyf < r2lo) {
        const float hin = sqrtf((float)(r2lo - dyf * dyf)) - 2.f;
        if (hin > 0.f) { ilo = (float)p.x - hin; ihi = (float)p.x + hin; }
    }
    // bucket ranges, merged where they touch, with the inner part removed
    int n = 0;
    int cx0 = 0, cx1 = -1;                               // the range being built
    auto emit_range = [&](float a, float b) {
        if (a > b) return;
        const int bx0 = max(0, (int)floorf(a / s)), bx1 = min(g.m1 - 1, (int)floorf(b / s));
        if (bx0 > bx1) return;
        if (cx1 >= cx0 && bx0 <= cx1 + 1) { cx0 = min(cx0, bx0); cx1 = max(cx1, bx1); return; }
        if (cx1 >= cx0) {
#pragma unroll
            for (int j = 0; j < K + 1; j++) if (j == n) { x0[j] = cx0; x1[j] = cx1; }
            n++;
        }
        cx0 = bx0;
        cx1 = bx1;
    };
#pragma unroll
    for (int j = 0; j < K; j++) {
        if (j >= nk) break;
        const float a = lo[j], b = hi[j];
        if (ilo <= ihi && a < ilo && b > ihi) {          // the inner part splits it
            emit_range(a, ilo);
            emit_range(ihi, b);
        } else if (ilo <= ihi && a >= ilo && b <= ihi) {  // entirely inside the inner disc
        } else if (ilo <= ihi && a < ilo && b >= ilo) {
            emit_range(a, ilo);
        } else if (ilo <= ihi && a <= ihi && b > ihi) {
            emit_range(ihi, b);
        } else {
            emit_range(a, b);
        }
    }
    if (cx1 >= cx0) {
#pragma unroll
        for (int j = 0; j < K + 1; j++) if (j == n) { x0[j] = cx0; x1[j] = cx1; }
        n++;
    }
    return n;
}

// Does the site n = a - p (c = |n|^2) cut the polygon of e vertices in
// S.vx/S.vy (relative to p)?  It does iff it lies strictly inside the disc
// of some vertex v through p: 2 <n, v> > c.  Float filter with a bound,
// exact (the vertex as N/D of its two lines) when the bound cannot decide.
template <class SM>
__device__ __forceinline__ bool cuts_polygon(const SM &S, int e, int nx, int ny, i64 cc) {
    const float fnx = (float)nx, fny = (float)ny, fc = fmaf(fnx, fnx, fny * fny);   // c (2u)
    for (int v = 0; v < e; v++) {
        const float vx = S.vx[v], vy = S.vy[v];
        const float f = 2.f * fmaf(fnx, vx, fny * vy) - fc;
        const float mg = 0x1p-16f * (2.f * (fabsf(fnx * vx) + fabsf(fny * vy)) + fc);
        if (f > mg) return true;
        if (f >= -mg) {
            const int la = S.emit[v], lb = S.emit[v + 1 < e ? v + 1 : 0];
            int n1x, n1y, n2x, n2y;
            i64 c1, c2, Nx, Ny, D;
            cand_int(S, la, n1x, n1y, c1);
            cand_int(S, lb, n2x, n2y, c2);
            intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
            const i128 lhs = 2 * dot128(nx, ny, Nx, Ny) * (i128)(D > 0 ? 1 : -1);
            const i128 rhs = (i128)cc * (D > 0 ? D : -D);
            if (lhs > rhs) return true;
        }
    }
    return false;
}

// Append to the candidates the sites a != p with r2lo < |a - p|^2 <= r2hi:
// all of them, or with cut_only those that cut the polygon S.vx/S.vy of e
// vertices.  With flower, only the parts of the rows that meet some vertex
// disc (S.vr radii) are read: a site outside every vertex disc cannot cut.
// Uses S.ncand as the append counter and sets S.flag when the table would
// grow past cap; with cut_only the cutters are also counted per distance
// bin in S.hist (32 bins of |a - p|^2 over (r2lo, r2hi]).  Returns the
// number of sites examined.
template <int G, int CMAX, int SMAX, int EMAX>
__device__ int scan_disc(const CellParams &P, const CellGrid &g, GroupSmem<CMAX, SMAX, EMAX> &S,
                         const int2 p, const int self, const i64 r2lo, const i64 r2hi,
                         const bool cut_only, const int e, const int cap, const int gl,
                         const unsigned gmask, Counters &cnt, const bool flower = false) {
    const int s = g.s;
    const int r = (int)ceilf(sqrtf((float)r2hi)) + 1;
    const int by0 = p.y - r <= 0 ? 0 : (p.y - r) / s;
    const int by1 = min(g.m2 - 1, (p.y + r) / s);
    const float binscale = 32.f / (float)max(r2hi - r2lo, (i64)1);
    auto visit = [&](int pos, int2 q) {
        if (pos == self) return;
        const int nx = q.x - p.x, ny = q.y - p.y;
        const i64 cc = (i64)nx * nx + (i64)ny * ny;
        if (cc <= r2lo || cc > r2hi) return;
        if (cut_only) {
            cnt.annulus++;
            if (!cuts_polygon(S, e, nx, ny, cc)) return;
            const int bin = min(31, max(0, (int)((float)(cc - r2lo) * binscale)));
            atomicAdd(&S.hist[bin], 1);
        }
        const int at = atomicAdd(&S.ncand, 1);
        if (at < cap) {
            const float fnx = (float)nx, fny = (float)ny, rc = 1.f / fmaf(fnx, fnx, fny * fny);
            S.cand[at] = make_float4(fnx, fny, rc, (float)(abs(nx) + abs(ny)) * rc);
            S.lab[at] = P.sid[pos] - g.site_base;
        } else {
            S.flag = 1;
        }
    };
    if (flower && CMAX >= 1024) {
        auto spans = [&](int row, int *x0, int *x1) -> int {
            return flower_row_spans(g, S, e, p, r2lo, r2hi, row, x0, x1);
        };
        return scan_rows<G, 5, 2>(g, P.sxy, by0, by1, gl, gmask, spans, visit);
    }
    if (flower) {
        // the bounding x-range of the vertex-disc chords in this row
        auto span = [&](int row, int *x0, int *x1) -> int {
            if (!disc_row_span(g, row, p.x, p.y, r2hi, x0[0], x1[0])) return 0;
            const float ylo = (float)row * (float)s, yhi = ylo + (float)s;
            float ulo = FLT_MAX, uhi = -FLT_MAX;
            for (int v = 0; v < e; v++) {
                const float vxa = (float)p.x + S.vx[v], vya = (float)p.y + S.vy[v], rv = S.vr[v];
                const float dv = fmaxf(0.f, fmaxf(ylo - vya, vya - yhi));
                if (dv > rv) continue;
                const float h = sqrtf(fmaxf(rv * rv - dv * dv, 0.f)) + 1.f;
                ulo = fminf(ulo, vxa - h);
                uhi = fmaxf(uhi, vxa + h);
            }
            if (ulo > uhi) return 0;
            x0[0] = max(x0[0], (int)floorf(fmaxf(ulo, -1.f) / (float)s));
            x1[0] = min(x1[0], (int)floorf(fminf(uhi, (float)g.W + 1.f) / (float)s));
            return x0[0] <= x1[0] ? 1 : 0;
        };
        return scan_rows<G, 1, 1>(g, P.sxy, by0, by1, gl, gmask, span, visit);
    }
    auto span = [&](int row, int *x0, int *x1) -> int {
        return disc_row_span(g, row, p.x, p.y, r2hi, x0[0], x1[0]) && x0[0] <= x1[0] ? 1 : 0;
    };
    return scan_rows<G, 1, 1>(g, P.sxy, by0, by1, gl, gmask, span, visit);
}

// vertices of the polygon (S.emit, e edges) into S.vx/S.vy; returns max |v-p|^2
template <int G, int CMAX, int SMAX, int EMAX>
__device__ float polygon_vertices(GroupSmem<CMAX, SMAX, EMAX> &S, const int e, const int gl,
                                  const unsigned gmask) {
    float R2 = 0.f;
    for (int q = gl; q < e; q += G) {
        const int a = S.emit[q], b = S.emit[q + 1 < e ? q + 1 : 0];
        int n1x, n1y, n2x, n2y;
        i64 c1, c2, Nx, Ny, D;
        cand_int(S, a, n1x, n1y, c1);
        cand_int(S, b, n2x, n2y, c2);
        intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
        if (D == 0) { S.flag = 2; continue; }
        const float rd = 1.f / (float)D;
        const float vx = (float)Nx * rd, vy = (float)Ny * rd;
        S.vx[q] = vx;
        S.vy[q] = vy;
        const float r2 = fmaf(vx, vx, vy * vy);
        // disc radius padded for the float vertex: relative 2^-10 (far above the
        // float error of v and of the chord computation r^2 - d^2) plus 2 units
        S.vr[q] = sqrtf(r2) * (1.f + 0x1p-10f) + 2.f;
        R2 = fmaxf(R2, r2);
    }
    return group_max<G>(R2, gmask);
}


// Large-cell certificate.  A site that is not a candidate can cut the
// polygon only if it lies strictly inside the disc of some vertex v (centre
// v, through p): the part of the polygon beyond the site's bisector holds a
// vertex v with |a - v| < |p - v| (the "flower" of the polygon is the union
// of these discs).  Invariant: every site within rho of p is a candidate or
// cuts no polygon from here on (the polygons only shrink, and so do their
// flowers).  Each round
//   1. stops when 2R <= rho (no site beyond rho can cut, Lemmas Byy'Syy' and
//      SitesInLargeSquare) or rho covers the whole box;
//   2. keeps only the candidates that carry an edge (the half-planes of the
//      others contain this polygon and every later one);
//   3. scans the annulus rho < |a - p| <= rho' (rho' = min(2 rho, 2R)),
//      reading only the parts of the bucket rows that meet the flower, and
//      adds the sites that cut the polygon (if the table would overflow, a
//      thinner annulus is scanned first);
//   4. reruns the projector with them; then every site within rho' is a
//      candidate or cuts no later polygon, and rho := rho'.
template <int G, int CMAX, int SMAX, int EMAX, int RMAX, bool ROUTE, bool PAR>
__device__ int certify_by_vertex_discs(const CellParams &P, const CellGrid &g,
                                       GroupSmem<CMAX, SMAX, EMAX> &S, const int2 p, const int i,
                                       i64 rho2, int &C, int &e, const int gl,
                                       const unsigned gmask, Counters &cnt) {
    const i64 cxf = max(p.x, g.W - p.x), cyf = max(p.y, g.H - p.y);
    const i64 far2 = cxf * cxf + cyf * cyf;            // no site is farther than a corner
    for (int round = 0; round < 4096; round++) {
        if (gl == 0) S.flag = 0;
        group_sync<G>(gmask);
        const float R2 = polygon_vertices<G>(S, e, gl, gmask);
        group_sync<G>(gmask);
        if (S.flag == 2) return CELL_FAIL;
        const i64 need = (i64)(4.f * (R2 * (1.f + 0x1p-12f) + 1.f)) + 1;   // > (2R)^2
        if (need <= rho2 || rho2 >= far2) return CELL_OK;
        if (gl == 0) {
            // keep the edge lines only: entries in ascending old index, then
            // renumber the edge list (vertex q stays between edges q, q+1)
            for (int q = 0; q < e; q++) S.tmp[q] = S.emit[q];
            for (int x = 1; x < e; x++) {
                const short key = S.tmp[x];
                int y = x - 1;
                while (y >= 0 && S.tmp[y] > key) { S.tmp[y + 1] = S.tmp[y]; y--; }
                S.tmp[y + 1] = key;
            }
            for (int q = 0; q < e; q++) {
                const int src = S.tmp[q];
                if (src != q) { S.cand[q] = S.cand[src]; S.lab[q] = S.lab[src]; }
            }
            for (int q = 0; q < e; q++) {
                int j = 0;
                while (S.tmp[j] != S.emit[q]) j++;
                S.emit[q] = (short)j;
            }
        }
        C = e;
        cnt.widen++;
        // a cell handed on to the block tier leaves this polygon (its edge
        // lines) for the block tier's first candidates
        auto hand_on = [&]() {
            if (P.seed_poly && e >= 3 && e <= SLOT_CAP) {
                const int k = P.sid[i];
                for (int q = gl; q < e; q += G) P.slot[(size_t)k * SLOT_CAP + q] = S.lab[S.emit[q]];
                if (gl == 0) P.ecount[k] = -e;
            }
            return CELL_DEFER;
        };
        i64 step2 = min(min(need, rho2 < ((i64)1 << 60) / 4 ? 4 * rho2 + 4 : rho2), far2);
        // the medium tier reads one bounding range per bucket row; a wide
        // annulus, or one over many sites (a cluster's core: the coarse
        // occupancy grid counts the sites of its bounding square), goes to
        // the block tier, which reads the vertex-disc chords row by row with
        // 8 warps
        if (CMAX < 1024 && 2.f * sqrtf((float)step2) > 256.f * (float)g.s) return hand_on();
        if (ROUTE) {
            const int r = (int)ceilf(sqrtf((float)step2)) + 1;
            const SetMeta &M = set_of(P.sets, P.sset, i);
            const int held = coarse_sites(P.coarse_sat, M, p.x - r, p.y - r, p.x + r, p.y + r);
            if (held > M_DEFER_SITES && held < M.n / 16) return hand_on();
        }
        for (int shrink = 0;; shrink++) {
            if (gl == 0) { S.ncand = C; S.flag = 0; }
            for (int q = gl; q < 32; q += G) S.hist[q] = 0;
            group_sync<G>(gmask);
            scan_disc<G>(P, g, S, p, i, rho2, step2, true, e, CMAX, gl, gmask, cnt, true);
            group_sync<G>(gmask);
            if (!S.flag) break;
            if (shrink >= 40 || step2 <= rho2 + 1) return CELL_DEFER;
            // too many cutters: the annulus up to the last distance bin whose
            // cutters, with all nearer ones, still fit (a quarter of it when
            // even the first bin does not fit)
            const int room = CMAX - C;
            int b = 0, sum = 0;
            while (b < 32 && sum + S.hist[b] <= room) sum += S.hist[b++];
            const i64 width = step2 - rho2;
            step2 = b > 0 ? rho2 + (i64)((double)width * b / 32.0) : rho2 + width / 4;
            if (step2 <= rho2) step2 = rho2 + 1;
        }
        rho2 = step2;
        const int ncut = S.ncand - C;
        if (ncut > 0) {
            cnt.reruns++;
            cnt.cands += ncut;
            C += ncut;
            e = run_projector<G, CMAX, SMAX, EMAX, RMAX, PAR>(S, C, gl, gmask, P.exact_only, cnt);
            if (e < 0) return CELL_DEFER;
            if (e < 3) return CELL_FAIL;
        }
    }
    return CELL_FAIL;
}

// Work limits of a pass: the first pass defers cells that need more.
template <bool LARGE>
struct Limits {
    static constexpr int widen = LARGE ? 64 : 2;          // certificate steps
    static constexpr int scan = LARGE ? (1 << 30) : 384;  // sites examined
};

template <int G, int CMAX, int SMAX, int EMAX, int RMAX, bool LARGE, bool ROUTE, bool PAR>
__device__ int process_cell(const CellParams &P, GroupSmem<CMAX, SMAX, EMAX> &S, int i, int gl,
                            unsigned gmask, Counters &cnt) {
    const int2 p = P.sxy[i];
    const int k = P.sid[i];                            // index in the batch
    const CellGrid g = cell_grid(P, i);
    const int kl = k - g.site_base;                    // index in its set

    // ---- 1. candidates: the sites within rho of p, then the four sides --------
    // rho is chosen so that about P.target sites fall in the disc, from the
    // site density of the 3x3 buckets around p's bucket
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
    const i64 cxf = max(p.x, g.W - p.x), cyf = max(p.y, g.H - p.y);
    const i64 far2 = cxf * cxf + cyf * cyf;           // no site is farther than a corner
    const float area = (float)nb9 * (float)s * (float)s;
    i64 rho2 = (i64)((float)P.target * area / (3.14159265f * (float)max(c9 - 1, 1)));
    rho2 = max(min(rho2, (i64)(16.f * (float)s * (float)s)), (i64)4);
    int scanned = 0;
    for (int attempt = 0;; attempt++) {
        if (gl == 0) { S.ncand = 0; S.flag = 0; }
        group_sync<G>(gmask);
        scanned += scan_disc<G>(P, g, S, p, i, -1, rho2, false, 0, CMAX - 4, gl, gmask, cnt);
        group_sync<G>(gmask);
        if (!S.flag) break;
        if (!LARGE || attempt >= 24 || rho2 <= 4) return CELL_DEFER;
        rho2 /= 4;                                     // too dense: a smaller disc
    }
    int C = S.ncand;
    if (LARGE && P.seed_poly) {
        // An earlier pass left the polygon its certificate could not accept
        // (ecount = -e, its lines in the slot).  Its sites outside the disc
        // join the candidates: extra candidates never change the cell, and
        // these lie near its final edges, so the first polygon is close to
        // the cell and the certificate's annuli find few cutters to rerun
        // the projector with.
        const int e1 = -P.ecount[k];
        if (e1 >= 3 && e1 <= SLOT_CAP) {
            const int nset = set_of(P.sets, P.sset, i).n;
            for (int q = gl; q < e1; q += G) {
                const int lab = P.slot[(size_t)k * SLOT_CAP + q];
                if (lab < 0 || lab >= nset || lab == kl) continue;
                const int2 a = __ldg(P.sites + g.site_base + lab);
                const int nx = a.x - p.x, ny = a.y - p.y;
                if ((i64)nx * nx + (i64)ny * ny <= rho2) continue;   // the disc listed it
                const int at = atomicAdd(&S.ncand, 1);
                if (at < CMAX - 4) {
                    const float fnx = (float)nx, fny = (float)ny, rc = 1.f / fmaf(fnx, fnx, fny * fny);
                    S.cand[at] = make_float4(fnx, fny, rc, (float)(abs(nx) + abs(ny)) * rc);
                    S.lab[at] = lab;
                }
            }
            group_sync<G>(gmask);
            C = min(S.ncand, CMAX - 4);
        }
    }
    if (gl == 0) {
        const int sx[4] = {0, g.W - p.x, 0, -p.x};
        const int sy[4] = {-p.y, 0, g.H - p.y, 0};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float cf = (float)(2 * ((i64)sx[q] * sx[q] + (i64)sy[q] * sy[q]));
            const float rc = 1.f / cf;
            S.cand[C + q] = make_float4((float)sx[q], (float)sy[q], rc,
                                        (float)(abs(sx[q]) + abs(sy[q])) * rc);
            S.lab[C + q] = -1 - q;
        }
    }
    C += 4;
    cnt.cands += C;
    group_sync<G>(gmask);

    // ---- 2. Algorithm 1 ----------------------------------------------------
    int e = run_projector<G, CMAX, SMAX, EMAX, RMAX, LARGE && PAR>(S, C, gl, gmask, P.exact_only, cnt);
    if (e < 0) return CELL_DEFER;
    if (e < 3) return CELL_FAIL;

    // ---- 3. security-radius certificate -------------------------------------
    if (LARGE) {
        const int rc = certify_by_vertex_discs<G, CMAX, SMAX, EMAX, RMAX, ROUTE, PAR>(P, g, S, p, i, rho2, C, e,
                                                                          gl, gmask, cnt);
        if (rc != CELL_OK) return rc;
    }
    // every site a with |a - p|^2 > rho2 has not been looked at and is
    // farther than rho
    for (int iter = 0; !LARGE; iter++) {
        const float R2 = polygon_vertices<G>(S, e, gl, gmask);
        group_sync<G>(gmask);
        if (S.flag == 2) return CELL_FAIL;
        const i64 need = (i64)(4.f * (R2 * (1.f + 0x1p-12f) + 1.f)) + 1;   // > (2R)^2
        if (need <= rho2 || rho2 >= far2) break;                          // certified
        if (iter >= Limits<LARGE>::widen) return LARGE ? CELL_FAIL : CELL_DEFER;
        cnt.widen++;
        const i64 grow = rho2 < ((i64)1 << 60) / 4 ? 4 * rho2 + 4 : rho2;
        const i64 rho2n = min(min(need, grow), far2);
        if (!LARGE) {
            const int r = (int)ceilf(sqrtf((float)rho2n)) + 1;
            const i64 nb = (i64)(2 * r / s + 2) * (2 * r / s + 2);
            if (nb * 4 > Limits<LARGE>::scan) return CELL_DEFER;
        }
        i64 step2 = rho2n;
        for (int shrink = 0;; shrink++) {
            if (gl == 0) { S.ncand = C; S.flag = 0; }
            group_sync<G>(gmask);
            scanned += scan_disc<G>(P, g, S, p, i, rho2, step2, true, e, CMAX, gl, gmask, cnt);
            group_sync<G>(gmask);
            if (!S.flag) break;
            // too many sites cut the polygon at once: test a thinner annulus
            // first (its cutters shrink the polygon, so fewer cut later)
            if (!LARGE || shrink >= 40 || step2 <= rho2 + 1) return CELL_DEFER;
            step2 = rho2 + (step2 - rho2) / 4;
        }
        rho2 = step2;
        const int ncut = S.ncand - C;
        if (ncut > 0) {
            cnt.reruns++;
            C += ncut;
            cnt.cands += ncut;
            e = run_projector<G, CMAX, SMAX, EMAX, RMAX, LARGE && PAR>(S, C, gl, gmask, P.exact_only, cnt);
            if (e < 0) return CELL_DEFER;
            if (e < 3) return CELL_FAIL;
        }
        if (!LARGE && scanned > Limits<LARGE>::scan) return CELL_DEFER;
    }

    // ---- 4. canonical order and output ----------------------------------
    int start = 0;
    {
        int bxn, byn;
        i64 dummy;
        cand_int(S, S.emit[0], bxn, byn, dummy);
        for (int q = 1; q < e; q++) {
            int qx, qy;
            cand_int(S, S.emit[q], qx, qy, dummy);
            if (angle_less(qx, qy, bxn, byn)) { start = q; bxn = qx; byn = qy; }
        }
    }
    int *dst;
    int off = -1;
    if (e <= SLOT_CAP) {
        dst = P.slot + (size_t)k * SLOT_CAP;
    } else {
        if (gl == 0) off = atomicAdd(&P.hdr->spill_top, e);
        off = __shfl_sync(gmask, off, 0, G);
        if (off + e > P.spill_cap) return CELL_DEFER;
        dst = P.spill + off;
    }
    int dcnt = 0;
    for (int q = gl; q < e; q += G) {
        int qq = start + q;
        if (qq >= e) qq -= e;
        const int lab = S.lab[S.emit[qq]];
        dst[q] = lab;
        dcnt += lab > kl ? 1 : 0;
    }
    dcnt = group_sum<G>(dcnt, gmask);
    if (gl == 0) {
        P.ecount[k] = e;
        P.dcount[k] = dcnt;
        P.loc[k] = off;
    }
    if ((unsigned long long)e > cnt.maxe) cnt.maxe = e;
    group_sync<G>(gmask);
    return CELL_OK;
}

template <int G, int CMAX, int SMAX, int EMAX, int RMAX, bool LARGE, bool ROUTE = false, bool PAR = false>
__global__ void __launch_bounds__(LARGE ? 32 : 16 * G, (LARGE && CMAX < 1024) ? 21 : 1)
cells_kernel(CellParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using SM = GroupSmem<CMAX, SMAX, EMAX>;
    if (P.hdr->err) return;
    const int lane = threadIdx.x & 31;
    const int gib = threadIdx.x / G;
    const int gl = threadIdx.x % G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((lane / G) * G));
    SM &S = reinterpret_cast<SM *>(smem_raw)[gib];
    const int gpb = blockDim.x / G;
    const int total = P.cell_list ? *P.list_count : P.n;
    Counters cnt{};
    // the large-cell pass takes cells one at a time from a shared counter
    // (their costs differ by orders of magnitude); the others stride
    int t = LARGE ? 0 : blockIdx.x * gpb + gib;
    for (;;) {
        if (LARGE) {
            if (gl == 0) t = atomicAdd(P.next_cell, 1);
            t = __shfl_sync(gmask, t, 0, G);
        }
        if (t >= total) break;
        const int i = P.cell_list ? P.cell_list[t] : t;
        const int rc = process_cell<G, CMAX, SMAX, EMAX, RMAX, LARGE, ROUTE, PAR>(P, S, i, gl, gmask, cnt);
        if (rc != CELL_OK && gl == 0) {
            if (rc == CELL_DEFER && P.deferred) {
                const int q = atomicAdd(P.deferred_count, 1);
                P.deferred[q] = i;
                cnt.deferred++;
            } else {
                atomicOr(&P.hdr->err, rc == CELL_DEFER ? ERRB_CAPACITY : ERRB_INTERNAL);
            }
        }
        group_sync<G>(gmask);
        if (!LARGE) t += gridDim.x * gpb;
    }
    if (P.collect_stats && gl == 0) {
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

// ---- configurations ----------------------------------------------------------
// first pass: 16 groups per block, small capacities, bounded certificate work
constexpr int F_CMAX = 48, F_SMAX = 20, F_EMAX = 40, F_RMAX = 40, F_GROUPS = 16;
// the medium tier: one warp per cell, one cell per block (about 7 KB of
// shared memory per warp); it hands the cells that exceed it to the
// block-per-cell tier (vor_cells_coop.cuh)
constexpr int M_CMAX = 256, M_SMAX = 64, M_EMAX = 64, M_RMAX = 256;

using FastSmem = GroupSmem<F_CMAX, F_SMAX, F_EMAX>;
using MediumSmem = GroupSmem<M_CMAX, M_SMAX, M_EMAX>;

template <int G>
cudaError_t launch_fast_g(const CellParams &P, cudaStream_t st) {
    auto kern = cells_kernel<G, F_CMAX, F_SMAX, F_EMAX, F_RMAX, false>;
    const int smem = F_GROUPS * (int)sizeof(FastSmem);
    int resident = 0;
    cudaError_t e = resident_grid((const void *)kern, F_GROUPS * G, smem, resident);
    if (e != cudaSuccess) return e;
    const int total = P.cell_list ? P.n_list : P.n;
    long long want = ((long long)total + F_GROUPS - 1) / F_GROUPS;
    long long grid = resident;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, F_GROUPS * G, smem, st>>>(P);
    return cudaGetLastError();
}

extern template cudaError_t launch_fast_g<2>(const CellParams &, cudaStream_t);
extern template cudaError_t launch_fast_g<4>(const CellParams &, cudaStream_t);
extern template cudaError_t launch_fast_g<8>(const CellParams &, cudaStream_t);
extern template cudaError_t launch_fast_g<16>(const CellParams &, cudaStream_t);
extern template cudaError_t launch_fast_g<32>(const CellParams &, cudaStream_t);

}  // namespace vor
