// vor_cells_thread.cuh -- the projector kernel, one thread per cell.
//
// The same steps as the group kernel (vor_cells.cuh): candidates from the
// disc around p, Algorithm 1 as a state machine issuing one ray per
// iteration, the FP32 filter with exact 128-bit fallback, the security-radius
// certificate and the canonical output.  Here every thread owns one cell, so
// the per-subedge control (stack, intersection, wedge test) runs once per
// cell and SIMT-parallel over the 32 cells of a warp, and a ray needs no
// cross-lane reduction.  The candidate table lives in shared memory with the
// thread index fastest (conflict-free 16-byte loads); the subedge stack, the
// edge list and the labels live in thread-local memory.
//
// The four sides of X are always candidates 0..3, so "c < 4" identifies them.
// Cells that exceed the capacities or the certificate work budget are
// deferred to the warp-per-cell pass with large capacities.
#pragma once

#include <cfloat>
#include <cmath>

#include "vor_device.cuh"
#include "vor_internal.h"

namespace vor {

namespace t1 {

struct Counters {
    unsigned long long rays, vtests, evals, exact, annulus, reruns, deferred, cands, maxe, widen;
};

enum { OK = 0, DEFER = 1, FAIL = 2 };

// candidate c of this thread: cb[c * NT] = (nx, ny, 1/c, (|nx|+|ny|)/c)
template <int NT>
struct Table {
    float4 *cb;
    __device__ __forceinline__ float4 get(int c) const { return cb[c * NT]; }
    __device__ __forceinline__ void put(int c, float4 v) const { cb[c * NT] = v; }
    __device__ __forceinline__ void line(int c, int &nx, int &ny, i64 &cc) const {
        const float4 q = get(c);
        nx = __float2int_rn(q.x);
        ny = __float2int_rn(q.y);
        cc = line_c(nx, ny, c < 4);
    }
};

__device__ __forceinline__ float4 cand_of(int nx, int ny, bool side) {
    const float cf = (float)line_c(nx, ny, side);
    const float rc = 1.f / cf;
    return make_float4((float)nx, (float)ny, rc, (float)(abs(nx) + abs(ny)) * rc);
}

// a strictly more counter-clockwise than b (normals in one open half-plane)
template <int NT>
__device__ __forceinline__ bool more_ccw(const Table<NT> &T, int a, int b) {
    int ax, ay, bx, by;
    i64 ca, cb;
    T.line(a, ax, ay, ca);
    T.line(b, bx, by, cb);
    return (i64)bx * ay - (i64)by * ax > 0;
}

// Exact endpoint over the candidates whose filter upper bound reaches thr
// (all candidates when use_thr is false); ties resolved per Remark A.4.
template <int NT>
__device__ void exact_argmax(const Table<NT> &T, int C, i64 tx, i64 ty, float fx, float fy,
                             float eth, bool use_thr, float thr, int &ccw, int &cw) {
    int best = -1;
    ccw = cw = -1;
    i128 bd = 0;
    i64 bc = 1;
    for (int c = 0; c < C; c++) {
        const float4 q = T.get(c);
        if (use_thr) {
            const float den = fmaf(q.x, fx, q.y * fy);
            if (!(fmaf(den, q.z, q.w * eth) >= thr)) continue;
        }
        int nx, ny;
        i64 cc;
        T.line(c, nx, ny, cc);
        const i128 d = dot128(nx, ny, tx, ty);
        if (d <= 0) continue;
        if (best < 0) { best = c; ccw = cw = c; bd = d; bc = cc; continue; }
        const i128 lhs = d * (i128)bc, rhs = bd * (i128)cc;     // key(c) vs key(best)
        if (lhs > rhs) { best = c; ccw = cw = c; bd = d; bc = cc; }
        else if (lhs == rhs) {
            if (more_ccw(T, c, ccw)) ccw = c;
            if (more_ccw(T, cw, c)) cw = c;
        }
    }
}

__device__ __forceinline__ int cross_sign(i64 ax, i64 ay, i64 bx, i64 by) {
    const float p = (float)ax * (float)by, q = (float)ay * (float)bx;
    const float v = p - q, bound = (fabsf(p) + fabsf(q)) * 0x1p-20f;
    if (v > bound) return 1;
    if (v < -bound) return -1;
    const i128 e = cross128(ax, ay, bx, by);
    return e > 0 ? 1 : (e < 0 ? -1 : 0);
}

// Algorithm 1 over C candidates; edges counter-clockwise into emit[].
// Returns the number of edges or -1 when a capacity is exceeded.
template <int NT, int SMAX, int EMAX, int RMAX>
__device__ int projector(const Table<NT> &T, const int C, unsigned char *emit,
                         const int exact_only, Counters &cnt) {
    long long stx[SMAX], sty[SMAX];
    unsigned char scw[SMAX], sccw[SMAX];
    int phase = 0;
    int h0c = -1, h0w = -1, h1c = -1, h1w = -1;
    i64 lx = 0, ly = 0;
    int llab = -1;
    int sp = 0, ne = 0, rays = 3, first = -1, last = -1;
    for (int guard = 0; guard < 4 * RMAX + 8; guard++) {
        // ---- the next ray ----
        bool utest = false;
        i64 tx = 0, ty = 0, Nx = 0, Ny = 0, D = 0;
        int la = -1, lb = -1;
        if (phase < 3) {
            tx = phase == 0 ? 2 : (phase == 1 ? 0 : -2);
            ty = phase == 1 ? 1 : -1;
        } else {
            bool have = false;
            while (sp > 0) {
                const int top = sp - 1;
                const i64 rx = stx[top], ry = sty[top];
                const int rcw = scw[top];
                if (llab == rcw) {                          // same line: no vertex here
                    if (llab != last) {
                        if (ne >= EMAX) return -1;
                        emit[ne++] = (unsigned char)llab;
                        if (first < 0) first = llab;
                        last = llab;
                    }
                    lx = rx; ly = ry; llab = sccw[top];
                    sp--;
                    continue;
                }
                int n1x, n1y, n2x, n2y;
                i64 c1, c2;
                T.line(llab, n1x, n1y, c1);
                T.line(rcw, n2x, n2y, c2);
                intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
                la = llab;
                lb = rcw;
                if (D == 0) {                               // parallel lines
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
                                     sg * cross_sign(Nx, Ny, rx, ry) >= 0;  // lambda >= 0
                    tx = sg * Nx;
                    ty = sg * Ny;
                    if (inw) {
                        utest = true;                       // the ray towards u
                    } else {
                        tx = -tx;                           // theta_3 := p - u
                        ty = -ty;
                        la = lb = -1;
                    }
                }
                have = true;
                break;
            }
            if (!have) break;                               // EdgeQueue is empty
        }
        // ---- the filter pass (two interleaved trackers for ILP) ----
        const float fx = (float)tx, fy = (float)ty;
        const float eth = fmaxf(fabsf(fx), fabsf(fy)) * 0x1p-19f;
        float u1a = -FLT_MAX, u2a = -FLT_MAX, lsa = -FLT_MAX, uxa = -FLT_MAX;
        float u1b = -FLT_MAX, u2b = -FLT_MAX, lsb = -FLT_MAX, uxb = -FLT_MAX;
        int i1a = -1, i1b = -1;
        int c = 0;
        for (; c + 1 < C; c += 2) {
            const float4 qa = T.get(c), qb = T.get(c + 1);
            const float da = fmaf(qa.x, fx, qa.y * fy), db = fmaf(qb.x, fx, qb.y * fy);
            const float ta = qa.w * eth, tb = qb.w * eth;
            const float Ua = fmaf(da, qa.z, ta), La = fmaf(da, qa.z, -ta);
            const float Ub = fmaf(db, qb.z, tb), Lb = fmaf(db, qb.z, -tb);
            if (Ua > u1a) { u2a = u1a; u1a = Ua; i1a = c; lsa = La; } else u2a = fmaxf(u2a, Ua);
            if (Ub > u1b) { u2b = u1b; u1b = Ub; i1b = c + 1; lsb = Lb; } else u2b = fmaxf(u2b, Ub);
            if (c != la && c != lb) uxa = fmaxf(uxa, Ua);
            if (c + 1 != la && c + 1 != lb) uxb = fmaxf(uxb, Ub);
        }
        if (c < C) {
            const float4 qa = T.get(c);
            const float da = fmaf(qa.x, fx, qa.y * fy);
            const float ta = qa.w * eth;
            const float Ua = fmaf(da, qa.z, ta), La = fmaf(da, qa.z, -ta);
            if (Ua > u1a) { u2a = u1a; u1a = Ua; i1a = c; lsa = La; } else u2a = fmaxf(u2a, Ua);
            if (c != la && c != lb) uxa = fmaxf(uxa, Ua);
        }
        // merge the trackers (ties go to the smaller index)
        float u1, u2, ls, ux = fmaxf(uxa, uxb);
        int i1;
        if (u1b > u1a || (u1b == u1a && i1b >= 0 && i1b < i1a)) {
            u1 = u1b; i1 = i1b; ls = lsb; u2 = fmaxf(fmaxf(u2a, u2b), u1a);
        } else {
            u1 = u1a; i1 = i1a; ls = lsa; u2 = fmaxf(fmaxf(u2a, u2b), u1b);
        }
        (void)u1;
        cnt.evals += C;
        // ---- decide ----
        int hc = -1, hw = -1;
        bool inside = false;
        if (utest) {
            cnt.vtests++;
            const i64 aD = D > 0 ? D : -D;
            const float kuf = (float)(aD / 2);              // key of u: |D|/2, an integer
            const float klo = kuf * (1.f - 0x1p-21f), khi = kuf * (1.f + 0x1p-21f);
            if (!exact_only && ux < klo) {
                inside = true;
            } else if (!exact_only && ls > u2 && ls > khi && i1 != la && i1 != lb) {
                hc = hw = i1;
            } else {
                cnt.exact++;
                // exact: u violates line c iff 2 <n_c, N> sgn(D) > c |D|
                bool viol = false;
                for (int q = 0; q < C && !viol; q++) {
                    if (q == la || q == lb) continue;
                    if (!exact_only) {
                        const float4 g = T.get(q);
                        const float den = fmaf(g.x, fx, g.y * fy);
                        if (fmaf(den, g.z, g.w * eth) < klo) continue;
                    }
                    int nx, ny;
                    i64 cc;
                    T.line(q, nx, ny, cc);
                    const i128 lhs = 2 * dot128(nx, ny, Nx, Ny) * (i128)(D > 0 ? 1 : -1);
                    if (lhs > (i128)cc * aD) viol = true;
                }
                if (!viol) inside = true;
                else exact_argmax(T, C, tx, ty, fx, fy, eth, !exact_only, ls, hc, hw);
            }
        } else {
            cnt.rays++;
            if (!exact_only && ls > u2 && ls > 0.f) {
                hc = hw = i1;
            } else {
                cnt.exact++;
                exact_argmax(T, C, tx, ty, fx, fy, eth, !exact_only, ls, hc, hw);
            }
        }
        // ---- update the subedge state ----
        if (phase < 3) {
            if (hc < 0) return -1;
            if (phase == 0) { h0c = hc; h0w = hw; }
            else if (phase == 1) { h1c = hc; h1w = hw; }
            else {
                lx = 2; ly = -1; llab = h0c;
                stx[0] = 2;  sty[0] = -1; scw[0] = (unsigned char)h0w; sccw[0] = (unsigned char)h0c;
                stx[1] = -2; sty[1] = -1; scw[1] = (unsigned char)hw;  sccw[1] = (unsigned char)hc;
                stx[2] = 0;  sty[2] = 1;  scw[2] = (unsigned char)h1w; sccw[2] = (unsigned char)h1c;
                sp = 3;
            }
            phase++;
        } else if (inside) {                                // u is a vertex: L1, L2 are edges
            const int top = sp - 1;
            if (la != last) {
                if (ne >= EMAX) return -1;
                emit[ne++] = (unsigned char)la;
                if (first < 0) first = la;
                last = la;
            }
            if (lb != last) {
                if (ne >= EMAX) return -1;
                emit[ne++] = (unsigned char)lb;
                if (first < 0) first = lb;
                last = lb;
            }
            lx = stx[top]; ly = sty[top]; llab = sccw[top];
            sp--;
        } else {                                            // divide the subedge at theta_3
            if (sp >= SMAX || ++rays > RMAX || hc < 0) return -1;
            stx[sp] = tx; sty[sp] = ty; scw[sp] = (unsigned char)hw; sccw[sp] = (unsigned char)hc;
            sp++;
        }
    }
    if (phase < 3 || sp > 0) return -1;
    if (ne > 1 && last == first) ne--;                      // the walk closes on its first edge
    return ne;
}

template <int NT, int CMAX, int SMAX, int EMAX, int RMAX, bool WIDEN>
__device__ int cell(const CellParams &P, const Table<NT> &T, int *lab, int i, Counters &cnt) {
    const int2 p = P.sxy[i];
    const int k = P.sid[i];
    const int s = P.hdr->s;

    // ---- 1. candidates: the four sides, then the sites within rho of p ------
    {
        const int sx[4] = {0, P.W - p.x, 0, -p.x};
        const int sy[4] = {-p.y, 0, P.H - p.y, 0};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            T.put(q, cand_of(sx[q], sy[q], true));
            lab[q] = -1 - q;
        }
    }
    int C = 4;
    const int bx = p.x / s, by = p.y / s;
    int c9 = 0, nb9 = 0;
    {
        const int x0 = max(bx - 1, 0), x1 = min(bx + 1, P.hdr->m1 - 1);
        for (int row = max(by - 1, 0); row <= min(by + 1, P.hdr->m2 - 1); row++) {
            c9 += P.bstart[row * P.hdr->m1 + x1 + 1] - P.bstart[row * P.hdr->m1 + x0];
            nb9 += x1 - x0 + 1;
        }
    }
    const i64 cxf = max(p.x, P.W - p.x), cyf = max(p.y, P.H - p.y);
    const i64 far2 = cxf * cxf + cyf * cyf;            // no site is farther than a corner
    const float area = (float)nb9 * (float)s * (float)s;
    i64 rho2 = (i64)((float)P.target * area / (3.14159265f * (float)max(c9 - 1, 1)));
    rho2 = max(min(rho2, (i64)(16.f * (float)s * (float)s)), (i64)4);
    int scanned = 0;
    {
        const int r = (int)ceilf(sqrtf((float)rho2)) + 1;
        const int bx0 = p.x - r <= 0 ? 0 : (p.x - r) / s, bx1 = min(P.hdr->m1 - 1, (p.x + r) / s);
        const int by0 = p.y - r <= 0 ? 0 : (p.y - r) / s, by1 = min(P.hdr->m2 - 1, (p.y + r) / s);
        for (int row = by0; row <= by1; row++) {
            const int a = P.bstart[row * P.hdr->m1 + bx0], b = P.bstart[row * P.hdr->m1 + bx1 + 1];
            scanned += b - a;
            for (int pos = a; pos < b; pos++) {
                if (pos == i) continue;
                const int2 q = P.sxy[pos];
                const int nx = q.x - p.x, ny = q.y - p.y;
                if ((i64)nx * nx + (i64)ny * ny > rho2) continue;
                if (C >= CMAX) return DEFER;
                T.put(C, cand_of(nx, ny, false));
                lab[C++] = P.sid[pos];
            }
        }
    }
    cnt.cands += C;

    // ---- 2. Algorithm 1 ----------------------------------------------------
    unsigned char emit[EMAX];
    int e = projector<NT, SMAX, EMAX, RMAX>(T, C, emit, P.exact_only, cnt);
    if (e < 0) return DEFER;
    if (e < 3) return FAIL;

    // ---- 3. security-radius certificate -------------------------------------
    float vx[EMAX], vy[EMAX];
    for (int iter = 0;; iter++) {
        float R2 = 0.f;
        for (int q = 0; q < e; q++) {
            int n1x, n1y, n2x, n2y;
            i64 c1, c2, Nx, Ny, D;
            T.line(emit[q], n1x, n1y, c1);
            T.line(emit[q + 1 < e ? q + 1 : 0], n2x, n2y, c2);
            intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
            if (D == 0) return FAIL;
            const float rd = 1.f / (float)D;
            vx[q] = (float)Nx * rd;
            vy[q] = (float)Ny * rd;
            R2 = fmaxf(R2, fmaf(vx[q], vx[q], vy[q] * vy[q]));
        }
        const i64 need = (i64)(4.f * (R2 * (1.f + 0x1p-12f) + 1.f)) + 1;   // > (2R)^2
        if (need <= rho2 || rho2 >= far2) break;                          // certified
        if (!WIDEN || iter >= 3) return DEFER;      // the first pass hands these cells on
        cnt.widen++;
        const i64 rho2n = min(min(need, 4 * rho2 + 4), far2);
        const int r = (int)ceilf(sqrtf((float)rho2n)) + 1;
        const int bx0 = p.x - r <= 0 ? 0 : (p.x - r) / s, bx1 = min(P.hdr->m1 - 1, (p.x + r) / s);
        const int by0 = p.y - r <= 0 ? 0 : (p.y - r) / s, by1 = min(P.hdr->m2 - 1, (p.y + r) / s);
        if ((by1 - by0 + 1) * (bx1 - bx0 + 1) > 128) return DEFER;
        const int C0 = C;
        for (int row = by0; row <= by1; row++) {
            const int a = P.bstart[row * P.hdr->m1 + bx0], b = P.bstart[row * P.hdr->m1 + bx1 + 1];
            scanned += b - a;
            for (int pos = a; pos < b; pos++) {
                const int2 q = P.sxy[pos];
                const int nx = q.x - p.x, ny = q.y - p.y;
                const i64 cc = (i64)nx * nx + (i64)ny * ny;
                if (cc <= rho2 || cc > rho2n) continue;
                cnt.annulus++;
                const float fnx = (float)nx, fny = (float)ny, fc = (float)cc;
                bool cut = false;
                for (int v = 0; v < e && !cut; v++) {
                    const float f = 2.f * fmaf(fnx, vx[v], fny * vy[v]) - fc;
                    const float mg = 0x1p-16f * (2.f * (fabsf(fnx * vx[v]) + fabsf(fny * vy[v])) + fc);
                    if (f > mg) cut = true;
                    else if (f >= -mg) {
                        int n1x, n1y, n2x, n2y;
                        i64 c1, c2, Nx, Ny, D;
                        T.line(emit[v], n1x, n1y, c1);
                        T.line(emit[v + 1 < e ? v + 1 : 0], n2x, n2y, c2);
                        intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
                        const i128 lhs = 2 * dot128(nx, ny, Nx, Ny) * (i128)(D > 0 ? 1 : -1);
                        if (lhs > (i128)cc * (D > 0 ? D : -D)) cut = true;
                    }
                }
                if (!cut) continue;
                if (C >= CMAX) return DEFER;
                T.put(C, cand_of(nx, ny, false));
                lab[C++] = P.sid[pos];
            }
        }
        rho2 = rho2n;
        if (C > C0) {
            cnt.reruns++;
            cnt.cands += C - C0;
            e = projector<NT, SMAX, EMAX, RMAX>(T, C, emit, P.exact_only, cnt);
            if (e < 0) return DEFER;
            if (e < 3) return FAIL;
        }
        if (scanned > 1024) return DEFER;
    }

    // ---- 4. canonical order and output ----------------------------------
    int start = 0;
    {
        int bxn, byn, qx, qy;
        i64 dummy;
        T.line(emit[0], bxn, byn, dummy);
        for (int q = 1; q < e; q++) {
            T.line(emit[q], qx, qy, dummy);
            if (angle_less(qx, qy, bxn, byn)) { start = q; bxn = qx; byn = qy; }
        }
    }
    int *dst;
    int off = -1;
    if (e <= SLOT_CAP) {
        dst = P.slot + (size_t)k * SLOT_CAP;
    } else {
        off = atomicAdd(&P.hdr->spill_top, e);
        if (off + e > P.spill_cap) return DEFER;
        dst = P.spill + off;
    }
    int dcnt = 0;
    for (int q = 0; q < e; q++) {
        int qq = start + q;
        if (qq >= e) qq -= e;
        const int l = lab[emit[qq]];
        dst[q] = l;
        dcnt += l > k ? 1 : 0;
    }
    P.ecount[k] = e;
    P.dcount[k] = dcnt;
    P.loc[k] = off;
    if ((unsigned long long)e > cnt.maxe) cnt.maxe = e;
    return OK;
}

}  // namespace t1

// WIDEN = false: first pass over all cells, the cells the disc does not
// certify are handed on; WIDEN = true: second pass over that list, the
// certificate may grow the disc.
template <int NT, int CMAX, int SMAX, int EMAX, int RMAX, bool WIDEN>
__global__ void __launch_bounds__(NT) cells_thread_kernel(CellParams P) {
    extern __shared__ __align__(16) float4 tbl_raw[];
    if (P.hdr->err) return;
    const t1::Table<NT> T{tbl_raw + threadIdx.x};
    int lab[CMAX];
    t1::Counters cnt{};
    const int total = P.cell_list ? *P.list_count : P.n;
    for (int t = blockIdx.x * NT + threadIdx.x; t < total; t += gridDim.x * NT) {
        const int i = P.cell_list ? P.cell_list[t] : t;
        const int rc = t1::cell<NT, CMAX, SMAX, EMAX, RMAX, WIDEN>(P, T, lab, i, cnt);
        if (rc != t1::OK) {
            if (rc == t1::DEFER && P.deferred) {
                const int q = atomicAdd(P.deferred_count, 1);
                P.deferred[q] = i;
                cnt.deferred++;
            } else {
                atomicOr(&P.hdr->err, rc == t1::DEFER ? ERRB_CAPACITY : ERRB_INTERNAL);
            }
        }
    }
    if (P.collect_stats) {
        // one atomic per warp and counter
        unsigned long long v[10] = {cnt.rays, cnt.vtests, cnt.evals, cnt.exact, cnt.annulus,
                                    cnt.reruns, cnt.deferred, cnt.cands, cnt.widen, cnt.maxe};
#pragma unroll
        for (int q = 0; q < 10; q++) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[q], off);
                v[q] = q == 9 ? (o > v[q] ? o : v[q]) : v[q] + o;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            unsigned long long *st = P.hdr->stats;
            atomicAdd(&st[STAT_RAYS], v[0]);
            atomicAdd(&st[STAT_VTESTS], v[1]);
            atomicAdd(&st[STAT_EVALS], v[2]);
            atomicAdd(&st[STAT_EXACT], v[3]);
            atomicAdd(&st[STAT_ANNULUS], v[4]);
            atomicAdd(&st[STAT_RERUNS], v[5]);
            atomicAdd(&st[STAT_DEFERRED], v[6]);
            atomicAdd(&st[STAT_CANDIDATES], v[7]);
            atomicAdd(&st[STAT_WIDEN], v[8]);
            atomicMax(&st[STAT_MAXE], v[9]);
        }
    }
}

// one thread per cell: 64 threads per block, 44 candidates per thread (4 sides + 40 sites)
constexpr int T_NT = 64, T_CMAX = 44, T_SMAX = 16, T_EMAX = 32, T_RMAX = 32;

}  // namespace vor
