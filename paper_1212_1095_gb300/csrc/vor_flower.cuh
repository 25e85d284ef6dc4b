// vor_flower.cuh -- the flower gather of the thread-per-cell flower passes:
// one warp lists the candidates of one cell from the polygon an earlier pass
// left in the cell's slot.
//
// A site a cuts a convex polygon P around p exactly when it lies strictly
// inside the disc of some vertex w of P through p: |x - p|^2 - |x - a|^2 is
// affine in x, so its maximum over P is reached at a vertex.  (The sites of
// P's own edges lie on such circles.)  The polygon's "flower" (the union of
// these discs) therefore holds every site that can still change the cell;
// the farther sites are never needed (the argument of Lemmas Byy'Syy' and
// SitesInLargeSquare, with the vertex discs in place of the disc of radius
// 2R).
//
// The warp reads the bucket rows that meet the flower, nearest p first and
// within a budget of sites (lanes over rows, a prefix sum over the row
// ranges so that every lane takes sites), tests each site against the
// vertex discs (a float test with a margin: a superset), and histograms the
// distances of the flower's sites from p.  When the whole flower was read
// and fits the list, the list is complete: the cell among the listed sites
// is the Voronoi cell, and its certificate radius is unbounded.  Otherwise
// the list takes the flower's sites nearest to p up to a distance rho that
// fits (and that the rows read cover), and the usual certificate 2R <= rho
// decides: every site within rho that could cut is listed, and the ones that
// cannot cut P cannot cut the smaller polygon computed from the list either.
// A cell the certificate does not accept leaves its new polygon for the
// next flower pass.
#pragma once

#include <climits>

#include "vor_cells.cuh"
#include "vor_cells_persist.cuh"

namespace vor {

constexpr int FL_WARPS = 4;            // warps per block
constexpr int FL_ROWS = 256;           // bucket rows a flower may span
constexpr int FL_SITES = 1024;         // sites the rows read may hold
// Below this many cells the pass is left out (every cell goes to the warp
// tier): a few cells of up to 124 candidates each on one thread take longer
// than the same cells spread over the lanes of a warp; the pass pays off
// when its cells fill the GPU.
constexpr int FL_MIN_CELLS = 16384;

// The line of label lab (a site of the cell's set, or a side -1..-4) in the
// cell of p: 2 <n, v - p> = c.
__device__ __forceinline__ void label_line(const CellParams &P, const CellGrid &g, int2 p, int lab,
                                           int &nx, int &ny, i64 &c) {
    if (lab >= 0) {
        const int2 a = __ldg(P.sites + g.site_base + lab);
        nx = a.x - p.x;
        ny = a.y - p.y;
        c = (i64)nx * nx + (i64)ny * ny;
        return;
    }
    nx = ny = 0;
    if (lab == VOR_SIDE_BOTTOM) ny = -p.y;
    else if (lab == VOR_SIDE_RIGHT) nx = g.W - p.x;
    else if (lab == VOR_SIDE_TOP) ny = g.H - p.y;
    else nx = -p.x;
    c = 2 * ((i64)nx * nx + (i64)ny * ny);
}

struct FlowerSmem {
    float wx[SLOT_CAP], wy[SLOT_CAP], wr[SLOT_CAP];   // vertices relative to p, padded radii
    int hist[32];
    int cnt;
    int held[FL_ROWS];                                 // sites in each row's range
    unsigned short disc[FL_ROWS];                      // vertex discs meeting each row's band
};

// does the site n = a - p lie inside or on (with a margin) one of the
// vertex discs in the bit set `discs` (those meeting the site's row band)?
__device__ __forceinline__ bool in_flower(const FlowerSmem &F, unsigned discs, int nx, int ny) {
    const float fnx = (float)nx, fny = (float)ny;
    const float nn = fmaf(fnx, fnx, fny * fny);
    while (discs) {
        const int q = __ffs(discs) - 1;
        discs &= discs - 1;
        const float px = fnx * F.wx[q], py = fny * F.wy[q];
        const float f = 2.f * (px + py) - nn;
        const float mg = 0x1p-16f * (2.f * (fabsf(px) + fabsf(py)) + nn) + 1.f;
        if (f > -mg) return true;
    }
    return false;
}

template <int GMAX>
__global__ void __launch_bounds__(32 * FL_WARPS) flower_gather_kernel(CellParams P, GatherOut G) {
    __shared__ FlowerSmem sm[FL_WARPS];
    if (P.hdr->err) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    FlowerSmem &F = sm[wib];
    const int listed = *P.list_count;
    const int total = listed < FL_MIN_CELLS ? 0 : min(listed, G.cap);
    const int nwarps = gridDim.x * FL_WARPS;
    for (int t = total + blockIdx.x * blockDim.x + threadIdx.x; t < listed; t += gridDim.x * blockDim.x)
        G.count[t] = -1;                                   // beyond the lists: the next tier
    for (int t = blockIdx.x * FL_WARPS + wib; t < total; t += nwarps) {
        const int i = P.cell_list[t];
        const int2 p = P.sxy[i];
        const CellGrid g = cell_grid(P, i);
        const int k = __ldg(P.sid + i);
        const int e1 = -P.ecount[k];
        if (e1 < 3 || e1 > SLOT_CAP) {                     // no polygon: the next tier
            if (lane == 0) { G.count[t] = -1; G.rho2[t] = 0; }
            continue;
        }
        // the polygon's lines, one per lane, then vertex q = lines q and q + 1
        int nx = 0, ny = 0;
        i64 c = 0;
        if (lane < e1) label_line(P, g, p, P.slot[(size_t)k * SLOT_CAP + lane], nx, ny, c);
        const int src = lane + 1 < e1 ? lane + 1 : 0;
        const int n2x = __shfl_sync(FULL, nx, src), n2y = __shfl_sync(FULL, ny, src);
        const i64 c2 = __shfl_sync(FULL, c, src);
        float ylo = FLT_MAX, yhi = -FLT_MAX, r2max = 0.f;
        int bad = 0;
        if (lane < e1) {
            i64 Nx, Ny, D;
            intersect(nx, ny, c, n2x, n2y, c2, Nx, Ny, D);
            if (D == 0) {
                bad = 1;
            } else {
                const float rd = 1.f / (float)D;
                const float wx = (float)Nx * rd, wy = (float)Ny * rd;
                // radius through p, padded for the float vertex
                const float wr = sqrtf(fmaf(wx, wx, wy * wy)) * (1.f + 0x1p-10f) + 2.f;
                F.wx[lane] = wx;
                F.wy[lane] = wy;
                F.wr[lane] = wr;
                ylo = (float)p.y + wy - wr;
                yhi = (float)p.y + wy + wr;
                const float far = sqrtf(fmaf(wx, wx, wy * wy)) + wr;   // farthest flower point from p
                r2max = far * far;
            }
        }
        F.hist[lane] = 0;
        if (lane == 0) F.cnt = 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            ylo = fminf(ylo, __shfl_xor_sync(FULL, ylo, off));
            yhi = fmaxf(yhi, __shfl_xor_sync(FULL, yhi, off));
            r2max = fmaxf(r2max, __shfl_xor_sync(FULL, r2max, off));
            bad |= __shfl_xor_sync(FULL, bad, off);
        }
        const int s = g.s;
        const int prow = p.y / s;
        // the rows of the flower, at most FL_ROWS of them around p's row
        int by0 = max(0, (int)floorf(ylo / (float)s));
        int by1 = min(g.m2 - 1, (int)floorf(yhi / (float)s));
        by0 = max(by0, prow - FL_ROWS / 2 + 1);
        by1 = min(by1, prow + FL_ROWS / 2);
        if (bad) {
            if (lane == 0) { G.count[t] = -1; G.rho2[t] = 0; }
            continue;
        }
        // distance from p to the band of a row (0 for p's own row)
        auto row_dist = [&](int row) -> float {
            return row > prow ? (float)row * (float)s - (float)p.y
                              : (row < prow ? (float)p.y - (float)(row + 1) * (float)s : 0.f);
        };
        __syncwarp();
        // the row ranges meeting the flower: the union of the vertex discs'
        // chords over the row's band
        unsigned discs = 0;                                // of the last row given to span
        auto span = [&](int row, int *x0, int *x1) -> int {
            const float fy0 = (float)row * (float)s, fy1 = fy0 + (float)s;
            float xlo = FLT_MAX, xhi = -FLT_MAX;
            discs = 0;
            for (int q = 0; q < e1; q++) {
                const float cy = (float)p.y + F.wy[q];
                const float dv = fmaxf(0.f, fmaxf(fy0 - cy, cy - fy1));
                if (dv > F.wr[q]) continue;
                const float h = sqrtf(fmaxf(F.wr[q] * F.wr[q] - dv * dv, 0.f)) + 1.f;
                const float cx = (float)p.x + F.wx[q];
                xlo = fminf(xlo, cx - h);
                xhi = fmaxf(xhi, cx + h);
                discs |= 1u << q;
            }
            if (xlo > xhi) return 0;
            x0[0] = max(0, (int)floorf(fmaxf(xlo, -1.f) / (float)s));
            x1[0] = min(g.m1 - 1, (int)floorf(fminf(xhi, (float)g.W + 1.f) / (float)s));
            return x0[0] <= x1[0] ? 1 : 0;
        };
        // the sites each row's range holds; the rows nearest p (in order of
        // |row - prow|) are read while they hold at most FL_SITES sites in
        // all, and the radius rt is the distance from p to the nearest row
        // left out (or cut off by the FL_ROWS window): every site closer to p
        // than rt lies in the rows read
        for (int r0 = by0; r0 <= by1; r0 += 32) {
            const int row = r0 + lane;
            int x0, x1;
            if (row <= by1) {
                F.held[row - by0] = span(row, &x0, &x1) ? g.bs[row * g.m1 + x1 + 1] - g.bs[row * g.m1 + x0] : 0;
                F.disc[row - by0] = (unsigned short)discs;
            }
        }
        __syncwarp();
        int lo = prow, hi = prow - 1;                      // rows read: [lo, hi]
        {
            int sum = 0;
            for (int kk = 0;; kk++) {
                const int h = (kk + 1) >> 1;
                const int row = (kk & 1) ? prow + h : prow - h;
                if (h > FL_ROWS) break;
                if (row < by0 || row > by1) {
                    if (prow + h > by1 && prow - h < by0) break;
                    continue;
                }
                const int add = F.held[row - by0];
                if (sum + add > FL_SITES) break;
                sum += add;
                lo = min(lo, row);
                hi = max(hi, row);
            }
        }
        float rt = FLT_MAX;
        if (hi >= lo) {
            // rows beyond [lo, hi] that the flower reaches, or the window cut
            const int top = min(g.m2 - 1, (int)floorf(yhi / (float)s));
            const int bot = max(0, (int)floorf(ylo / (float)s));
            if (hi < top) rt = fminf(rt, row_dist(hi + 1));
            if (lo > bot) rt = fminf(rt, row_dist(lo - 1));
        }
        if (hi < lo || rt < 1.f) {                         // not even p's own row fits
            if (lane == 0) { G.count[t] = -1; G.rho2[t] = 0; }
            __syncwarp();
            continue;
        }
        const int rb0 = by0;                               // the pre-pass's first row (F.held, F.disc)
        by0 = lo;
        by1 = hi;
        // the listed sites lie closer than sqrt(lim2) (integer, at most rt^2)
        i64 lim2 = LLONG_MAX;
        if (rt < FLT_MAX) {
            lim2 = (i64)(rt * rt * (1.f - 0x1p-20f));
            if (lim2 < 2) {
                if (lane == 0) { G.count[t] = -1; G.rho2[t] = 0; }
                __syncwarp();
                continue;
            }
            r2max = fminf(r2max, (float)lim2);
        }
        // two walks over the same rows with one copy of the walk's code: the
        // first counts the flower's sites by distance from p (32 bins of
        // |a - p|^2), the second lists those that fit (entry order does not
        // change the cell)
        const float binscale = 32.f / fmaxf(r2max, 1.f);
        bool listing = false;
        i64 rho2 = 0;
        auto visit = [&](int pos, int2 q) {
            if (pos == i) return;
            const int ax = q.x - p.x, ay = q.y - p.y;
            const i64 dd = (i64)ax * ax + (i64)ay * ay;
            if (dd >= lim2 || !in_flower(F, F.disc[q.y / s - rb0], ax, ay)) return;
            if (!listing) {
                atomicAdd(&F.hist[min(31, (int)((float)dd * binscale))], 1);
                return;
            }
            const int at = atomicAdd(&F.cnt, 1);
            if (at < GMAX) {
                G.tab[G.at(t, at)] = t1::cand_of(ax, ay);
                G.lab[G.at(t, at)] = __ldg(P.sid + pos) - g.site_base;
            }
        };
        bool done = false;
#pragma unroll 1
        for (int walk = 0; walk < 2; walk++) {
            scan_rows<32, 1, 2>(g, P.sxy, by0, by1, lane, FULL, span, visit);
            __syncwarp();
            if (walk == 1) break;
            // the nearest bins that fit: all of them (a complete list), or
            // those below bin b (every flower site with |a - p|^2 < b r2max / 32)
            int b = 0, sum = 0;
            while (b < 32 && sum + F.hist[b] <= GMAX) sum += F.hist[b++];
            if (b < 32) lim2 = min(lim2, (i64)((float)b / binscale));   // the bins below b
            // certificate radius: unbounded when the whole flower is listed,
            // else every flower site with |a - p|^2 <= rho2 is listed
            rho2 = lim2 == LLONG_MAX ? LLONG_MAX : lim2 - 1;
            if (rho2 < 1) {
                if (lane == 0) { G.count[t] = -1; G.rho2[t] = 0; }
                done = true;
                break;
            }
            listing = true;
        }
        if (done) continue;
        if (lane == 0) {
            const int n_list = F.cnt;
            G.count[t] = n_list <= GMAX ? n_list : -1;
            G.rho2[t] = rho2;
        }
        __syncwarp();
    }
}

}  // namespace vor
