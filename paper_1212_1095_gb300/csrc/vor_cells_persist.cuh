// vor_cells_persist.cuh -- the first pass of the projector: gather kernel and
// persistent one-thread-per-cell projector kernel.
//
// gather_kernel (one thread per cell): picks the disc radius rho from the
// site density of the 3x3 buckets around p (about `target` sites inside) and
// lists the sites within rho (offset from p and label).
//
// cells_persist_kernel: every thread works through a sequence of cells; a
// cell is loaded from its list into the thread's shared-memory candidate
// table, Algorithm 1 runs one ray per loop iteration, and when the cell's
// EdgeQueue is empty the thread finalises it (certificate check, canonical
// output) and takes its next cell.  Loading and finalising are batched with
// warp ballots: a thread that finished waits until every lane of its warp is
// idle, so the per-cell bookkeeping (latency-bound: loads, the certificate)
// runs once per generation of 32 cells with all lanes active, and the cells
// of a generation start together, which keeps their rays' candidate scans
// converged (measured: 1.24 ms with refills at 8 idle lanes, 0.97 ms with
// all 32, uniform 1M sites).  A cell whose disc does not certify the polygon
// (2R > rho) is handed to the second pass, which grows the disc.
#pragma once

#include <climits>

#include "vor_cells_thread.cuh"

namespace vor {

constexpr int P_NT = 64, P_SMAX = 16, P_EMAX = 16, P_RMAX = 32;
constexpr int P_REFILL = 32;         // idle lanes that trigger a batched refill (all)
// first pass: 4 sides + up to 40 sites; second pass (the cells the first
// disc did not certify): a disc with about 2.2 times the sites, 4 + 72
// entries; flower passes: the flower of the polygon an earlier pass left
// (vor_flower.cuh), 4 + 124 entries
constexpr int P1_CMAX = 44, P2_CMAX = 76, P3_CMAX = 128;

// cp.async (sm_80+): an 8-byte copy from global to shared memory that runs
// without registers; wait_all waits for this thread's copies only
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

struct GatherOut {
    int *count;        // sites in the disc per cell (-1: more than gmax, or t >= cap)
    long long *rho2;   // squared disc radius per cell
    float2 *tab;       // gmax candidates per cell: (nx, ny) = site - p, as floats (exact)
    int *lab;          // gmax labels per cell: the site's index in its set
    int gmax;
    int cap;           // cells the lists hold (later cells go to the next pass)
    // The rows are stored in tiles of 32 consecutive rows; inside a tile
    // entry-major, so that entry q of the 32 rows a projector warp loads
    // together is one contiguous 256-byte range and the warp's whole load
    // stays inside one tile (a few pages, however many rows there are).
    // The buffers hold whole tiles.
    __device__ __forceinline__ size_t at(int t, int q) const {
        return (size_t)(t >> 5) * ((size_t)gmax * 32) + (size_t)q * 32 + (t & 31);
    }
};

// The first disc of the cell of p: the radius rho (squared) for about
// `target` sites inside, from the site density of the 3x3 buckets around p,
// and the bucket rows it meets.
struct Disc {
    i64 rho2;
    int r, by0, by1;        // r >= rho + 1, rows by0..by1
};

// the rows of the disc of squared radius rho2 around p
__device__ __forceinline__ Disc disc_of(const CellGrid &g, int2 p, i64 rho2) {
    Disc d;
    d.rho2 = rho2;
    d.r = (int)ceilf(sqrtf((float)d.rho2)) + 1;
    d.by0 = p.y - d.r <= 0 ? 0 : (p.y - d.r) / g.s;
    d.by1 = min(g.m2 - 1, (p.y + d.r) / g.s);
    return d;
}

__device__ __forceinline__ Disc first_disc(const CellGrid &g, int2 p, float target) {
    const int s = g.s;
    const int bx = p.x / s, by = p.y / s;
    int c9 = 0;
    float area;
    const int b = by * g.m1 + bx;
    const int off = g.fd ? g.fd[b] : -1;
    if (off >= 0) {
        // a divided bucket: the density of the (up to) 3 x 3 sub-buckets
        // around p's inside the bucket
        const int a0 = g.bs[b];
        const int F = 1 << fine_log2(g.bs[b + 1] - a0);
        const int sx = (p.x - bx * s) * F / s, sy = (p.y - by * s) * F / s;
        const int x0 = max(sx - 1, 0), x1 = min(sx + 1, F - 1);
        const int y0 = max(sy - 1, 0), y1 = min(sy + 1, F - 1);
        const int *sp = g.fp + off;
        for (int j = y0; j <= y1; j++) c9 += sp[j * F + x1 + 1] - sp[j * F + x0];
        const float ss = (float)s / (float)F;
        area = (float)((x1 - x0 + 1) * (y1 - y0 + 1)) * ss * ss;
    } else {
        int nb9 = 0;
        const int x0 = max(bx - 1, 0), x1 = min(bx + 1, g.m1 - 1);
        for (int row = max(by - 1, 0); row <= min(by + 1, g.m2 - 1); row++) {
            c9 += g.bs[row * g.m1 + x1 + 1] - g.bs[row * g.m1 + x0];
            nb9 += x1 - x0 + 1;
        }
        area = (float)nb9 * (float)s * (float)s;
    }
    i64 rho2 = (i64)(target * area / (3.14159265f * (float)max(c9 - 1, 1)));
    rho2 = max(min(rho2, (i64)(16.f * (float)s * (float)s)), (i64)4);
    return disc_of(g, p, rho2);
}

// The buckets bx0..bx1 of bucket row `row` that meet the disc (its chord,
// widened by one unit); false when none does.  bx0 >= (p.x - r) / s and
// bx1 <= (p.x + r) / s.
__device__ __forceinline__ bool chord_cols(const CellGrid &g, int2 p, i64 rho2, int row, int &bx0,
                                           int &bx1) {
    const int s = g.s;
    const i64 ylo = (i64)row * s, yhi = ylo + s;
    const i64 dy = p.y < ylo ? ylo - p.y : (p.y > yhi ? p.y - yhi : 0);
    if (dy * dy > rho2) return false;
    const float h = sqrtf((float)(rho2 - dy * dy)) + 1.f;
    bx0 = max(0, (int)floorf(((float)p.x - h) / (float)s));
    bx1 = min(g.m1 - 1, (int)floorf(((float)p.x + h) / (float)s));
    return bx0 <= bx1;
}

// The sites of bucket row `row`, buckets bx0..bx1 (the chord of the disc of
// squared radius rho2 around p), as ranges [a, b) of sorted positions passed
// to fn in ascending order: a bucket that is not divided whole (neighbours
// merged into one range), a divided bucket only its sub-buckets that meet
// the disc: the sub-rows within reach and in each the columns of the chord
// at that sub-row's band.  Every site of those buckets within the disc lies
// in a range.
template <class Fn>
__device__ __forceinline__ void disc_row_ranges(const CellGrid &g, int2 p, i64 rho2, int row, int bx0,
                                                int bx1, Fn fn) {
    const int *rb = g.bs + (size_t)row * g.m1;
    if (!g.fd) {
        fn(rb[bx0], rb[bx1 + 1]);
        return;
    }
    const int *rf = g.fd + (size_t)row * g.m1;
    const int s = g.s;
    int run = rb[bx0];                                 // start of the pending whole buckets
    for (int bx = bx0; bx <= bx1; bx++) {
        const int off = rf[bx];
        if (off < 0) continue;
        const int a0 = rb[bx], a1 = rb[bx + 1];
        if (a0 > run) fn(run, a0);
        run = a1;
        const int F = 1 << fine_log2(a1 - a0);
        const int *sp = g.fp + off;
        // sub-rows j hold the sites with (y - row s) F / s = j (integer division)
        const int r = (int)ceilf(sqrtf((float)rho2)) + 1;
        const int y0 = row * s;
        const int lya = max(p.y - r - y0, 0), lyb = min(p.y + r - y0, s - 1);
        if (lya > lyb) continue;
        const int xb0 = bx * s;
        for (int j = lya * F / s; j <= lyb * F / s; j++) {
            // the integer band of sub-row j: y0 + ceil(j s / F) .. y0 + ceil((j + 1) s / F) - 1
            const int ylo = y0 + (j * s + F - 1) / F, yhi = y0 + ((j + 1) * s + F - 1) / F - 1;
            if (ylo > yhi) continue;
            const i64 dy = p.y < ylo ? ylo - p.y : (p.y > yhi ? p.y - yhi : 0);
            if (dy * dy > rho2) continue;
            const float h = sqrtf((float)(rho2 - dy * dy)) + 1.f;   // as chord_cols
            const int xa = max((int)floorf((float)p.x - h) - xb0, 0);
            const int xe = min((int)floorf((float)p.x + h) - xb0, s - 1);
            if (xa > xe) continue;
            const int u = sp[j * F + xa * F / s], v = sp[j * F + xe * F / s + 1];
            if (v > u) fn(a0 + u, a0 + v);
        }
    }
    if (rb[bx1 + 1] > run) fn(run, rb[bx1 + 1]);
}

// One thread per cell: the cells are the sorted positions t < P.n, or
// P.cell_list[t] for t < *P.list_count; outputs are indexed by t.  Each
// candidate is written in the form the projector's table holds, so loading a
// cell is a plain copy.  With STAGE, a block stages its cells' lists in
// shared memory (one padded row per cell) and writes them out as one
// contiguous range; without, each thread writes its own row (the second
// pass, whose longer lists would limit the block to one warp).
template <int NT, int GMAX, bool STAGE, bool FINE>
__global__ void __launch_bounds__(NT) gather_kernel(CellParams P, GatherOut G, float target) {
    __shared__ float2 stab[STAGE ? NT * (GMAX + 1) : 1];
    __shared__ int slab[STAGE ? NT * (GMAX + 1) : 1];
    if (P.hdr->err) return;
    const int total = P.cell_list ? *P.list_count : P.n;
    const int t0 = blockIdx.x * NT;
    if (t0 >= total) return;
    const int t = t0 + threadIdx.x;
    float2 *rtab = STAGE ? stab + threadIdx.x * (GMAX + 1) : G.tab + G.at(t, 0);
    int *rlab = STAGE ? slab + threadIdx.x * (GMAX + 1) : G.lab + G.at(t, 0);
    const int rs = STAGE ? 1 : 32;                         // entry stride of a row
    if (t < total && t >= G.cap) G.count[t] = -1;
    if (t < total && t < G.cap) {
        const int i = P.cell_list ? P.cell_list[t] : t;
        const int2 p = P.sxy[i];
        CellGrid g = cell_grid(P, i);
        if (!FINE) g.fd = nullptr;                     // sub-buckets unused: no checks compiled in
        const Disc rule = first_disc(g, p, target);
        Disc d = rule;
        if (P.need_in) {
            // A cell the first pass could not certify: its polygon, which only
            // shrinks with more candidates, needs rho^2 >= need.  That disc is
            // taken when it is not much larger than the density-based one, or
            // else tried first when it is at least 16 times larger (in area)
            // and spans at most 64 bucket rows (the hull cells of small
            // clusters: a large disc over mostly empty space), with the
            // density-based disc as the fallback when it overflows the list.
            const float nf = P.need_in[i];
            if (nf > 0.f) {
                const Disc dn = disc_of(g, p, max((i64)nf, (i64)4));
                if (nf <= 1.5f * (float)rule.rho2 || (nf >= 16.f * (float)rule.rho2 && dn.by1 - dn.by0 < 64))
                    d = dn;
            }
        }
        int cnt = 0;
        auto list = [&](const Disc &dd) {
            const i64 rho2 = dd.rho2;
            cnt = 0;
            for (int row = dd.by0; row <= dd.by1 && cnt <= GMAX; row++) {
                int bx0, bx1;
                if (!chord_cols(g, p, rho2, row, bx0, bx1)) continue;
                disc_row_ranges(g, p, rho2, row, bx0, bx1, [&](int a, int b) {
                    // four independent site loads in flight per step
                    for (int pos0 = a; pos0 < b; pos0 += 4) {
                        int2 q[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) q[u] = pos0 + u < b ? __ldg(P.sxy + pos0 + u) : p;
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int pos = pos0 + u;
                            if (pos >= b || pos == i) continue;
                            const int nx = q[u].x - p.x, ny = q[u].y - p.y;
                            if ((i64)nx * nx + (i64)ny * ny > rho2) continue;
                            if (cnt < GMAX) {
                                rtab[cnt * rs] = t1::cand_of(nx, ny);
                                rlab[cnt * rs] = __ldg(P.sid + pos) - g.site_base;
                            }
                            cnt++;
                        }
                    }
                });
            }
        };
        list(d);
        if (cnt > GMAX && d.rho2 > rule.rho2) {          // the need disc overflowed
            d = rule;
            list(d);
        }
        // a crowded disc (the density of the 3 x 3 buckets underestimates a
        // cluster's core): a quarter of the area, up to three times
        for (int shrink = 0; shrink < 3 && cnt > GMAX && d.rho2 > 16; shrink++) {
            d = disc_of(g, p, d.rho2 / 4);
            list(d);
        }
        const i64 rho2 = d.rho2;
        G.count[t] = cnt > GMAX ? -1 : cnt;
        G.rho2[t] = rho2;
    }
    if (!STAGE) return;
    __syncthreads();
    // entry q of the block's rows [t0, t0 + rows) is a contiguous range
    const int rows = min(min(total, G.cap), t0 + NT) - t0;
    if (rows <= 0) return;
    for (int idx = threadIdx.x; idx < rows * GMAX; idx += NT) {
        const int q = idx / rows, rr = idx - q * rows;
        G.tab[G.at(t0 + rr, q)] = stab[rr * (GMAX + 1) + q];
        G.lab[G.at(t0 + rr, q)] = slab[rr * (GMAX + 1) + q];
    }
}

// Strip gather (the first pass, which lists every cell): the NT cells of a
// block are consecutive in sorted order, i.e. mostly neighbours along one
// bucket row, and their discs overlap.  The block takes its cells in
// segments of equal (set, bucket row).  For a segment it loads the bucket
// starts and the sites of the rectangle of buckets that covers the
// segment's discs into shared memory once (asynchronous copies, mostly from
// L2); each thread lists its cell's candidates as indices into that copy,
// then the segment's threads write their rows entry by entry in step, so
// that entry q of the consecutive rows goes out at once (whole sectors;
// rows with fewer entries get padding, which the projector never reads).  A segment whose
// rectangle does not fit the shared arrays (large discs in sparse regions)
// lists from global memory and writes its rows directly, like
// gather_kernel.  The lists and counts are the same as gather_kernel's (the
// same disc, the same chord buckets, the same order).
template <int NT, int GMAX, int SCAP, int BCAP, int RCAP, bool FINE>
__global__ void __launch_bounds__(NT) gather_strip_kernel(CellParams P, GatherOut G, float target) {
    static_assert(SCAP <= 65536, "shared site indices are 16-bit");
    __shared__ int2 s_xy[SCAP];
    __shared__ int s_id[SCAP];
    __shared__ int s_bs[BCAP];
    __shared__ unsigned short s_ent[GMAX * NT];        // entry q of thread r: s_ent[q * NT + r]
    __shared__ int s_roff[RCAP + 1];
    __shared__ long long s_key[NT];
    __shared__ int s_cnt[NT];                           // -1: the row was written directly
    __shared__ int s_box[5];
    if (P.hdr->err) return;
    const int total = min(P.n, G.cap);
    const int t0 = blockIdx.x * NT;
    if (t0 >= total) return;
    const int tid = threadIdx.x;
    const int t = t0 + tid;
    const bool act = t < total;
    const int nact = min(NT, total - t0);
    int2 p = make_int2(0, 0);
    CellGrid g{};
    Disc d{};
    if (act) {
        p = P.sxy[t];
        g = cell_grid(P, t);
        if (!FINE) g.fd = nullptr;                     // sub-buckets unused: no checks compiled in
        d = first_disc(g, p, target);
        // segment key: (set, bucket row); non-decreasing along t
        s_key[tid] = ((long long)(P.sset ? P.sset[t] : 0) << 21) | (p.y / g.s);
    }
    int cnt = 0;
    // a row from global memory, written directly (rows outside the staged
    // rectangle; none by construction of the rectangle)
    auto list_global = [&](int row, int bx0, int bx1) {
        disc_row_ranges(g, p, d.rho2, row, bx0, bx1, [&](int a, int b) {
            for (int pos0 = a; pos0 < b; pos0 += 4) {
                int2 q[4];
#pragma unroll
                for (int u = 0; u < 4; u++) q[u] = pos0 + u < b ? __ldg(P.sxy + pos0 + u) : p;
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int pos = pos0 + u;
                    if (pos >= b || pos == t) continue;
                    const int nx = q[u].x - p.x, ny = q[u].y - p.y;
                    if ((i64)nx * nx + (i64)ny * ny > d.rho2) continue;
                    if (cnt < GMAX) {
                        G.tab[G.at(t, cnt)] = t1::cand_of(nx, ny);
                        G.lab[G.at(t, cnt)] = __ldg(P.sid + pos) - g.site_base;
                    }
                    cnt++;
                }
            }
        });
    };
    __syncthreads();
    for (int lo = 0; lo < nact;) {
        const long long key = s_key[lo];
        const bool mine = act && s_key[tid] == key;
        if (tid == 0) { s_box[0] = INT_MAX; s_box[1] = -1; s_box[2] = INT_MAX; s_box[3] = -1; s_box[4] = 0; }
        __syncthreads();
        if (mine) {
            // every chord's buckets lie in these columns: chord_cols' bounds
            // with the half-width h <= r, the same float operations
            atomicMin(&s_box[0], d.by0);
            atomicMax(&s_box[1], d.by1);
            atomicMin(&s_box[2], max(0, (int)floorf(((float)p.x - (float)d.r) / (float)g.s)));
            atomicMax(&s_box[3], min(g.m1 - 1, (int)floorf(((float)p.x + (float)d.r) / (float)g.s)));
        }
        const int len = __syncthreads_count(mine);     // the segment is threads lo .. lo + len - 1
        const int R0 = s_box[0], R = s_box[1] - R0 + 1, C0 = s_box[2], C1 = s_box[3] - C0 + 2;
        bool staged = R <= RCAP && R * C1 <= BCAP;
        const CellGrid gs = cell_grid(P, t0 + lo);      // the segment's set
        if (staged) {
            for (int k = tid; k < R * C1; k += NT) {
                const int rr = k / C1;
                cp_async4(s_bs + k, gs.bs + (R0 + rr) * gs.m1 + C0 + (k - rr * C1));
            }
            cp_async_wait_all();
        }
        __syncthreads();
        if (staged && tid == 0) {
            int acc = 0;
            for (int rr = 0; rr < R; rr++) {
                s_roff[rr] = acc;
                acc += s_bs[rr * C1 + C1 - 1] - s_bs[rr * C1];
            }
            s_roff[R] = acc;
        }
        __syncthreads();
        staged = staged && s_roff[R] <= SCAP;
        if (staged) {
            // the rectangle's sites: row rr's buckets C0 .. C0 + C1 - 2 hold the
            // sorted positions s_bs[rr * C1] .. s_bs[rr * C1 + C1 - 1] - 1
            for (int rr = 0; rr < R; rr++) {
                const int a = s_bs[rr * C1], nr = s_bs[rr * C1 + C1 - 1] - a, o = s_roff[rr];
                for (int j = tid; j < nr; j += NT) {
                    cp_async8(s_xy + o + j, P.sxy + a + j);
                    cp_async4(s_id + o + j, P.sid + a + j);
                }
            }
            cp_async_wait_all();
        }
        __syncthreads();
        if (mine) {
            bool direct = !staged;
            auto list_staged = [&]() {
                cnt = 0;
                for (int row = d.by0; row <= d.by1 && !direct; row++) {
                    int bx0, bx1;
                    if (!chord_cols(g, p, d.rho2, row, bx0, bx1)) continue;
                    if (bx0 < C0 || bx1 + 1 - C0 >= C1) { direct = true; break; }
                    const int *rb = s_bs + (row - R0) * C1;
                    const int sb = s_roff[row - R0] - rb[0];    // shared index of position pos: pos + sb
                    auto take = [&](int pos, int2 q) {
                        const int nx = q.x - p.x, ny = q.y - p.y;
                        if (pos == t || (i64)nx * nx + (i64)ny * ny > d.rho2) return;
                        if (cnt < GMAX) s_ent[cnt * NT + tid] = (unsigned short)(pos + sb);
                        cnt++;
                    };
                    auto take_range = [&](int a, int b) {
                        int pos = a;
                        for (; pos + 1 < b; pos += 2) {          // two sites per step
                            const int2 q0 = s_xy[pos + sb], q1 = s_xy[pos + 1 + sb];
                            take(pos, q0);
                            take(pos + 1, q1);
                        }
                        if (pos < b) take(pos, s_xy[pos + sb]);
                    };
                    if (!g.fd) take_range(rb[bx0 - C0], rb[bx1 + 1 - C0]);
                    else disc_row_ranges(g, p, d.rho2, row, bx0, bx1, take_range);
                }
            };
            auto list_direct = [&]() {
                cnt = 0;
                for (int row = d.by0; row <= d.by1; row++) {
                    int bx0, bx1;
                    if (chord_cols(g, p, d.rho2, row, bx0, bx1)) list_global(row, bx0, bx1);
                }
            };
            if (!direct) list_staged();
            if (direct) list_direct();
            // a crowded disc (the density of the 3 x 3 buckets underestimates
            // a cluster's core): a quarter of the area, up to three times; the
            // smaller disc lies inside the staged rectangle
            for (int shrink = 0; shrink < 3 && cnt > GMAX && d.rho2 > 16; shrink++) {
                d = disc_of(g, p, d.rho2 / 4);
                if (!direct) list_staged();
                if (direct) list_direct();
            }
            if (direct) {
                s_cnt[tid] = -1;
            } else {
                s_cnt[tid] = cnt;
                atomicMax(&s_box[4], min(cnt, GMAX));
            }
        }
        __syncthreads();
        if (staged && mine && s_cnt[tid] >= 0) {
            // the thread writes its own row, entry by entry in step with the
            // segment's other threads: entry q of consecutive rows is one
            // contiguous range of each list
            const int M = s_box[4];
            for (int q = 0; q < M; q++) {
                float2 v = make_float2(0.f, 0.f);
                int lab = -1;
                if (q < cnt) {
                    const int e = s_ent[q * NT + tid];
                    const int2 a = s_xy[e];
                    v = t1::cand_of(a.x - p.x, a.y - p.y);
                    lab = s_id[e] - g.site_base;
                }
                G.tab[G.at(t, q)] = v;
                G.lab[G.at(t, q)] = lab;
            }
        }
        __syncthreads();                                 // the shared arrays are reused
        lo += len;
    }
    if (act) {
        G.count[t] = cnt > GMAX ? -1 : cnt;
        G.rho2[t] = d.rho2;
    }
}

template <int NT, int CMAX, int SMAX, int EMAX, int RMAX>
__global__ void __launch_bounds__(NT) cells_persist_kernel(CellParams P, GatherOut G) {
    extern __shared__ __align__(16) float2 tbl_raw[];
    if (P.hdr->err) return;
    const t1::Table<NT> T{tbl_raw + threadIdx.x};
    const unsigned FULL = 0xffffffffu;
    static_assert(EMAX <= 16, "edge labels are packed into two 64-bit registers");
    // Per-thread state lives in registers.  The edge list (candidate indices,
    // one byte each) is packed into em0/em1.  The subedge stack keeps its top
    // four entries in registers (s0 = the top) and only deeper entries in the
    // local arrays, which few cells reach.
    unsigned long long em0 = 0, em1 = 0;
    auto emit_get = [&](int q) -> int {
        return (int)(((q < 8 ? em0 : em1) >> ((q & 7) * 8)) & 0xff);
    };
    auto emit_put = [&](int q, int lab) {
        const unsigned long long v = (unsigned long long)lab << ((q & 7) * 8);
        if (q < 8) em0 |= v; else em1 |= v;
    };
    i64 s0x = 0, s0y = 0, s1x = 0, s1y = 0, s2x = 0, s2y = 0, s3x = 0, s3y = 0;
    int s0l = 0, s1l = 0, s2l = 0, s3l = 0;           // clockwise line | counter-clockwise << 8
    long long dsx[SMAX], dsy[SMAX];
    int dsl[SMAX];
    int sp = 0;
    auto push = [&](i64 x, i64 y, int cw, int ccw) {
        if (sp >= 4) { dsx[sp - 4] = s3x; dsy[sp - 4] = s3y; dsl[sp - 4] = s3l; }
        s3x = s2x; s3y = s2y; s3l = s2l;
        s2x = s1x; s2y = s1y; s2l = s1l;
        s1x = s0x; s1y = s0y; s1l = s0l;
        s0x = x; s0y = y; s0l = cw | (ccw << 8);
        sp++;
    };
    auto pop = [&]() {
        s0x = s1x; s0y = s1y; s0l = s1l;
        s1x = s2x; s1y = s2y; s1l = s2l;
        s2x = s3x; s2y = s3y; s2l = s3l;
        if (sp > 4) { s3x = dsx[sp - 5]; s3y = dsy[sp - 5]; s3l = dsl[sp - 5]; }
        sp--;
    };
    t1::Counters cnt{};
    const int stride = gridDim.x * NT;
    int t = blockIdx.x * NT + threadIdx.x;
    const int total = P.cell_list ? *P.list_count : P.n;

    // state of the thread's current cell
    int i = -1, C = 0, ctt = 0;      // ctt: the cell's entry in the gather lists
    int kcell = 0;                   // the cell's index in the batch
    int2 p = make_int2(0, 0);
    int cW = 0, cH = 0, cbase = 0;   // the cell's box and the first site of its set
    i64 rho2 = 0;
    float sbf = 0.f;                 // (1 + 2^-18) / (2 dmin), dmin = p's distance to the box
    int phase = 0, h0c = -1, h0w = -1, h1c = -1, h1w = -1;
    i64 lx = 0, ly = 0;
    int llab = -1, ne = 0, rays = 3, first = -1, last = -1;
    bool have = false;     // a cell is loaded and its projector runs
    bool fin = false;      // the projector finished: certificate and output pending
    bool ok = true;        // the projector stayed within the capacities
    bool retired = false;  // no cells left for this thread

    for (;;) {
        // ---- batched finalise + load ------------------------------------------
        const bool idle = !have && !retired;
        const unsigned idlem = __ballot_sync(FULL, idle);
        const unsigned busym = __ballot_sync(FULL, have);
        if (idlem != 0 && (__popc(idlem) >= P_REFILL || busym == 0)) {
            if (idle) {
                if (fin) {
                    fin = false;
                    bool defer = !ok;
                    int e = ne;
                    float needf = 0.f;           // the squared radius a deferred polygon needs
                    if (!defer) {
                        if (e > 1 && last == first) e--;           // the walk closes
                        if (e < 3) defer = true;
                    }
                    // the edges' labels, loaded first so that their latency
                    // overlaps the certificate below (independent loads)
                    int lq[EMAX];
                    {
                        const int *__restrict__ gl = G.lab + G.at(ctt, 0);
#pragma unroll
                        for (int q = 0; q < EMAX; q++) {
                            const int c = q < e ? emit_get(q) : 0;
                            lq[q] = (!defer && c >= 4) ? __ldg(gl + (c - 4) * 32) : -1 - c;
                        }
                    }
                    if (!defer) {
                        // security-radius certificate: 2R <= rho
                        float R2 = 0.f;
                        for (int q = 0; q < e; q++) {
                            int n1x, n1y, n2x, n2y;
                            i64 c1, c2, Nx, Ny, D;
                            T.line(emit_get(q), n1x, n1y, c1);
                            T.line(emit_get(q + 1 < e ? q + 1 : 0), n2x, n2y, c2);
                            intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
                            if (D == 0) { defer = true; break; }
                            const float rd = t1::rcp_approx((float)D);
                            const float vx = (float)Nx * rd, vy = (float)Ny * rd;
                            R2 = fmaxf(R2, fmaf(vx, vx, vy * vy));
                        }
                        const i64 cxf = max(p.x, cW - p.x), cyf = max(p.y, cH - p.y);
                        const i64 need = (i64)(4.f * (R2 * (1.f + 0x1p-12f) + 1.f)) + 1;
                        if (!(need <= rho2 || rho2 >= cxf * cxf + cyf * cyf)) {
                            defer = true;
                            needf = __ll2float_ru(need);
                        }
                    }
                    if (!defer) {
                        // canonical order: start at the smallest normal angle
                        int start = 0, bxn, byn, qx, qy;
                        i64 dummy;
                        T.line(emit_get(0), bxn, byn, dummy);
                        for (int q = 1; q < e; q++) {
                            T.line(emit_get(q), qx, qy, dummy);
                            if (angle_less(qx, qy, bxn, byn)) { start = q; bxn = qx; byn = qy; }
                        }
                        const int k = kcell;
                        const int kl = k - cbase;
                        int *dst;
                        int off = -1;
                        if (e <= SLOT_CAP) {
                            dst = P.slot + (size_t)k * SLOT_CAP;
                        } else {
                            off = atomicAdd(&P.hdr->spill_top, e);
                            if (off + e > P.spill_cap) defer = true;
                            dst = P.spill + off;
                        }
                        if (!defer) {
                            // edge q goes to position (q - start) mod e
                            int dcnt = 0;
#pragma unroll
                            for (int q = 0; q < EMAX; q++) {
                                if (q < e) {
                                    const int at = q >= start ? q - start : q - start + e;
                                    dst[at] = lq[q];
                                    dcnt += lq[q] > kl ? 1 : 0;
                                }
                            }
                            P.ecount[k] = e;
                            P.dcount[k] = dcnt;
                            P.loc[k] = off;
                            if ((unsigned long long)e > cnt.maxe) cnt.maxe = e;
                        }
                    }
                    if (defer) {
                        if (P.deferred) {
                            const int q = atomicAdd(P.deferred_count, 1);
                            P.deferred[q] = i;
                            if (P.need_out) P.need_out[i] = needf;
                            if (P.store_poly) {
                                // a polygon the certificate could not accept:
                                // its lines (counter-clockwise) go to the
                                // cell's slot for the next pass's flower list
                                // (a later polygon replaces an earlier one; a
                                // first pass without one clears the mark)
                                const int k = kcell;
                                if (needf > 0.f) {
                                    int *dst = P.slot + (size_t)k * SLOT_CAP;
#pragma unroll
                                    for (int q2 = 0; q2 < EMAX; q2++)
                                        if (q2 < e) dst[q2] = lq[q2];
                                    P.ecount[k] = -e;
                                } else if (P.need_out) {
                                    P.ecount[k] = 0;
                                }
                            }
                            cnt.deferred++;
                        } else {
                            atomicOr(&P.hdr->err, ERRB_CAPACITY);
                        }
                    }
                }
                // load the next cell: with a dynamic schedule the idle lanes take
                // consecutive entries with one atomic (the warp's generation),
                // else the thread's own sequence t, t + stride, ...
                if (P.next_cell) {
                    const int lane = threadIdx.x & 31, leader = __ffs(idlem) - 1;
                    int base = 0;
                    if (lane == leader) base = atomicAdd(P.next_cell, __popc(idlem));
                    base = __shfl_sync(idlem, base, leader);
                    t = base + __popc(idlem & ((1u << lane) - 1));
                }
                while (t < total) {
                    const int tt = t;
                    i = P.cell_list ? P.cell_list[t] : t;
                    t += stride;
                    // the whole list row, copied while the count is still on
                    // its way (entries past the count are never read)
                    if (tt < G.cap) {
                        const float2 *src = G.tab + G.at(tt, 0);
#pragma unroll 8
                        for (int q = 0; q < CMAX - 4; q++)
                            cp_async8(&tbl_raw[(4 + q) * NT + threadIdx.x], src + q * 32);
                    }
                    const int nc = G.count[tt];
                    if (nc < 0) {                                   // disc too crowded
                        cp_async_wait_all();      // the table is reused by the next cell
                        if (P.deferred) {
                            const int q = atomicAdd(P.deferred_count, 1);
                            P.deferred[q] = i;
                            if (P.need_out) {
                                P.need_out[i] = 0.f;
                                P.ecount[__ldg(P.sid + i)] = 0;       // no polygon
                            }
                            cnt.deferred++;
                        } else {
                            atomicOr(&P.hdr->err, ERRB_CAPACITY);
                        }
                        if (P.next_cell) t = atomicAdd(P.next_cell, 1);
                        continue;
                    }
                    p = P.sxy[i];
                    kcell = __ldg(P.sid + i);
                    rho2 = G.rho2[tt];
                    {
                        const SetMeta &M = set_of(P.sets, P.sset, i);
                        cW = M.W;
                        cH = M.H;
                        cbase = (int)M.site_base;
                    }
                    sbf = (1.f + 0x1p-18f) / (2.f * (float)min(min(p.x, p.y), min(cW - p.x, cH - p.y)));
                    T.put(0, t1::cand_of(0, -p.y));
                    T.put(1, t1::cand_of(cW - p.x, 0));
                    T.put(2, t1::cand_of(0, cH - p.y));
                    T.put(3, t1::cand_of(-p.x, 0));
                    cp_async_wait_all();
                    ctt = tt;
                    C = nc + 4;
                    cnt.cands += C;
                    phase = 0; sp = 0; ne = 0; rays = 3; first = -1; last = -1; llab = -1;
                    em0 = em1 = 0;
                    ok = true;
                    have = true;
                    break;
                }
                if (!have) retired = true;
            }
        }
        if (__ballot_sync(FULL, !retired) == 0) break;

        // ---- choose the next ray of this thread's cell -------------------------
        bool query = false, utest = false;
        i64 tx = 0, ty = 0, Nx = 0, Ny = 0, D = 0;
        int la = -1, lb = -1;
        if (have) {
            if (phase < 3) {
                tx = phase == 0 ? 2 : (phase == 1 ? 0 : -2);
                ty = phase == 1 ? 1 : -1;
                query = true;
            } else {
                while (sp > 0) {
                    const i64 rx = s0x, ry = s0y;
                    const int rcw = s0l & 0xff;
                    if (llab == rcw) {                           // same line: no vertex
                        if (llab != last) {
                            if (ne >= EMAX) { ok = false; sp = 0; break; }
                            emit_put(ne++, llab);
                            if (first < 0) first = llab;
                            last = llab;
                        }
                        lx = rx; ly = ry; llab = s0l >> 8;
                        pop();
                        continue;
                    }
                    int n1x, n1y, n2x, n2y;
                    i64 c1, c2;
                    T.line(llab, n1x, n1y, c1);
                    T.line(rcw, n2x, n2y, c2);
                    intersect(n1x, n1y, c1, n2x, n2y, c2, Nx, Ny, D);
                    la = llab;
                    lb = rcw;
                    if (D == 0) {                                // parallel lines
                        tx = -(i64)n1y;
                        ty = (i64)n1x;
                        if (!(cross128(lx, ly, tx, ty) >= 0 && cross128(tx, ty, rx, ry) >= 0)) {
                            tx = -tx;
                            ty = -ty;
                        }
                        la = lb = -1;
                    } else {
                        const int sg = D > 0 ? 1 : -1;
                        const bool inw = sg * t1::cross_sign(lx, ly, Nx, Ny) >= 0 &&
                                         sg * t1::cross_sign(Nx, Ny, rx, ry) >= 0;
                        tx = sg * Nx;
                        ty = sg * Ny;
                        if (inw) {
                            utest = true;                        // the ray towards u
                        } else {
                            tx = -tx;                            // theta_3 := p - u
                            ty = -ty;
                            la = lb = -1;
                        }
                    }
                    query = true;
                    break;
                }
                if (!query) { have = false; fin = true; }       // EdgeQueue is empty
            }
        }

        // ---- the filter pass (converged across the warp) ------------------------
        const int Cq = query ? C : 0;
        const float fx = (float)tx, fy = (float)ty;
        const float eth = fmaxf(fabsf(fx), fabsf(fy)) * 0x1p-19f;
        // A ray towards u (the vertex of lines la and lb) leaves those two lines
        // out: their entries read (0, 0) during the pass, which makes both of
        // their bounds NaN (1/0 times 0), and a NaN neither wins a comparison
        // nor raises a maximum.  The best remaining upper bound is then the
        // bound ux of the vertex test.
        float2 ea = make_float2(0.f, 0.f), eb = ea;
        if (utest) {
            ea = T.get(la);
            eb = T.get(lb);
            T.put(la, make_float2(0.f, 0.f));
            T.put(lb, make_float2(0.f, 0.f));
        }
        // the sites (two streams of candidates)
        float u1a = -FLT_MAX, u2a = -FLT_MAX, lsa = -FLT_MAX;
        float u1b = -FLT_MAX, u2b = -FLT_MAX, lsb = -FLT_MAX;
        int i1a = -1, i1b = -1;
        int c = 4;
        // unrolled twice: the next pair's loads and keys overlap this pair's
        // comparisons (measured: 0.857 -> 0.842 ms; four streams instead of
        // two cost registers and ran at 1.04 ms)
#pragma unroll 2
        for (; c + 1 < Cq; c += 2) {
            float Ua, La, Ub, Lb;
            t1::filter_keys(T.get(c), false, fx, fy, eth, Ua, La);
            t1::filter_keys(T.get(c + 1), false, fx, fy, eth, Ub, Lb);
            if (Ua > u1a) { u2a = u1a; u1a = Ua; i1a = c; lsa = La; } else u2a = fmaxf(u2a, Ua);
            if (Ub > u1b) { u2b = u1b; u1b = Ub; i1b = c + 1; lsb = Lb; } else u2b = fmaxf(u2b, Ub);
        }
        if (c < Cq) {
            float Ua, La;
            t1::filter_keys(T.get(c), false, fx, fy, eth, Ua, La);
            if (Ua > u1a) { u2a = u1a; u1a = Ua; i1a = c; lsa = La; } else u2a = fmaxf(u2a, Ua);
        }
        if (!query) continue;
        float u1, u2, ls;
        int i1;
        if (u1b > u1a || (u1b == u1a && i1b >= 0 && i1b < i1a)) {
            i1 = i1b; u1 = u1b; ls = lsb; u2 = fmaxf(fmaxf(u2a, u2b), u1a);
        } else {
            i1 = i1a; u1 = u1a; ls = lsa; u2 = fmaxf(fmaxf(u2a, u2b), u1b);
        }
        // The four sides of X, only when one of them could reach the best
        // site: the key of a side at distance d from p is +-t/(2d) for a
        // component t of theta, at most max(|tx|,|ty|) / (2 dmin) <= sb
        // (sbf carries a relative margin of 2^-18 over the float roundings).
        // Otherwise sb stands in for their upper bounds.
        const float sb = fmaxf(fabsf(fx), fabsf(fy)) * sbf;
        if (!(sb < ls)) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                float U, L;
                t1::filter_keys(T.get(q), true, fx, fy, eth, U, L);
                if (U > u1) { u2 = u1; u1 = U; i1 = q; ls = L; } else u2 = fmaxf(u2, U);
            }
        } else {
            u2 = fmaxf(u2, sb);
            u1 = fmaxf(u1, sb);
        }
        const float ux = u1;
        if (utest) {
            T.put(la, ea);
            T.put(lb, eb);
        }
        cnt.evals += C;

        // ---- decide ----------------------------------------------------------
        int hc = -1, hw = -1;
        bool inside = false;
        if (utest) {
            cnt.vtests++;
            const i64 aD = D > 0 ? D : -D;
            const float kuf = (float)(aD / 2);             // key of u: |D|/2, an integer
            const float klo = kuf * (1.f - 0x1p-21f), khi = kuf * (1.f + 0x1p-21f);
            if (!P.exact_only && ux < klo) {
                inside = true;
            } else if (!P.exact_only && ls > u2 && ls > khi && i1 != la && i1 != lb) {
                hc = hw = i1;
            } else {
                cnt.exact++;
                bool viol = false;
                for (int q = 0; q < C && !viol; q++) {
                    if (q == la || q == lb) continue;
                    if (!P.exact_only) {
                        float Ug, Lg;
                        t1::filter_keys(T.get(q), q < 4, fx, fy, eth, Ug, Lg);
                        if (Ug < klo) continue;
                    }
                    int nx, ny;
                    i64 cc;
                    T.line(q, nx, ny, cc);
                    const i128 lhs = 2 * dot128(nx, ny, Nx, Ny) * (i128)(D > 0 ? 1 : -1);
                    if (lhs > (i128)cc * aD) viol = true;
                }
                if (!viol) inside = true;
                else t1::exact_argmax(T, C, tx, ty, fx, fy, eth, !P.exact_only, ls, hc, hw);
            }
        } else {
            cnt.rays++;
            if (!P.exact_only && ls > u2 && ls > 0.f) {
                hc = hw = i1;
            } else {
                cnt.exact++;
                t1::exact_argmax(T, C, tx, ty, fx, fy, eth, !P.exact_only, ls, hc, hw);
            }
        }

        // ---- update the subedge state ------------------------------------------
        if (phase < 3) {
            if (hc < 0) { ok = false; have = false; fin = true; continue; }
            if (phase == 0) { h0c = hc; h0w = hw; }
            else if (phase == 1) { h1c = hc; h1w = hw; }
            else {
                lx = 2; ly = -1; llab = h0c;
                sp = 0;
                push(2, -1, h0w, h0c);
                push(-2, -1, hw, hc);
                push(0, 1, h1w, h1c);
            }
            phase++;
        } else if (inside) {                               // u is a vertex: L1, L2 are edges
            if (la != last) {
                if (ne >= EMAX) { ok = false; have = false; fin = true; continue; }
                emit_put(ne++, la);
                if (first < 0) first = la;
                last = la;
            }
            if (lb != last) {
                if (ne >= EMAX) { ok = false; have = false; fin = true; continue; }
                emit_put(ne++, lb);
                if (first < 0) first = lb;
                last = lb;
            }
            lx = s0x; ly = s0y; llab = s0l >> 8;
            pop();
        } else {                                           // divide the subedge at theta_3
            if (sp >= SMAX || ++rays > RMAX || hc < 0) { ok = false; have = false; fin = true; continue; }
            push(tx, ty, hw, hc);
        }
    }
    if (P.collect_stats) {
        unsigned long long v[10] = {cnt.rays, cnt.vtests, cnt.evals, cnt.exact, cnt.annulus,
                                    cnt.reruns, cnt.deferred, cnt.cands, cnt.widen, cnt.maxe};
#pragma unroll
        for (int q = 0; q < 10; q++) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(FULL, v[q], off);
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
            if (!P.cell_list) {                 // first pass: its own share of the work
                atomicAdd(&st[STAT_EVALS1], v[2]);
                atomicAdd(&st[STAT_RAYS1], v[0]);
            } else {
                atomicAdd(&st[STAT_EVALS2], v[2]);
            }
        }
    }
}

}  // namespace vor
