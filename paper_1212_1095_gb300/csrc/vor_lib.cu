// vor_lib.cu -- planning, bucketing, scans, compaction and the C ABI of libvor.so.
//
// A build runs a batch of independent point sets (a single diagram is a
// batch of one set).  Pipeline (all on one stream, no host synchronisation):
//   K0  plan           per set: box, sizes of its grids, offsets (one block)
//       site_set       per site: its set (batches only)
//   K1  probe          per set: site counts on a coarse occupancy grid and
//                      the density a typical site sees
//       coarse_sat     the coarse grid's summed-area table
//       pick_grid      per set: bucket side s (Method A.5) and bucket offsets
//       bucket_count   validate sites (interior of X, Section 2), count sites
//                      per bucket, record each site's rank inside its bucket
//       scan           bucket counts -> bucket start offsets
//       fine_*         optional sub-buckets of the dense buckets
//       bucket_scatter sites sorted by set, then bucket (and sub-bucket),
//                      with their index
//       dup_check      equal sites share a bucket: compare within buckets
//   K2  cells          the projector per cell (vor_cells*.cu): two
//                      thread-per-cell passes, flower passes (batches), the
//                      warp tier and the block tier over the cells each
//                      earlier stage deferred
//       scan x2        e_k -> cell_ptr, Delaunay counts -> offsets
//   K3  compact        CSR edge labels, float64 vertices (Section 5) and the
//                      Delaunay pairs (Section 6), labels local to the set
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <cuda_runtime.h>

#include "vor.h"
#include "vor_device.cuh"
#include "vor_internal.h"

namespace vor {

// ---------------------------------------------------------------------------
// K0: per-set plan (a single build is a batch of one set)
// ---------------------------------------------------------------------------

// One block of SCAN_T threads: per set, its sites, box and grid sizes
// (plan_set, the same function that sized the workspace on the host) and the
// offsets of its density-probe grid.  The device copy of the set offsets is
// checked against what the host planned with (hn_total, hm_sum, hg_sum): a
// mismatch stops the build before any kernel indexes with it.
__global__ void k_plan(const long long *__restrict__ set_ptr, const vor_box *__restrict__ boxes,
                       int n_sets, long long n1, vor_box box1, int s_fixed, int load_pct,
                       long long hn_total, long long hm_sum, long long hg_sum,
                       SetMeta *__restrict__ sets, WsHeader *hdr);

// per site: the set it belongs to (binary search in the set offsets)
__global__ void k_site_set(const long long *__restrict__ set_ptr, int n_sets, int n,
                           int *__restrict__ sset, const WsHeader *hdr) {
    if (hdr->err) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = n_sets;             // invariant: set_ptr[lo] <= i < set_ptr[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (set_ptr[mid] <= i) lo = mid;
        else hi = mid;
    }
    sset[i] = lo;
}

// ---------------------------------------------------------------------------
// K1: bucketing
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool outside(int2 p, const SetMeta &M) {
    return p.x <= 0 || p.x >= M.W || p.y <= 0 || p.y >= M.H;
}

__device__ __forceinline__ long long bucket_of(int2 p, const SetMeta &M) {
    return M.bucket_base + (long long)(p.y / M.s) * M.m1 + p.x / M.s;
}

// Site density probe: the bucket side is chosen so that a bucket around a
// typical site holds about two sites.  A coarse G x G grid per set counts
// the sites; the typical neighbourhood count is the geometric mean, over the
// set's sites, of the count of their own coarse cell.
__global__ void k_probe_count(const int2 *__restrict__ sites, int n, const SetMeta *__restrict__ sets,
                              const int *__restrict__ sset, int *__restrict__ coarse,
                              const WsHeader *hdr) {
    if (hdr->err) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SetMeta &M = set_of(sets, sset, i);
    const int2 p = sites[i];
    if (outside(p, M)) return;                              // reported by k_bucket_count
    // 0 <= p < W <= 2^20 and G <= 1024: the products fit 32 bits
    const int cx = (int)((unsigned)p.x * (unsigned)M.G / (unsigned)M.W);
    const int cy = (int)((unsigned)p.y * (unsigned)M.G / (unsigned)M.H);
    atomicAdd(&coarse[M.coarse_base + (long long)cy * M.G + cx], 1);
}

__global__ void k_probe_mean(const int2 *__restrict__ sites, int n, SetMeta *__restrict__ sets,
                             const int *__restrict__ sset, const int *__restrict__ coarse,
                             const WsHeader *hdr) {
    __shared__ float sh[8];
    if (hdr->err) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j0 = sset ? sset[blockIdx.x * blockDim.x] : 0;
    int j = j0;
    float v = 0.f;
    if (i < n) {
        j = sset ? sset[i] : 0;
        const SetMeta &M = sets[j];
        const int2 p = sites[i];
        if (!outside(p, M)) {
            const int cx = (int)((unsigned)p.x * (unsigned)M.G / (unsigned)M.W);
            const int cy = (int)((unsigned)p.y * (unsigned)M.G / (unsigned)M.H);
            v = log2f((float)max(coarse[M.coarse_base + (long long)cy * M.G + cx], 1));
        }
    }
    // blocks inside one set reduce first; blocks across a set boundary add per site
    if (!__syncthreads_and(j == j0)) {
        if (v != 0.f) atomicAdd(&sets[j].acc, (double)v);
        return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
        atomicAdd(&sets[j0].acc, (double)t);
    }
}

// Summed-area table of each set's coarse occupancy grid, in place: entry
// (cy, cx) becomes the number of the set's sites in coarse cells (0..cx) x
// (0..cy).  Rows by warp scans (four rows per warp at a time, for loads in
// flight), then columns with a running sum per thread, eight rows loaded
// ahead.  16 <= G <= 1024.
constexpr int SAT_T = 1024;
__global__ void __launch_bounds__(SAT_T) k_coarse_sat(const SetMeta *__restrict__ sets, int n_sets,
                                                      int *__restrict__ coarse, const WsHeader *hdr) {
    if (hdr->err) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = blockIdx.x; j < n_sets; j += gridDim.x) {
        const int G = sets[j].G;
        int *c = coarse + sets[j].coarse_base;
        for (int r0 = 4 * w; r0 < G; r0 += 4 * nw) {
            int carry[4] = {0, 0, 0, 0};
            for (int x0 = 0; x0 < G; x0 += 32) {
                const int x = x0 + lane;
                int v[4];
#pragma unroll
                for (int u = 0; u < 4; u++) v[u] = (r0 + u < G && x < G) ? c[(r0 + u) * G + x] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int y = __shfl_up_sync(0xffffffffu, v[u], o);
                        if (lane >= o) v[u] += y;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (r0 + u < G && x < G) c[(r0 + u) * G + x] = carry[u] + v[u];
                    carry[u] += __shfl_sync(0xffffffffu, v[u], 31);
                }
            }
        }
        __syncthreads();
        for (int x = threadIdx.x; x < G; x += blockDim.x) {
            int run = 0;
            for (int r0 = 0; r0 < G; r0 += 8) {
                int v[8];
#pragma unroll
                for (int u = 0; u < 8; u++) v[u] = r0 + u < G ? c[(r0 + u) * G + x] : 0;
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    run += v[u];
                    if (r0 + u < G) c[(r0 + u) * G + x] = run;
                }
            }
        }
        __syncthreads();
    }
}

// One block of SCAN_T threads: per set, the bucket side (from the probe, or
// fixed), its grid, and the offset of its buckets in the batch's bucket array.
__global__ void k_pick_grid(SetMeta *__restrict__ sets, int n_sets, int s_fixed, WsHeader *hdr);

__global__ void k_bucket_count(const int2 *__restrict__ sites, int n, const SetMeta *__restrict__ sets,
                               const int *__restrict__ sset, int *__restrict__ bcount,
                               int *__restrict__ rank, WsHeader *hdr) {
    if (hdr->err) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SetMeta &M = set_of(sets, sset, i);
    const int2 p = sites[i];
    if (outside(p, M)) {
        atomicOr(&hdr->err, ERRB_OUTSIDE);
        rank[i] = -1;
        return;
    }
    rank[i] = atomicAdd(&bcount[bucket_of(p, M)], 1);
}

// Adaptive buckets, the second level (Section 9, fourth closing remark: a
// bucketing structure fitted to the distribution of the sites).  A bucket
// whose count reaches `split` gets F x F sub-buckets (fine_log2) and F^2 + 1
// zeroed entries of the pool for their counts, later their starts.
__global__ void k_fine_plan(const int *__restrict__ bstart, int m_max, int split, int *__restrict__ fdesc,
                            int *__restrict__ fpool, long long pool_cap, WsHeader *hdr) {
    if (hdr->err) return;
    const int m = min(m_max, hdr->m_total);
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < m; b += gridDim.x * blockDim.x) {
        const int c = bstart[b + 1] - bstart[b];
        int off = -1;
        if (c >= split) {
            const int F = 1 << fine_log2(c);
            const int need = F * F + 1;
            off = atomicAdd(&hdr->fine_top, need);
            if ((long long)off + need > pool_cap) {
                off = -1;                                  // no room: the bucket stays whole
            } else {
                for (int q = 0; q < need; q++) fpool[off + q] = 0;
                atomicAdd(&hdr->fine_count, 1);
            }
        }
        fdesc[b] = off;
    }
}

// sub-bucket of site p in bucket (bx, by) of side s divided F x F
__device__ __forceinline__ int fine_sub(int2 p, const SetMeta &M, int F) {
    const int lx = p.x - (p.x / M.s) * M.s, ly = p.y - (p.y / M.s) * M.s;
    return (ly * F / M.s) * F + lx * F / M.s;          // lx, ly < s <= 2^20, F <= 16: no overflow
}

// The rank of a site of a divided bucket within its sub-bucket.
__global__ void k_fine_rank(const int2 *__restrict__ sites, int n, const SetMeta *__restrict__ sets,
                            const int *__restrict__ sset, const int *__restrict__ bstart,
                            const int *__restrict__ fdesc, int *__restrict__ fpool,
                            int *__restrict__ rank, const WsHeader *hdr) {
    if (hdr->err) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SetMeta &M = set_of(sets, sset, i);
    const int2 p = sites[i];
    const long long b = bucket_of(p, M);
    const int off = fdesc[b];
    if (off < 0) return;
    const int F = 1 << fine_log2(bstart[b + 1] - bstart[b]);
    rank[i] = atomicAdd(&fpool[off + fine_sub(p, M, F)], 1);
}

// Sub-bucket counts -> starts relative to the bucket's first position.
__global__ void k_fine_scan(const int *__restrict__ bstart, int m_max, const int *__restrict__ fdesc,
                            int *__restrict__ fpool, const WsHeader *hdr) {
    if (hdr->err) return;
    const int m = min(m_max, hdr->m_total);
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < m; b += gridDim.x * blockDim.x) {
        const int off = fdesc[b];
        if (off < 0) continue;
        const int c = bstart[b + 1] - bstart[b];
        const int F2 = 1 << (2 * fine_log2(c));
        int run = 0;
        for (int q = 0; q < F2; q++) {
            const int v = fpool[off + q];
            fpool[off + q] = run;
            run += v;
        }
        fpool[off + F2] = run;                             // = c
    }
}

// Sites sorted by set, then bucket (row-major inside the set's grid), then,
// in a divided bucket, sub-bucket: the sets' bucket ranges follow each
// other, so set j occupies the sorted positions [site_base_j, site_base_j +
// n_j) like the original order.
__global__ void k_bucket_scatter(const int2 *__restrict__ sites, int n, const SetMeta *__restrict__ sets,
                                 const int *__restrict__ sset, const int *__restrict__ bstart,
                                 const int *__restrict__ rank, const int *__restrict__ fdesc,
                                 const int *__restrict__ fpool, int2 *__restrict__ sxy,
                                 int *__restrict__ sid, const WsHeader *hdr) {
    if (hdr->err) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SetMeta &M = set_of(sets, sset, i);
    const int2 p = sites[i];
    const long long b = bucket_of(p, M);
    int pos = bstart[b] + rank[i];
    if (fdesc) {
        const int off = fdesc[b];
        if (off >= 0) pos += fpool[off + fine_sub(p, M, 1 << fine_log2(bstart[b + 1] - bstart[b]))];
    }
    sxy[pos] = p;
    sid[pos] = i;
}

// Distinct sites (Section 2): equal sites of a set fall into the same
// bucket, so a comparison inside each bucket finds every duplicate.
__global__ void k_dup_check(const int2 *__restrict__ sxy, int n, const SetMeta *__restrict__ sets,
                            const int *__restrict__ sset, const int *__restrict__ bstart,
                            WsHeader *hdr) {
    if (hdr->err) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SetMeta &M = set_of(sets, sset, i);
    const int2 p = sxy[i];
    const long long b = bucket_of(p, M);
    const int a = bstart[b], e = bstart[b + 1];
    for (int j = a; j < e; j++) {
        if (j == i) continue;
        const int2 q = sxy[j];
        if (q.x == p.x && q.y == p.y) { atomicOr(&hdr->err, ERRB_DUPLICATE); return; }
    }
}

// ---------------------------------------------------------------------------
// exclusive scan: block totals, then a downsweep; the downsweep sums the
// preceding block totals itself when there are few blocks (quadratic in
// the block count, but one launch less), else a one-block scan of the
// totals runs in between
// ---------------------------------------------------------------------------

constexpr int SCAN_T = 256, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;

template <class T>
__device__ T block_exclusive(T v, T *sh, T &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = lane < SCAN_T / 32 ? sh[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SCAN_T / 32) sh[lane] = t;
    }
    __syncthreads();
    total = sh[SCAN_T / 32 - 1];
    const T before = w > 0 ? sh[w - 1] : T(0);
    __syncthreads();
    return before + x - v;
}

template <class T>
__global__ void k_scan_reduce(const int *__restrict__ in, int n, const int *n_dev,
                              T *__restrict__ partial, const WsHeader *hdr) {
    __shared__ T sh[32];
    if (hdr->err) return;
    if (n_dev) n = min(n, *n_dev);
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_I;
    T s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_I; q++) s += (base + q < n) ? (T)in[base + q] : T(0);
    T total;
    block_exclusive<T>(s, sh, total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

template <class T>
__global__ void k_scan_partials(T *__restrict__ partial, int nb, const WsHeader *hdr) {
    __shared__ T sh[32];
    if (hdr->err) return;
    T carry = 0;
    for (int c0 = 0; c0 < nb; c0 += SCAN_T) {
        const int i = c0 + threadIdx.x;
        const T v = i < nb ? partial[i] : T(0);
        T total;
        const T ex = block_exclusive<T>(v, sh, total);
        if (i < nb) partial[i] = carry + ex;
        carry += total;
    }
}

constexpr int SCAN_SELF_MAX = 4096;      // block counts up to which the downsweep sums the totals

// out[i] = sum of in[0..i) for i < n, and out[n] = total; optionally *tot = total.
// partial: with self_carry the blocks' totals, else their exclusive prefix.
template <class T>
__global__ void k_scan_down(const int *__restrict__ in, int n, const int *n_dev,
                            const T *__restrict__ partial, T *__restrict__ out, long long *tot,
                            bool self_carry, const WsHeader *hdr) {
    __shared__ T sh[32];
    if (hdr->err) return;
    if (n_dev) n = min(n, *n_dev);
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_I;
    T v[SCAN_I];
    T s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_I; q++) {
        v[q] = (base + q < n) ? (T)in[base + q] : T(0);
        s += v[q];
    }
    T carry;
    if (self_carry) {
        // the totals of the blocks before this one (fewer than SCAN_SELF_MAX)
        T before = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += SCAN_T) before += partial[b];
        block_exclusive<T>(before, sh, carry);
    } else {
        carry = partial[blockIdx.x];
    }
    T total;
    T run = carry + block_exclusive<T>(s, sh, total);
#pragma unroll
    for (int q = 0; q < SCAN_I; q++) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        const T t = carry + total;
        out[n] = t;
        if (tot) *tot = (long long)t;
    }
}

// Exclusive scan of in[0..n) (n = min(n_max, *n_dev) when n_dev is given).
// Returns the number of kernels launched.
template <class T>
static int scan(const int *in, int n_max, const int *n_dev, T *out, T *partial, long long *tot,
                WsHeader *hdr, cudaStream_t st) {
    const int nb = (n_max + SCAN_TILE - 1) / SCAN_TILE;
    const int nbb = nb > 0 ? nb : 1;
    const bool self_carry = nbb <= SCAN_SELF_MAX;
    k_scan_reduce<T><<<nbb, SCAN_T, 0, st>>>(in, n_max, n_dev, partial, hdr);
    if (!self_carry) k_scan_partials<T><<<1, SCAN_T, 0, st>>>(partial, nbb, hdr);
    k_scan_down<T><<<nbb, SCAN_T, 0, st>>>(in, n_max, n_dev, partial, out, tot, self_carry, hdr);
    return self_carry ? 2 : 3;
}

// ---------------------------------------------------------------------------
// K0/K1 planning kernels (single block)
// ---------------------------------------------------------------------------

__global__ void k_plan(const long long *__restrict__ set_ptr, const vor_box *__restrict__ boxes,
                       int n_sets, long long n1, vor_box box1, int s_fixed, int load_pct,
                       long long hn_total, long long hm_sum, long long hg_sum,
                       SetMeta *__restrict__ sets, WsHeader *hdr) {
    __shared__ long long sh[32];
    long long gcarry = 0, mcarry = 0;
    int bad = 0;
    for (int j0 = 0; j0 < n_sets; j0 += SCAN_T) {
        const int j = j0 + threadIdx.x;
        long long g2 = 0, mm = 0;
        SetMeta M = {};
        if (j < n_sets) {
            const long long a = set_ptr ? set_ptr[j] : 0, b = set_ptr ? set_ptr[j + 1] : n1;
            const vor_box bx = boxes ? boxes[j] : box1;
            SetPlan pl;
            if (b < a || (j == 0 && a != 0) || !plan_set(b - a > 0 ? b - a : 1, bx.w, bx.h, s_fixed, pl)) {
                bad = 1;
            } else {
                M.site_base = a;
                M.n = (int)(b - a);
                M.W = bx.w;
                M.H = bx.h;
                M.G = pl.G;
                M.s_min = pl.s_min;
                M.s_max = pl.s_max;
                M.s_fixed = s_fixed;
                M.m_max = pl.m_max;
                M.load_pct = load_pct;
                g2 = (long long)pl.G * pl.G;
                mm = pl.m_max;
            }
            if (j == n_sets - 1 && b != hn_total) bad = 1;
        }
        long long gt, mt;
        const long long gex = block_exclusive<long long>(g2, sh, gt);
        block_exclusive<long long>(mm, sh, mt);
        if (j < n_sets) {
            M.coarse_base = gcarry + gex;
            sets[j] = M;
        }
        gcarry += gt;
        mcarry += mt;
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0 && (bad || gcarry > hg_sum || mcarry > hm_sum)) atomicOr(&hdr->err, ERRB_ARG);
}

__global__ void k_pick_grid(SetMeta *__restrict__ sets, int n_sets, int s_fixed, WsHeader *hdr) {
    __shared__ long long sh[32];
    if (hdr->err) return;
    long long carry = 0;
    for (int j0 = 0; j0 < n_sets; j0 += SCAN_T) {
        const int j = j0 + threadIdx.x;
        long long m = 0;
        int s = 1, m1 = 1, m2 = 1;
        if (j < n_sets) {
            const SetMeta &M = sets[j];
            s = s_fixed;
            if (s <= 0) {
                if (M.n > 0) {
                    const double cmed = exp2(M.acc / (double)M.n);   // typical sites per coarse cell
                    const double area = ((double)M.W / M.G) * ((double)M.H / M.G);
                    s = (int)sqrt(0.01 * M.load_pct * area / cmed);
                } else {
                    s = M.s_max;
                }
                s = max(M.s_min, min(M.s_max, s));
            }
            s = max(s, 1);
            m1 = (M.W + s - 1) / s;
            m2 = (M.H + s - 1) / s;
            m = (long long)m1 * m2;
        }
        long long total;
        const long long ex = block_exclusive<long long>(m, sh, total);
        if (j < n_sets) {
            SetMeta &M = sets[j];
            M.s = s;
            M.m1 = m1;
            M.m2 = m2;
            M.bucket_base = carry + ex;
        }
        carry += total;
    }
    if (threadIdx.x == 0) hdr->m_total = (int)carry;
}

// ---------------------------------------------------------------------------
// K3: compaction (CSR cells, float64 vertices, Delaunay pairs)
// ---------------------------------------------------------------------------

struct CompactParams {
    const int2 *sites;
    int n;
    int share;                  // 1: a vertex is computed once, by the smallest site among its cells
    const SetMeta *sets;
    const int *sset;
    const int *ecount, *dcount, *loc, *slot, *spill;
    const long long *cell_ptr, *del_ptr;
    int *edge_label;
    double *vx, *vy;
    int *del_edge;
    long long edge_cap, del_cap;
    WsHeader *hdr;
};

// line of label `lab` of the cell of p: 2 <n, v - p> = c (set_sites: the
// sites of p's set, indexed by local label)
__device__ __forceinline__ void line_of(const int2 *set_sites, int W, int H, int2 p, int lab, int &nx,
                                        int &ny, i64 &c) {
    if (lab >= 0) {
        const int2 a = set_sites[lab];
        nx = a.x - p.x;
        ny = a.y - p.y;
        c = (i64)nx * nx + (i64)ny * ny;
    } else {
        nx = ny = 0;
        if (lab == VOR_SIDE_BOTTOM) ny = -p.y;
        else if (lab == VOR_SIDE_RIGHT) nx = W - p.x;
        else if (lab == VOR_SIDE_TOP) ny = H - p.y;
        else nx = -p.x;
        c = 2 * ((i64)nx * nx + (i64)ny * ny);
    }
}

// Vertex coordinates without float64 arithmetic (the float64 pipe of this
// GPU is narrow, and 64-bit integer <-> float conversions issue to it).  A
// coordinate is the quotient q = num / D of two integers with 0 <= q <= 2^20
// (the vertex lies in the box), 0 < D < 2^44 and num < 2^63 after taking
// D's sign into num.  q is computed as a float-float pair (about 44 correct
// bits, on the FMA pipe), turned into the fixed-point integer F ~ q 2^40,
// snapped to the exact k 2^40 when the nearest integer k has k D == num, and
// written as a float64 assembled from F's bits (IEEE 754 binary64: sign,
// 11-bit exponent biased by 1023, 52-bit fraction).  Error below 2^-42 q +
// 2^-39, far inside the 1e-9 tolerance of the vertices; integer
// coordinates are exact (tests/test_gpu_vertex_quotient.py checks both at
// the extremes through vor_vertex_quotients).
//
// The quotient of two float-float numbers is the double-length division of
// T. J. Dekker, "A floating-point technique for extending the available
// precision", Numer. Math. 18 (1971): a first quotient qh, the residual
// a - qh d, and one correction term.  The product qh dh is formed exactly
// as ph + pl with one fused multiply-add (the FMA form of Dekker's exact
// product, "TwoProductFMA" in Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005)).

// 0 <= v < 2^63 as a float-float pair h + l: h holds v's top 24 bits
// exactly, l the rest rounded (relative error of h + l below 2^-46)
__device__ __forceinline__ void u63_to_ff(unsigned long long v, float &h, float &l) {
    const int top = 63 - __clzll(v);
    const int sh = top > 23 ? top - 23 : 0;
    const unsigned hi = (unsigned)(v >> sh);
    const unsigned long long rem = v - ((unsigned long long)hi << sh);
    h = (float)hi * __uint_as_float((unsigned)(127 + sh) << 23);      // hi 2^sh, exact
    l = fmaf((float)(unsigned)(rem >> 32), 4294967296.f, (float)(unsigned)rem);
}

// a / d in float-float, a and d given as float-float pairs, r ~ 1 / dh
__device__ __forceinline__ void ff_div(float ah, float al, float dh, float dl, float r,
                                       float &qh, float &ql) {
    qh = ah * r;
    const float ph = qh * dh, pl = fmaf(qh, dh, -ph);  // qh dh exactly, as ph + pl
    const float e = ((ah - ph) - pl) + al - qh * dl;    // a - qh d, to a few ulp of it
    ql = e * r;
}

// x 2^40 truncated to an integer, |x| < 2^21
__device__ __forceinline__ long long f32_fixed40(float x) {
    const unsigned u = __float_as_uint(x);
    const int e = (int)((u >> 23) & 0xff) - 110;       // x = m 2^(e - 40), m the 24-bit significand
    const unsigned long long m = (u & 0x7fffffu) | 0x800000u;
    const unsigned long long v = e >= 0 ? m << e : (e > -24 ? m >> -e : 0ull);
    return (u >> 31) ? -(long long)v : (long long)v;
}

// num / D (D > 0) from the float-float quotient qh + ql, as described above
__device__ __forceinline__ double vertex_coord(long long num, unsigned long long D, float qh, float ql) {
    long long F = f32_fixed40(qh) + f32_fixed40(ql);
    const long long k = (F + (1ll << 39)) >> 40;
    if (k >= 0 && (unsigned long long)k * D == (unsigned long long)num) F = k << 40;
    const unsigned long long sgn = F < 0 ? 1ull << 63 : 0ull;
    const unsigned long long mag = F < 0 ? 0ull - (unsigned long long)F : (unsigned long long)F;
    if (mag == 0) return 0.0;
    const int top = 63 - __clzll(mag);                   // 2^top <= mag < 2^61
    const unsigned long long m = top > 52 ? mag >> (top - 52) : mag << (52 - top);
    const unsigned long long bits = sgn | ((unsigned long long)(top - 40 + 1023) << 52) |
                                    (m & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

// num / D for 0 <= num < 2^63, 0 < D < 2^44, num < 2^21 D: the float-float
// denominator (with the approximate reciprocal of its head) is shared by the
// two coordinates of a vertex
struct FFDen { float h, l, r; };

__device__ __forceinline__ FFDen ff_den(unsigned long long D) {
    FFDen d;
    u63_to_ff(D, d.h, d.l);
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(d.r) : "f"(d.h));
    return d;
}

__device__ __forceinline__ double ff_quotient(long long num, unsigned long long D, const FFDen &d) {
    float xh, xl, qh, ql;
    u63_to_ff((unsigned long long)num, xh, xl);
    ff_div(xh, xl, d.h, d.l, d.r, qh, ql);
    return vertex_coord(num, D, qh, ql);
}

__global__ void k_vertex_quotients(const long long *__restrict__ num,
                                   const unsigned long long *__restrict__ den, long long n,
                                   double *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long a = num[i];
    const unsigned long long D = den[i];
    // outside the domain of the conversion: NaN
    if (a < 0 || D == 0 || D >= (1ull << 44) || (unsigned long long)a / D >= (1ull << 21)) {
        out[i] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    out[i] = ff_quotient(a, D, ff_den(D));
}

// The line of a side of X for the cell of p (labels -1..-4)
__device__ __forceinline__ void side_line(int W, int H, int2 p, int lab, int &nx, int &ny, i64 &c) {
    nx = ny = 0;
    if (lab == VOR_SIDE_BOTTOM) ny = -p.y;
    else if (lab == VOR_SIDE_RIGHT) nx = W - p.x;
    else if (lab == VOR_SIDE_TOP) ny = H - p.y;
    else nx = -p.x;
    c = 2 * ((i64)nx * nx + (i64)ny * ny);
}

// The vertex between edge q (line a, label a_lab) and edge q + 1 (line b) of
// the cell of p, its label, and the Delaunay pair (kl, a_lab) when a_lab > kl,
// at rank = the number of the cell's labels between kl and a_lab (labs[0..e))
// The float64 vertex (p D + N) / D of the lines (ax, ay, ac), (bx, by, bc)
// of the cell of p.
__device__ __forceinline__ void vertex_of(int2 p, int ax, int ay, i64 ac, int bx, int by, i64 bc,
                                          double &vx, double &vy) {
    i64 Nx, Ny, D;
    intersect(ax, ay, ac, bx, by, bc, Nx, Ny, D);
    // absolute vertex (p D + N) / D; the numerators lie in [0, W |D|]
    const i64 numx = (i64)((unsigned long long)p.x * (unsigned long long)D + (unsigned long long)Nx);
    const i64 numy = (i64)((unsigned long long)p.y * (unsigned long long)D + (unsigned long long)Ny);
    // the quotients with D > 0 (numerators >= 0: the vertex is in the box)
    const unsigned long long aD = D < 0 ? 0ull - (unsigned long long)D : (unsigned long long)D;
    const long long ax_ = D < 0 ? -numx : numx, ay_ = D < 0 ? -numy : numy;
    const FFDen fd = ff_den(aD);
    vx = ff_quotient(ax_, aD, fd);
    vy = ff_quotient(ay_, aD, fd);
}

// A vertex of cell kl between its edges a_lab and b_lab belongs to the cells
// of kl and of the neighbour sites among a_lab, b_lab (sides are no cells).
// Its owner is the cell of the smallest of these sites.
__device__ __forceinline__ bool owns_vertex(int kl, int a_lab, int b_lab) {
    return (a_lab < 0 || kl < a_lab) && (b_lab < 0 || kl < b_lab);
}

// The vertex as its owner sees it: the meeting point of the owner's lines to
// the other two members (sites, or a side of X), relative to the owner's
// site.  Every cell that lists the vertex computes it from the same integers,
// so all of them hold the same float64 coordinates (the order of the two
// lines only flips the signs of N and D, which the division undoes).
// p: the site of cell kl; A, B: the sites a_lab, b_lab (ignored for sides).
__device__ __forceinline__ void vertex_canonical(int W, int H, int kl, int2 p, int a_lab, int2 A,
                                                 int b_lab, int2 B, double &vx, double &vy) {
    int ol = kl, m1 = a_lab, m2 = b_lab;
    int2 r = p, s1 = A, s2 = B;
    if (a_lab >= 0 && a_lab < ol && (b_lab < 0 || a_lab < b_lab)) {
        ol = a_lab; r = A; m1 = kl; s1 = p;
    } else if (b_lab >= 0 && b_lab < ol) {
        ol = b_lab; r = B; m2 = kl; s2 = p;
    }
    int ax, ay, bx, by;
    i64 ac, bc;
    if (m1 >= 0) { ax = s1.x - r.x; ay = s1.y - r.y; ac = (i64)ax * ax + (i64)ay * ay; }
    else side_line(W, H, r, m1, ax, ay, ac);
    if (m2 >= 0) { bx = s2.x - r.x; by = s2.y - r.y; bc = (i64)bx * bx + (i64)by * by; }
    else side_line(W, H, r, m2, bx, by, bc);
    vertex_of(r, ax, ay, ac, bx, by, bc, vx, vy);
}

__device__ __forceinline__ void emit_vertex(const CompactParams &Q, int2 p, int kl, int W, int H,
                                            long long off, long long doff, const int *labs, int e,
                                            int q, int a_lab, int2 A, int b_lab, int2 B) {
    Q.edge_label[off + q] = a_lab;
    // with sharing, only the owner computes; k_share_vertices copies it
    if (!Q.share || owns_vertex(kl, a_lab, b_lab)) {
        double vx, vy;
        vertex_canonical(W, H, kl, p, a_lab, A, b_lab, B, vx, vy);
        Q.vx[off + q] = vx;
        Q.vy[off + q] = vy;
    }
    if (a_lab > kl) {
        int rank = 0;
        for (int j = 0; j < e; j++) {
            const int o = labs[j];
            rank += (o > kl && o < a_lab) ? 1 : 0;
        }
        Q.del_edge[2 * (doff + rank)] = kl;
        Q.del_edge[2 * (doff + rank) + 1] = a_lab;
    }
}

// A warp takes 32 consecutive cells.  Their labels and neighbour sites are
// staged in shared memory (one entry per edge, the cells' edges end to end
// after a prefix sum of e_k over the lanes), and then every lane computes
// one vertex at a time, whatever cell it belongs to: the lanes stay busy
// however the cells' edge counts differ.  A warp whose cells have more
// edges than its staging area lists each cell on one lane from global memory.
constexpr int COMPACT_W = 4;                 // warps per block
constexpr int COMPACT_T = 32 * COMPACT_W;
constexpr int COMPACT_V = 32 * SLOT_CAP;     // staged edges per warp

struct CompactCell {
    const int *src;                          // the cell's labels (fixed slot or spill)
    int2 p;
    int W, H, kl, e, start;                  // kl: the cell's index in its set
    long long off, doff;                     // first edge, first Delaunay pair
};

__global__ void __launch_bounds__(COMPACT_T) k_compact(CompactParams Q) {
    __shared__ int s_lab[COMPACT_W][COMPACT_V];
    __shared__ int2 s_nb[COMPACT_W][COMPACT_V];
    __shared__ CompactCell s_cell[COMPACT_W][32];
    if (Q.hdr->err) return;
    const unsigned FULL = 0xffffffffu;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k0 = (blockIdx.x * COMPACT_W + w) * 32;
    if (k0 >= Q.n) return;                                   // warp-uniform
    const int k = k0 + lane;
    CompactCell ci{};
    const int2 *ss = Q.sites;
    if (k < Q.n) {
        const SetMeta &M = set_of(Q.sets, Q.sset, k);
        ss = Q.sites + M.site_base;
        ci.p = Q.sites[k];
        ci.W = M.W;
        ci.H = M.H;
        ci.kl = k - (int)M.site_base;
        ci.e = Q.ecount[k];
        ci.off = Q.cell_ptr[k];
        ci.doff = Q.del_ptr[k];
        const int l = Q.loc[k];
        ci.src = l < 0 ? Q.slot + (size_t)k * SLOT_CAP : Q.spill + l;
        if (ci.off + ci.e > Q.edge_cap || ci.doff + Q.dcount[k] > Q.del_cap) {
            atomicOr(&Q.hdr->err, ERRB_SPILL);
            ci.e = 0;
        }
    }
    // the cells' edges end to end: an inclusive prefix sum over the lanes
    int incl = ci.e;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    const int V = __shfl_sync(FULL, incl, 31);
    ci.start = incl - ci.e;
    if (V > COMPACT_V) {
        // more edges than the staging area: each lane its own cell
        for (int q = 0; q < ci.e; q++) {
            const int a_lab = ci.src[q];
            const int b_lab = ci.src[q + 1 < ci.e ? q + 1 : 0];
            const int2 A = a_lab >= 0 ? ss[a_lab] : ci.p, B = b_lab >= 0 ? ss[b_lab] : ci.p;
            emit_vertex(Q, ci.p, ci.kl, ci.W, ci.H, ci.off, ci.doff, ci.src, ci.e, q, a_lab, A, b_lab, B);
        }
        return;
    }
    s_cell[w][lane] = ci;
    __syncwarp();
    // the cell (lane) that owns edge v: the first lane with incl > v
    auto owner = [&](int v) {
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int x = __shfl_sync(FULL, incl, lo + step - 1);
            if (x <= v) lo += step;
        }
        return lo;
    };
    int *lab_w = s_lab[w];
    int2 *nb_w = s_nb[w];
    for (int v0 = 0; v0 < V; v0 += 32) {                    // stage labels and neighbour sites
        const int v = v0 + lane;
        const int c = owner(min(v, V - 1));
        if (v < V) {
            const CompactCell &cc = s_cell[w][c];
            const int lab = __ldg(cc.src + (v - cc.start));
            lab_w[v] = lab;
            nb_w[v] = lab >= 0 ? __ldg(Q.sites + (k0 + c - cc.kl) + lab) : make_int2(0, 0);
        }
    }
    __syncwarp();
    for (int v0 = 0; v0 < V; v0 += 32) {                    // one vertex per lane
        const int v = v0 + lane;
        const int c = owner(min(v, V - 1));
        if (v < V) {
            const CompactCell &cc = s_cell[w][c];
            const int q = v - cc.start;
            const int vb = q + 1 < cc.e ? v + 1 : cc.start;
            const int a_lab = lab_w[v], b_lab = lab_w[vb];
            emit_vertex(Q, cc.p, cc.kl, cc.W, cc.H, cc.off, cc.doff, lab_w + cc.start, cc.e, q, a_lab,
                        nb_w[v], b_lab, nb_w[vb]);
        }
    }
}

// Vertex sharing (opts.share_vertices), after k_compact: each vertex a cell
// does not own is copied from the owning neighbour o, where it lies between
// o's edges for this cell and for the vertex's third line.  Where o lists no
// such pair (a vertex shared by four or more cells, when more than three
// sites lie on one empty circle) the cell computes the vertex itself.  One
// thread per cell.
__global__ void k_share_vertices(CompactParams Q) {
    if (Q.hdr->err) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Q.n) return;
    const SetMeta &M = set_of(Q.sets, Q.sset, k);
    const int base = (int)M.site_base;
    const int kl = k - base;
    const long long off = Q.cell_ptr[k];
    const int e = (int)(Q.cell_ptr[k + 1] - off);
    const int2 *ss = Q.sites + base;
    for (int q = 0; q < e; q++) {
        const int a = Q.edge_label[off + q], b = Q.edge_label[off + (q + 1 < e ? q + 1 : 0)];
        if (owns_vertex(kl, a, b)) continue;
        const int o = (a >= 0 && (b < 0 || a < b)) ? a : b;      // the owner: a site < kl
        const int x = o == a ? b : a;                             // the vertex's third line
        const long long ob = Q.cell_ptr[base + o];
        const int oe = (int)(Q.cell_ptr[base + o + 1] - ob);
        int j = -1;
        for (int r = 0; r < oe && j < 0; r++) {
            const int l1 = Q.edge_label[ob + r], l2 = Q.edge_label[ob + (r + 1 < oe ? r + 1 : 0)];
            if ((l1 == kl && l2 == x) || (l1 == x && l2 == kl)) j = r;
        }
        if (j >= 0) {
            Q.vx[off + q] = Q.vx[ob + j];
            Q.vy[off + q] = Q.vy[ob + j];
        } else {
            const int2 p = Q.sites[k];
            double vx, vy;
            vertex_canonical(M.W, M.H, kl, p, a, a >= 0 ? ss[a] : p, b, b >= 0 ? ss[b] : p, vx, vy);
            Q.vx[off + q] = vx;
            Q.vy[off + q] = vy;
        }
    }
}

// per set: offset of its Delaunay pairs (out[n_sets] = total)
__global__ void k_set_del_ptr(const SetMeta *__restrict__ sets, int n_sets, int n,
                              const long long *__restrict__ del_ptr, long long *__restrict__ out,
                              const WsHeader *hdr) {
    if (hdr->err) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n_sets) return;
    out[j] = del_ptr[j < n_sets ? sets[j].site_base : n];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct Layout {
    int s_fixed, lanes, target, n_sets, load_pct, fine_split, block;
    long long n, m_sum, g_sum;
    size_t hdr, sets, sset, bstart, rank, sxy, sid, partial, ecount, dcount, loc, del_ptr, slot,
        spill, deferred, deferred2, deferred3, deferred4, deferred5, gcount, grho2, gtab, glab, coarse,
        fdesc, fpool, coop, total;
    int spill_cap;
    int n_partial;
    long long n_max;          // largest set
    int coop_slices;          // global-memory slices of the block-per-cell tier
};

// Slices of the block-per-cell tier's global-memory mode: one slice holds a
// cell of the largest set whatever its size; a batch of many sets gets up to
// 64 slices within 16 bytes per site.
constexpr int COOP_MAX_SLICES = 64;
static int coop_slices_for(long long n_total, long long n_max) {
    const long long slice = coop_slice_bytes(n_max);
    long long k = slice > 0 ? 16 * n_total / slice : 1;
    if (k < 1) k = 1;
    if (k > COOP_MAX_SLICES) k = COOP_MAX_SLICES;
    return (int)k;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Sizes of the workspace of a batch (set_ptr null: one set of n1 sites in
// box1).  Every per-set size comes from plan_set, which the planning kernel
// evaluates again on the device.
static bool resolve(const int64_t *set_ptr, const vor_box *boxes, int n_sets, int64_t n1,
                    vor_box box1, const vor_opts *o, Layout &L) {
    vor_opts d;
    vor_opts_default(&d);
    if (!o) o = &d;
    if (n_sets < 1 || n_sets > (1 << 24)) return false;
    L.s_fixed = 0;
    if (o->bucket_side > 0) {
        if (o->bucket_side > (1 << 20)) return false;
        L.s_fixed = o->bucket_side;
    }
    L.n_sets = n_sets;
    L.m_sum = 0;
    L.g_sum = 0;
    L.n_max = 1;
    if (set_ptr && set_ptr[0] != 0) return false;
    for (int j = 0; j < n_sets; j++) {
        const int64_t a = set_ptr ? set_ptr[j] : 0, b = set_ptr ? set_ptr[j + 1] : n1;
        const vor_box bx = boxes ? boxes[j] : box1;
        if (b < a) return false;
        if (!set_ptr && b < 1) return false;
        SetPlan pl;
        if (!plan_set(b - a > 0 ? b - a : 1, bx.w, bx.h, L.s_fixed, pl)) return false;
        L.m_sum += pl.m_max;
        L.g_sum += (long long)pl.G * pl.G;
        if (b - a > L.n_max) L.n_max = b - a;
    }
    L.n = set_ptr ? set_ptr[n_sets] : n1;
    if (L.n < 0 || L.n > (1 << 27) || L.m_sum > (1ll << 30)) return false;
    L.lanes = o->lanes_per_cell > 0 ? o->lanes_per_cell : 1;
    if (L.lanes != 1 && L.lanes != 2 && L.lanes != 4 && L.lanes != 8 && L.lanes != 16 && L.lanes != 32) return false;
    // defaults from a sweep of the uniform 1M build (target x load: 24 and
    // 6 sites per bucket, 1.634 ms against 1.715 ms with 20 and 2)
    L.target = o->target > 0 ? o->target : 24;
    if (L.target > 40) return false;
    L.load_pct = o->bucket_load_pct > 0 ? o->bucket_load_pct : 600;
    if (L.load_pct < 25 || L.load_pct > 1600) return false;
    L.fine_split = o->fine_split;
    if (L.fine_split != 0 && (L.fine_split < 4 || L.fine_split > 65536)) return false;
    L.block = o->block_threads > 0 ? o->block_threads : 64;
    if (L.block != 32 && L.block != 64 && L.block != 128) return false;
    const size_t m = (size_t)L.m_sum;
    const size_t nn = (size_t)(L.n > 0 ? L.n : 1);
    const int nb_b = (int)((m + SCAN_TILE - 1) / SCAN_TILE), nb_n = (int)((nn + SCAN_TILE - 1) / SCAN_TILE);
    L.n_partial = (nb_b > nb_n ? nb_b : nb_n) + 1;
    L.spill_cap = (int)(nn * 10 < (1u << 30) ? nn * 10 : (1u << 30));
    size_t at = 0;
    L.hdr = at;      at = align256(at + 256);
    L.sets = at;     at = align256(at + (size_t)n_sets * sizeof(SetMeta));
    L.sset = at;     at = align256(at + (set_ptr ? nn * 4 : 0));
    L.bstart = at;   at = align256(at + (m + 1) * 4);
    L.rank = at;     at = align256(at + nn * 4);    // bucket ranks; then the first pass's disc needs
    L.sxy = at;      at = align256(at + nn * 8);
    L.sid = at;      at = align256(at + nn * 4);
    L.partial = at;  at = align256(at + (size_t)L.n_partial * 8);
    L.ecount = at;   at = align256(at + nn * 4);
    L.dcount = at;   at = align256(at + nn * 4);
    L.loc = at;      at = align256(at + nn * 4);
    L.del_ptr = at;  at = align256(at + (nn + 1) * 8);
    L.slot = at;     at = align256(at + nn * SLOT_CAP * 4);
    L.spill = at;    at = align256(at + (size_t)L.spill_cap * 4);
    L.deferred = at; at = align256(at + nn * 4);
    L.deferred2 = at; at = align256(at + nn * 4);
    L.deferred3 = at; at = align256(at + nn * 4);
    L.deferred4 = at; at = align256(at + nn * 4);
    L.deferred5 = at; at = align256(at + nn * 4);   // flower passes alternate with deferred2
    L.gcount = at;   at = align256(at + nn * 4);
    L.grho2 = at;    at = align256(at + nn * 8);
    L.gtab = at;     at = align256(at + (size_t)gather_rows(nn) * 8 * (size_t)pass_gather_width());
    L.glab = at;     at = align256(at + (size_t)gather_rows(nn) * 4 * (size_t)pass_gather_width());
    L.coarse = at;   at = align256(at + (size_t)L.g_sum * 4);
    const bool fine = L.fine_split > 0;
    L.fdesc = at;    at = align256(at + (fine ? m * 4 : 0));
    L.fpool = at;    at = align256(at + (fine ? (size_t)fine_pool_cap((long long)nn) * 4 : 0));
    L.coop_slices = coop_slices_for((long long)nn, L.n_max);
    L.coop = at;     at = align256(at + (size_t)L.coop_slices * (size_t)coop_slice_bytes(L.n_max));
    L.total = at;
    return true;
}

// stage timing (vor_stage_timing / vor_stage_ms): events 0..N_STAGES
constexpr int N_STAGES = 6;
static bool g_timing = false;
static cudaEvent_t g_ev[N_STAGES + 1];
static bool g_ev_made = false;
static bool g_ev_recorded = false;

static void mark(int i, cudaStream_t st) {
    if (!g_timing) return;
    // inside a stream capture the events become record nodes of the graph
    // (external records), so that every replay records them
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(g_ev[i], st, cudaEventRecordExternal);
    else
        cudaEventRecord(g_ev[i], st);
}

// kernels launched by this library in this process (vor_kernel_launches)
static std::atomic<long long> g_launches{0};

struct BatchArgs {
    const int2 *sites;
    const long long *set_ptr;   // device; null: one set
    const vor_box *boxes;       // device; null: one set
    long long n1;
    vor_box box1;
    long long *del_set_ptr;     // device output; may be null for one set
};

static int launch_build(const BatchArgs &A, const vor_opts *o, void *ws, const Layout &L,
                        const vor_out *out, cudaStream_t st) {
    vor_opts d;
    vor_opts_default(&d);
    if (!o) o = &d;
    const int n = (int)L.n;
    char *base = (char *)ws;
    WsHeader *hdr = (WsHeader *)(base + L.hdr);
    SetMeta *sets = (SetMeta *)(base + L.sets);
    int *sset = A.set_ptr ? (int *)(base + L.sset) : nullptr;
    int *bstart = (int *)(base + L.bstart);
    int *rank = (int *)(base + L.rank);
    int2 *sxy = (int2 *)(base + L.sxy);
    int *sid = (int *)(base + L.sid);
    long long *partial = (long long *)(base + L.partial);
    int *ecount = (int *)(base + L.ecount);
    int *dcount = (int *)(base + L.dcount);
    int *loc = (int *)(base + L.loc);
    long long *del_ptr = (long long *)(base + L.del_ptr);
    int *slot = (int *)(base + L.slot);
    int *spill = (int *)(base + L.spill);
    int *deferred = (int *)(base + L.deferred);
    int *deferred2 = (int *)(base + L.deferred2);
    int *deferred3 = (int *)(base + L.deferred3);
    int *deferred4 = (int *)(base + L.deferred4);
    int *deferred5 = (int *)(base + L.deferred5);
    int *coarse = (int *)(base + L.coarse);
    const int2 *sites = A.sites;

    long long launched = 0;
    struct Count {                    // adds this build's launches to the total
        long long &n;
        ~Count() { g_launches += n; }
    } count_on_exit{launched};
    mark(0, st);
    if (cudaMemsetAsync(hdr, 0, 256, st) != cudaSuccess) return VOR_E_CUDA;
    k_plan<<<1, SCAN_T, 0, st>>>(A.set_ptr, A.boxes, L.n_sets, A.n1, A.box1, L.s_fixed, L.load_pct,
                                 L.n, L.m_sum, L.g_sum, sets, hdr);
    launched++;
    if (n == 0) {
        // nothing but empty sets: empty outputs
        if (cudaMemsetAsync(out->cell_ptr, 0, 8, st) != cudaSuccess ||
            cudaMemsetAsync(out->totals, 0, 16, st) != cudaSuccess ||
            (A.del_set_ptr &&
             cudaMemsetAsync(A.del_set_ptr, 0, (size_t)(L.n_sets + 1) * 8, st) != cudaSuccess))
            return VOR_E_CUDA;
        for (int i = 1; i <= N_STAGES; i++) mark(i, st);
        if (g_timing) g_ev_recorded = true;
        return cudaGetLastError() == cudaSuccess ? VOR_OK : VOR_E_CUDA;
    }
    if (cudaMemsetAsync(bstart, 0, (size_t)(L.m_sum + 1) * 4, st) != cudaSuccess) return VOR_E_CUDA;
    const int T = 256;
    const int gn = (n + T - 1) / T;
    if (sset) {
        k_site_set<<<gn, T, 0, st>>>(A.set_ptr, L.n_sets, n, sset, hdr);
        launched++;
    }
    // the coarse occupancy grid: the density probe of the bucket side, then
    // its summed-area table (the sites of any rectangle of coarse cells)
    if (cudaMemsetAsync(coarse, 0, (size_t)L.g_sum * 4, st) != cudaSuccess) return VOR_E_CUDA;
    k_probe_count<<<gn, T, 0, st>>>(sites, n, sets, sset, coarse, hdr);
    launched++;
    if (L.s_fixed <= 0) {
        k_probe_mean<<<gn, T, 0, st>>>(sites, n, sets, sset, coarse, hdr);
        launched++;
    }
    k_coarse_sat<<<L.n_sets < 152 * 2 ? L.n_sets : 152 * 2, SAT_T, 0, st>>>(sets, L.n_sets, coarse, hdr);
    launched++;
    k_pick_grid<<<1, SCAN_T, 0, st>>>(sets, L.n_sets, L.s_fixed, hdr);
    k_bucket_count<<<gn, T, 0, st>>>(sites, n, sets, sset, bstart, rank, hdr);
    launched += scan<int>(bstart, (int)L.m_sum, &hdr->m_total, bstart, (int *)partial, nullptr, hdr, st);
    int *fdesc = nullptr, *fpool = nullptr;
    if (L.fine_split > 0) {
        // the second level of the adaptive buckets: divide the dense buckets
        fdesc = (int *)(base + L.fdesc);
        fpool = (int *)(base + L.fpool);
        const int gm = (int)((L.m_sum + T - 1) / T < 152 * 64 ? (L.m_sum + T - 1) / T : 152 * 64);
        k_fine_plan<<<gm, T, 0, st>>>(bstart, (int)L.m_sum, L.fine_split, fdesc, fpool,
                                      fine_pool_cap(L.n), hdr);
        k_fine_rank<<<gn, T, 0, st>>>(sites, n, sets, sset, bstart, fdesc, fpool, rank, hdr);
        k_fine_scan<<<gm, T, 0, st>>>(bstart, (int)L.m_sum, fdesc, fpool, hdr);
        launched += 3;
    }
    k_bucket_scatter<<<gn, T, 0, st>>>(sites, n, sets, sset, bstart, rank, fdesc, fpool, sxy, sid, hdr);
    launched += 3;                    // pick, count, scatter
    if (o->check_duplicates) {
        k_dup_check<<<gn, T, 0, st>>>(sxy, n, sets, sset, bstart, hdr);
        launched++;
    }
    if (cudaGetLastError() != cudaSuccess) return VOR_E_CUDA;
    mark(1, st);

    CellParams P;
    memset(&P, 0, sizeof(P));
    P.sites = sites; P.sxy = sxy; P.sid = sid; P.bstart = bstart;
    P.sets = sets; P.sset = sset;
    P.n = n;
    P.target = L.target; P.exact_only = o->exact_only; P.collect_stats = o->collect_stats;
    P.ecount = ecount; P.dcount = dcount; P.loc = loc; P.slot = slot; P.spill = spill;
    P.spill_cap = L.spill_cap;
    P.cell_list = nullptr; P.list_count = nullptr; P.n_list = 0;
    P.fdesc = fdesc; P.fpool = fpool;
    P.coarse_sat = coarse;
    P.hdr = hdr;
    int *med_list = deferred2, *med_count = &hdr->ndeferred2;   // the medium tier's cells
    if (L.lanes == 1) {
        int *gcount = (int *)(base + L.gcount), *glab = (int *)(base + L.glab);
        float2 *gtab = (float2 *)(base + L.gtab);
        long long *grho2 = (long long *)(base + L.grho2);
        // first pass over all cells: the cells its disc does not certify
        // (or that exceed its table) go on to the second pass
        P.deferred = deferred;
        P.deferred_count = &hdr->ndeferred;
        // the bucket ranks are free after bucketing: they carry the first
        // pass's disc needs to the second pass
        P.need_out = (float *)rank;
        P.store_poly = 1;
        if (launch_gather_pass(P, 1, gcount, grho2, gtab, glab, st) != cudaSuccess) return VOR_E_CUDA;
        mark(2, st);
        CellParams P1 = P;
        P1.next_cell = &hdr->pass_next[0];          // cells by warp generations from a counter
        if (launch_cells_pass(P1, 1, gcount, grho2, gtab, glab, L.block, st) != cudaSuccess) return VOR_E_CUDA;
        mark(3, st);
        // second pass: a disc with about 2.2 times the sites
        CellParams P2 = P;
        P2.cell_list = deferred;
        P2.list_count = &hdr->ndeferred;
        P2.n_list = n;
        P2.deferred = deferred2;
        P2.deferred_count = &hdr->ndeferred2;
        P2.need_out = nullptr;
        P2.need_in = (const float *)rank;
        if (launch_gather_pass(P2, 2, gcount, grho2, gtab, glab, st) != cudaSuccess) return VOR_E_CUDA;
        P2.next_cell = &hdr->pass_next[1];
        if (launch_cells_pass(P2, 2, gcount, grho2, gtab, glab, L.block, st) != cudaSuccess) return VOR_E_CUDA;
        // flower passes (batches of several sets, where small clustered sets
        // leave many cells uncertified; a single set leaves too few for a
        // pass that fills the GPU): the flower of the polygon an earlier
        // pass left, its sites nearest p first, up to 124 entries; a cell its
        // certificate does not accept leaves the new polygon for the next
        // flower pass, and what is left after the last goes to the medium tier
        int *fin = deferred2, *fin_count = &hdr->ndeferred2;
        const int passes = L.n_sets > 1 ? FLOWER_PASSES : 0;
        for (int f = 0; f < passes; f++) {
            int *fout = (f & 1) ? deferred2 : deferred5;
            CellParams P3 = P2;
            P3.cell_list = fin;
            P3.list_count = fin_count;
            P3.deferred = fout;
            P3.deferred_count = &hdr->fcount[f];
            P3.need_in = nullptr;
            P3.store_poly = 1;
            P3.next_cell = nullptr;
            if (launch_gather_pass(P3, 3, gcount, grho2, gtab, glab, st) != cudaSuccess) return VOR_E_CUDA;
            P3.next_cell = &hdr->fnext[f];
            if (launch_cells_pass(P3, 3, gcount, grho2, gtab, glab, L.block, st) != cudaSuccess) return VOR_E_CUDA;
            fin = fout;
            fin_count = &hdr->fcount[f];
        }
        med_list = fin;
        med_count = fin_count;
        if (passes && cudaMemsetAsync(&hdr->flower_passes, passes, 1, st) != cudaSuccess) return VOR_E_CUDA;
        launched += 4 + 2 * passes;
        mark(4, st);
    } else {
        P.deferred = deferred2;
        P.deferred_count = &hdr->ndeferred2;
        mark(2, st);
        if (launch_cells_fast(P, L.lanes, st) != cudaSuccess) return VOR_E_CUDA;
        launched++;
        mark(3, st);
        mark(4, st);
    }
    // what is left: one warp per cell (medium capacities), then one block per
    // cell with its arrays in shared memory, then in global memory (room for
    // every site of the set: no valid cell is refused)
    CellParams PM = P;
    PM.need_out = nullptr;
    PM.need_in = nullptr;
    PM.store_poly = 0;
    PM.seed_poly = L.lanes == 1 ? 1 : 0;     // the thread passes left their polygons
    PM.cell_list = med_list;
    PM.list_count = med_count;
    PM.n_list = n;
    PM.deferred = deferred3;
    PM.deferred_count = &hdr->ndeferred3;
    PM.next_cell = &hdr->large_next;
    if (launch_cells_medium(PM, n, L.n_max, L.n_sets == 1, st) != cudaSuccess) return VOR_E_CUDA;
    CellParams PL = PM;
    PL.cell_list = deferred3;
    PL.list_count = &hdr->ndeferred3;
    PL.deferred = deferred4;
    PL.deferred_count = &hdr->ndeferred4;
    PL.next_cell = &hdr->coop_next;
    char *arena = base + L.coop;
    if (launch_cells_coop(PL, false, arena, L.coop_slices, L.n_max, n, st) != cudaSuccess)
        return VOR_E_CUDA;
    CellParams PG = PL;
    PG.cell_list = deferred4;
    PG.list_count = &hdr->ndeferred4;
    PG.deferred = nullptr;
    PG.deferred_count = nullptr;
    PG.next_cell = &hdr->coop_next2;
    if (launch_cells_coop(PG, true, arena, L.coop_slices, L.n_max, n, st) != cudaSuccess)
        return VOR_E_CUDA;
    launched += 3;
    mark(5, st);

    launched += scan<long long>(ecount, n, nullptr, (long long *)out->cell_ptr, partial,
                                (long long *)out->totals, hdr, st);
    launched += scan<long long>(dcount, n, nullptr, del_ptr, partial, (long long *)out->totals + 1, hdr, st);
    CompactParams Q;
    Q.sites = sites; Q.n = n; Q.sets = sets; Q.sset = sset;
    Q.ecount = ecount; Q.dcount = dcount; Q.loc = loc; Q.slot = slot; Q.spill = spill;
    Q.cell_ptr = (const long long *)out->cell_ptr; Q.del_ptr = del_ptr;
    Q.edge_label = out->edge_label; Q.vx = out->vx; Q.vy = out->vy; Q.del_edge = out->del_edge;
    Q.edge_cap = out->edge_cap; Q.del_cap = out->del_cap; Q.hdr = hdr;
    Q.share = o->share_vertices ? 1 : 0;
    k_compact<<<(n + COMPACT_T - 1) / COMPACT_T, COMPACT_T, 0, st>>>(Q);   // a warp per 32 cells
    launched += 1;                    // compaction
    if (Q.share) {
        k_share_vertices<<<(n + 255) / 256, 256, 0, st>>>(Q);
        launched += 1;
    }
    if (A.del_set_ptr) {
        k_set_del_ptr<<<(L.n_sets + 1 + T - 1) / T, T, 0, st>>>(sets, L.n_sets, n, del_ptr,
                                                                 A.del_set_ptr, hdr);
        launched++;
    }
    if (cudaGetLastError() != cudaSuccess) return VOR_E_CUDA;
    mark(N_STAGES, st);
    if (g_timing) g_ev_recorded = true;
    return VOR_OK;
}

cudaError_t resident_grid(const void *kern, int threads, int smem, int &grid) {
    struct Entry { const void *kern; int dev, threads, smem, grid; };
    static std::mutex mu;
    static Entry table[256];
    static int used = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < used; i++) {
        const Entry &t = table[i];
        if (t.kern == kern && t.dev == dev && t.threads == threads && t.smem == smem) {
            grid = t.grid;
            return cudaSuccess;
        }
    }
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    grid = sms * (per_sm < 1 ? 1 : per_sm);
    if (used < 256) table[used++] = Entry{kern, dev, threads, smem, grid};
    return cudaSuccess;
}

static int map_err(unsigned e) {
    if (e & ERRB_ARG) return VOR_E_INVALID_ARG;
    if (e & ERRB_OUTSIDE) return VOR_E_SITE_OUTSIDE;
    if (e & ERRB_DUPLICATE) return VOR_E_DUPLICATE;
    if (e & ERRB_INTERNAL) return VOR_E_INTERNAL;
    if (e & ERRB_CAPACITY) return VOR_E_CAPACITY;
    if (e & ERRB_SPILL) return VOR_E_OOM;
    return VOR_OK;
}

int status_of_error_bits(unsigned e) { return map_err(e); }

}  // namespace vor

using namespace vor;

extern "C" {

void vor_opts_default(vor_opts *o) {
    if (!o) return;
    o->bucket_side = 0;
    o->lanes_per_cell = 0;
    o->target = 0;
    o->exact_only = 0;
    o->check_duplicates = 1;
    o->collect_stats = 0;
    o->bucket_load_pct = 0;
    o->share_vertices = 0;
    o->fine_split = 0;
    o->block_threads = 0;
}

int64_t vor_edge_capacity(int64_t n) { return n < 1 ? 0 : 10 * n + 4; }
int64_t vor_delaunay_capacity(int64_t n) { return n < 3 ? 1 : 3 * n; }

int64_t vor_workspace_bytes(int64_t n, vor_box box, const vor_opts *opts) {
    Layout L;
    if (!resolve(nullptr, nullptr, 1, n, box, opts, L)) return -1;
    return (int64_t)L.total;
}

static bool out_ok(const vor_out *out) {
    return out && out->cell_ptr && out->edge_label && out->vx && out->vy && out->del_edge && out->totals;
}

int vor_build_async(const vor_site *d_sites, int64_t n, vor_box box, const vor_opts *opts,
                    void *d_workspace, int64_t ws_bytes, const vor_out *out, void *stream) {
    if (!d_sites || !d_workspace || !out_ok(out)) return VOR_E_INVALID_ARG;
    if (box.w < 2 || box.h < 2 || box.w > (1 << 20) || box.h > (1 << 20)) return VOR_E_BOX_TOO_LARGE;
    Layout L;
    if (!resolve(nullptr, nullptr, 1, n, box, opts, L)) return VOR_E_INVALID_ARG;
    if (ws_bytes < (int64_t)L.total || ((uintptr_t)d_workspace & 255)) return VOR_E_OOM;
    if (out->edge_cap < 1 || out->del_cap < 1) return VOR_E_OOM;
    BatchArgs A = {(const int2 *)d_sites, nullptr, nullptr, n, box, nullptr};
    return launch_build(A, opts, d_workspace, L, out, (cudaStream_t)stream);
}

int64_t vor_batch_edge_capacity(int64_t n_total, int32_t n_sets) {
    return n_total < 0 || n_sets < 1 ? 0 : 10 * n_total + 4 * (int64_t)n_sets;
}

int64_t vor_batch_delaunay_capacity(int64_t n_total, int32_t n_sets) {
    return n_total < 0 || n_sets < 1 ? 0 : 3 * n_total + n_sets;
}

int64_t vor_batch_workspace_bytes(const int64_t *h_set_ptr, int32_t n_sets, const vor_box *h_boxes,
                                  const vor_opts *opts) {
    if (!h_set_ptr || !h_boxes) return -1;
    Layout L;
    if (!resolve(h_set_ptr, h_boxes, n_sets, 0, vor_box{0, 0}, opts, L)) return -1;
    return (int64_t)L.total;
}

int vor_build_batch_async(const vor_site *d_sites, const int64_t *d_set_ptr,
                          const int64_t *h_set_ptr, int32_t n_sets, const vor_box *d_boxes,
                          const vor_box *h_boxes, const vor_opts *opts, void *d_workspace,
                          int64_t ws_bytes, const vor_out *out, int64_t *d_del_set_ptr,
                          void *stream) {
    if (!d_set_ptr || !h_set_ptr || !d_boxes || !h_boxes || !d_workspace || !out_ok(out) ||
        !d_del_set_ptr || n_sets < 1)
        return VOR_E_INVALID_ARG;
    for (int j = 0; j < n_sets; j++) {
        const vor_box b = h_boxes[j];
        if (b.w < 2 || b.h < 2 || b.w > (1 << 20) || b.h > (1 << 20)) return VOR_E_BOX_TOO_LARGE;
    }
    Layout L;
    if (!resolve(h_set_ptr, h_boxes, n_sets, 0, vor_box{0, 0}, opts, L)) return VOR_E_INVALID_ARG;
    if (L.n > 0 && !d_sites) return VOR_E_INVALID_ARG;
    if (ws_bytes < (int64_t)L.total || ((uintptr_t)d_workspace & 255)) return VOR_E_OOM;
    if (out->edge_cap < 1 || out->del_cap < 1) return VOR_E_OOM;
    BatchArgs A = {(const int2 *)d_sites, (const long long *)d_set_ptr, d_boxes, 0, vor_box{0, 0},
                   (long long *)d_del_set_ptr};
    return launch_build(A, opts, d_workspace, L, out, (cudaStream_t)stream);
}

int vor_status(const void *d_workspace, void *stream, vor_stats *stats) {
    if (!d_workspace) return VOR_E_INVALID_ARG;
    WsHeader h;
    // ordered on the caller's stream only (no device-wide synchronisation)
    const cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, d_workspace, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return VOR_E_CUDA;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->rays = h.stats[STAT_RAYS];
        stats->vertex_tests = h.stats[STAT_VTESTS];
        stats->evals = h.stats[STAT_EVALS];
        stats->exact_rays = h.stats[STAT_EXACT];
        stats->annulus_sites = h.stats[STAT_ANNULUS];
        stats->reruns = h.stats[STAT_RERUNS];
        stats->deferred = h.stats[STAT_DEFERRED];
        stats->candidates = h.stats[STAT_CANDIDATES];
        stats->max_edges = h.stats[STAT_MAXE];
        stats->widenings = h.stats[STAT_WIDEN];
        stats->evals_first_pass = h.stats[STAT_EVALS1];
        stats->rays_first_pass = h.stats[STAT_RAYS1];
        stats->evals_second_pass = h.stats[STAT_EVALS2];
        const int third = h.flower_passes ? h.ndeferred2 : 0;
        const int medium = h.flower_passes ? h.fcount[h.flower_passes - 1] : h.ndeferred2;
        stats->third_pass_cells = (uint64_t)(third > 0 ? third : 0);
        stats->medium_cells = (uint64_t)(medium > 0 ? medium : 0);
        stats->large_cells = (uint64_t)(h.ndeferred3 > 0 ? h.ndeferred3 : 0);
        stats->global_cells = (uint64_t)(h.ndeferred4 > 0 ? h.ndeferred4 : 0);
        stats->divided_buckets = (uint64_t)(h.fine_count > 0 ? h.fine_count : 0);
    }
    return map_err(h.err);
}

int vor_build(const vor_site *d_sites, int64_t n, vor_box box, const vor_opts *opts, void *stream,
              vor_out *out, int64_t *n_edges, int64_t *n_del, vor_stats *stats) {
    if (!out) return VOR_E_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    const int64_t ws = vor_workspace_bytes(n, box, opts);
    if (ws < 0) return VOR_E_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    void *w = nullptr;
    out->edge_cap = vor_edge_capacity(n);
    out->del_cap = vor_delaunay_capacity(n);
    if (cudaMalloc(&w, (size_t)ws) != cudaSuccess ||
        cudaMalloc((void **)&out->cell_ptr, (size_t)(n + 1) * 8) != cudaSuccess ||
        cudaMalloc((void **)&out->edge_label, (size_t)out->edge_cap * 4) != cudaSuccess ||
        cudaMalloc((void **)&out->vx, (size_t)out->edge_cap * 8) != cudaSuccess ||
        cudaMalloc((void **)&out->vy, (size_t)out->edge_cap * 8) != cudaSuccess ||
        cudaMalloc((void **)&out->del_edge, (size_t)out->del_cap * 8) != cudaSuccess ||
        cudaMalloc((void **)&out->totals, 16) != cudaSuccess) {
        cudaFree(w);
        vor_free_result(out, stream);
        return VOR_E_OOM;
    }
    int rc = vor_build_async(d_sites, n, box, opts, w, ws, out, stream);
    if (rc == VOR_OK) rc = vor_status(w, stream, stats);
    if (rc == VOR_OK) {
        int64_t t[2];
        if (cudaMemcpyAsync(t, out->totals, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = VOR_E_CUDA;
        if (n_edges) *n_edges = t[0];
        if (n_del) *n_del = t[1];
    }
    cudaStreamSynchronize(st);
    cudaFree(w);
    if (rc != VOR_OK) vor_free_result(out, stream);
    return rc;
}

int vor_free_result(vor_out *out, void *stream) {
    if (!out) return VOR_E_INVALID_ARG;
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(out->cell_ptr);
    cudaFree(out->edge_label);
    cudaFree(out->vx);
    cudaFree(out->vy);
    cudaFree(out->del_edge);
    cudaFree(out->totals);
    memset(out, 0, sizeof(*out));
    return VOR_OK;
}

int64_t vor_host_scratch_bytes(int64_t n) {
    if (n < 1) return -1;
    size_t at = 0;
    at = align256(at + (size_t)n * 8);                          // sites
    at = align256(at + (size_t)(n + 1) * 8);                    // cell_ptr
    at = align256(at + (size_t)vor_edge_capacity(n) * 4);       // labels
    at = align256(at + (size_t)vor_edge_capacity(n) * 8);       // vx
    at = align256(at + (size_t)vor_edge_capacity(n) * 8);       // vy
    at = align256(at + (size_t)vor_delaunay_capacity(n) * 8);   // del
    at = align256(at + 16);                                     // totals
    return (int64_t)at;
}

int vor_build_host(const vor_site *h_sites, int64_t n, vor_box box, const vor_opts *opts,
                   void *d_workspace, int64_t ws_bytes, void *d_scratch, int64_t scratch_bytes,
                   int64_t *h_cell_ptr, int32_t *h_edge_label, double *h_vx, double *h_vy,
                   int32_t *h_del_edge, int64_t edge_cap, int64_t del_cap, int64_t *n_edges,
                   int64_t *n_del, void *stream) {
    if (!h_sites || !d_scratch || !h_cell_ptr || !h_edge_label || !h_vx || !h_vy || !h_del_edge)
        return VOR_E_INVALID_ARG;
    if (n < 1) return VOR_E_INVALID_ARG;
    if (scratch_bytes < vor_host_scratch_bytes(n) || ((uintptr_t)d_scratch & 255)) return VOR_E_OOM;
    cudaStream_t st = (cudaStream_t)stream;
    char *b = (char *)d_scratch;
    size_t at = 0;
    vor_site *d_sites = (vor_site *)(b + at); at = align256(at + (size_t)n * 8);
    vor_out o;
    o.cell_ptr = (int64_t *)(b + at); at = align256(at + (size_t)(n + 1) * 8);
    o.edge_label = (int32_t *)(b + at); at = align256(at + (size_t)vor_edge_capacity(n) * 4);
    o.vx = (double *)(b + at); at = align256(at + (size_t)vor_edge_capacity(n) * 8);
    o.vy = (double *)(b + at); at = align256(at + (size_t)vor_edge_capacity(n) * 8);
    o.del_edge = (int32_t *)(b + at); at = align256(at + (size_t)vor_delaunay_capacity(n) * 8);
    o.totals = (int64_t *)(b + at);
    o.edge_cap = vor_edge_capacity(n);
    o.del_cap = vor_delaunay_capacity(n);
    if (cudaMemcpyAsync(d_sites, h_sites, (size_t)n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return VOR_E_CUDA;
    int rc = vor_build_async(d_sites, n, box, opts, d_workspace, ws_bytes, &o, stream);
    if (rc != VOR_OK) return rc;
    int64_t t[2] = {0, 0};
    if (cudaMemcpyAsync(t, o.totals, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess) return VOR_E_CUDA;
    rc = vor_status(d_workspace, stream, nullptr);
    if (rc != VOR_OK) return rc;
    if (t[0] > edge_cap || t[1] > del_cap) return VOR_E_OOM;
    if (cudaMemcpyAsync(h_cell_ptr, o.cell_ptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_edge_label, o.edge_label, (size_t)t[0] * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_vx, o.vx, (size_t)t[0] * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_vy, o.vy, (size_t)t[0] * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_del_edge, o.del_edge, (size_t)t[1] * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return VOR_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return VOR_E_CUDA;
    if (n_edges) *n_edges = t[0];
    if (n_del) *n_del = t[1];
    return VOR_OK;
}

int vor_stage_timing(int enable) {
    if (enable && !g_ev_made) {
        for (int i = 0; i <= N_STAGES; i++)
            if (cudaEventCreate(&g_ev[i]) != cudaSuccess) return VOR_E_CUDA;
        g_ev_made = true;
    }
    g_timing = enable != 0;
    g_ev_recorded = false;
    return VOR_OK;
}

int vor_stage_ms(float *ms, int max_stages) {
    if (!ms || max_stages < 1) return VOR_E_INVALID_ARG;
    if (!g_ev_made || !g_ev_recorded) return VOR_E_INVALID_ARG;
    if (cudaEventSynchronize(g_ev[N_STAGES]) != cudaSuccess) return VOR_E_CUDA;
    int k = 0;
    for (int i = 0; i < N_STAGES && k < max_stages; i++, k++)
        if (cudaEventElapsedTime(&ms[i], g_ev[i], g_ev[i + 1]) != cudaSuccess) return VOR_E_CUDA;
    return k;
}

int64_t vor_kernel_launches(void) { return (int64_t)g_launches.load(); }

int vor_vertex_quotients(const int64_t *d_num, const uint64_t *d_den, int64_t n, double *d_out,
                         void *stream) {
    if (n < 0 || (n > 0 && (!d_num || !d_den || !d_out))) return VOR_E_INVALID_ARG;
    if (n == 0) return VOR_OK;
    const int T = 256;
    k_vertex_quotients<<<(unsigned)((n + T - 1) / T), T, 0, (cudaStream_t)stream>>>(
        (const long long *)d_num, (const unsigned long long *)d_den, (long long)n, d_out);
    g_launches++;
    return cudaGetLastError() == cudaSuccess ? VOR_OK : VOR_E_CUDA;
}

int32_t vor_autotune_grid(vor_opts *cand, int32_t max) {
    // rays per warp and block shape (one thread per cell with blocks of 32,
    // 64 or 128 threads, or eight lanes per cell in blocks of 16 groups) x
    // first-disc size x bucket load (the grid-bucket size)
    static const int lanes[] = {1, 1, 1, 8};
    static const int block[] = {32, 64, 128, 0};
    static const int target[] = {16, 20, 24};
    static const int load[] = {200, 400, 600};
    int k = 0;
    for (int a = 0; a < 4; a++)
        for (int b : target)
            for (int c : load) {
                if (k < max && cand) {
                    vor_opts_default(&cand[k]);
                    cand[k].lanes_per_cell = lanes[a];
                    cand[k].block_threads = block[a];
                    cand[k].target = b;
                    cand[k].bucket_load_pct = c;
                }
                k++;
            }
    return k < max ? k : max;
}

int vor_autotune_batch(const vor_site *d_sites, const int64_t *d_set_ptr, const int64_t *h_set_ptr,
                       int32_t n_sets, const vor_box *d_boxes, const vor_box *h_boxes,
                       const vor_opts *candidates, int32_t n_candidates, int32_t reps,
                       void *d_workspace, int64_t ws_bytes, const vor_out *out,
                       int64_t *d_del_set_ptr, void *stream, int32_t *best, float *ms) {
    if (!candidates || n_candidates < 1 || reps < 1 || !best || !ms) return VOR_E_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return VOR_E_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return VOR_E_CUDA;
    }
    int rc_all = VOR_OK;
    *best = -1;
    for (int c = 0; c < n_candidates; c++) {
        ms[c] = INFINITY;
        auto run = [&]() {
            return vor_build_batch_async(d_sites, d_set_ptr, h_set_ptr, n_sets, d_boxes, h_boxes,
                                         &candidates[c], d_workspace, ws_bytes, out, d_del_set_ptr,
                                         stream);
        };
        int rc = run();
        if (rc == VOR_E_INVALID_ARG || rc == VOR_E_BOX_TOO_LARGE) { rc_all = rc; break; }
        if (rc != VOR_OK || vor_status(d_workspace, stream, nullptr) != VOR_OK) continue;
        float total = 0.f;
        bool ok = true;
        for (int r = 0; r < reps && ok; r++) {
            float t = 0.f;
            ok = cudaEventRecord(e0, st) == cudaSuccess && run() == VOR_OK &&
                 cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&t, e0, e1) == cudaSuccess &&
                 vor_status(d_workspace, stream, nullptr) == VOR_OK;
            total += t;
        }
        if (!ok) continue;
        ms[c] = total / reps;
        if (*best < 0 || ms[c] < ms[*best]) *best = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc_all;
}

const char *vor_strerror(int code) {
    switch (code) {
    case VOR_OK: return "ok";
    case VOR_E_INVALID_ARG: return "invalid argument (or set offsets that differ between host and device)";
    case VOR_E_SITE_OUTSIDE: return "a site lies on or outside the boundary of the box";
    case VOR_E_DUPLICATE: return "two sites are equal";
    case VOR_E_BOX_TOO_LARGE: return "box side outside [2, 2^20]";
    case VOR_E_OOM: return "workspace or output buffer too small, or out of memory";
    case VOR_E_CAPACITY: return "a cell exceeded a capacity of the build";
    case VOR_E_CUDA: return "CUDA runtime error";
    case VOR_E_INTERNAL: return "internal consistency check failed";
    case VOR_E_SCRATCH_LIMIT: return "n needs more workspace than the static scratch of vor_build_noalloc";
    case VOR_E_SERVER_FULL: return "request larger than a server budget, or no room before the timeout";
    case VOR_E_TIMEOUT: return "the request is still pending";
    case VOR_E_CANCELLED: return "the request was cancelled";
    case VOR_PENDING: return "pending";
    default: return "unknown error";
    }
}

}  // extern "C"
