// vor_internal.h -- shared declarations of the library's translation units.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "vor.h"

namespace vor {

// error bits set on the device (one 32-bit word at the head of the workspace)
enum : unsigned {
    ERRB_OUTSIDE = 1u,
    ERRB_DUPLICATE = 2u,
    ERRB_CAPACITY = 4u,
    ERRB_INTERNAL = 8u,
    ERRB_SPILL = 16u,
    ERRB_ARG = 32u,          // the device copy of the set offsets disagrees with the host's
};

// per-build counters (vor_stats order)
enum {
    STAT_RAYS = 0, STAT_VTESTS, STAT_EVALS, STAT_EXACT, STAT_ANNULUS, STAT_RERUNS,
    STAT_DEFERRED, STAT_CANDIDATES, STAT_MAXE, STAT_WIDEN, STAT_EVALS1, STAT_RAYS1, STAT_EVALS2, STAT_N = 16
};

// Thread-per-cell passes over the flower of the polygon an earlier pass left
// (batches).  Measured on the 4,096-set batch: three passes leave 252 k cells
// to the warp tier, two leave 284 k, but the third pass costs more than the
// warp tier spends on the difference (batch 110.1 ms with three, 108.8 ms
// with two, 111.8 ms with one).
constexpr int FLOWER_PASSES = 2;

// Workspace header (first 256 bytes of the workspace).
struct WsHeader {
    unsigned err;
    int spill_top;
    int ndeferred;          // cells handed from the first to the second pass
    int ndeferred2;         // cells handed to the warp-per-cell pass
    unsigned long long stats[STAT_N];
    int large_next;         // next cell of the medium-cell pass (dynamic schedule)
    int m_total;            // buckets over all sets (set by the grid choice)
    int ndeferred3;         // cells handed from the medium tier to the block-per-cell tier
    int coop_next;          // next cell of the block-per-cell tier (shared-memory mode)
    int pass_next[2];       // next list entry of the first two thread-per-cell passes
    int ndeferred4;         // cells handed on to the global-memory mode of that tier
    int coop_next2;         // next cell of the global-memory mode
    int flower_passes;      // flower passes that ran (set by a memset; 0: none)
    int fcount[FLOWER_PASSES];  // cells each flower pass hands on
    int fnext[FLOWER_PASSES];   // next list entry of each flower pass
    int fine_top;           // sub-bucket starts handed out (adaptive buckets)
    int fine_count;         // buckets divided into sub-buckets
    long long pad[4];
};
static_assert(sizeof(WsHeader) <= 256, "header");

// Cells a first-pass group stores in fixed slots (larger ones spill).
constexpr int SLOT_CAP = 16;


// One point set of a batch (a single build is a batch of one set).
struct SetMeta {
    long long site_base;    // index of the set's first site in the batch
    long long bucket_base;  // first bucket of the set's grid in the batch's bucket array
    long long coarse_base;  // first cell of the set's density-probe grid
    int n, W, H;            // sites, box [0,W] x [0,H]
    int s, m1, m2;          // bucket side and grid (chosen on the device)
    int G;                  // side of the density-probe grid
    int s_min, s_max, s_fixed, m_max;
    int load_pct;           // sites per bucket the automatic side aims at (hundredths)
    int pad0;
    double acc;             // probe: sum over the set's sites of log2(coarse count)
};

// Sizes of a set's grids, computed identically on the host (workspace
// sizing) and on the device (planning kernel).
struct SetPlan { int s_min, s_max, m_max, G; };

__host__ __device__ inline long long isqrt_floor_ll(long long v) {
    if (v <= 0) return 0;
    long long r = (long long)sqrt((double)v);
    while (r * r > v) r--;
    while ((r + 1) * (r + 1) <= v) r++;
    return r;
}

// bucket side between s_min (at most max(4n, 4096) buckets) and s_max (the
// side of a bucket holding 8 sites at the average density), or fixed by the
// caller
__host__ __device__ inline bool plan_set(long long n, int W, int H, int s_fixed, SetPlan &pl) {
    if (n < 1 || W < 2 || H < 2 || W > (1 << 20) || H > (1 << 20)) return false;
    if (s_fixed < 0 || s_fixed > (1 << 20)) return false;
    const long long area = (long long)W * H;
    const long long mcap = n * 4 > 4096 ? n * 4 : 4096;
    long long smin = isqrt_floor_ll(area / mcap);
    while (smin * smin * mcap < area) smin++;
    long long smax = isqrt_floor_ll(8 * area / n);
    if (smax < smin) smax = smin;
    if (smax > (1 << 20)) smax = 1 << 20;
    if (smin > (1 << 20)) smin = 1 << 20;
    pl.s_min = (int)smin;
    pl.s_max = (int)smax;
    const long long sm = s_fixed > 0 ? s_fixed : smin;
    const long long m1 = (W + sm - 1) / sm, m2 = (H + sm - 1) / sm;
    if (m1 * m2 > (1ll << 28)) return false;
    pl.m_max = (int)(m1 * m2);
    long long g = isqrt_floor_ll(n) / 8;
    pl.G = (int)(g < 16 ? 16 : (g > 1024 ? 1024 : g));
    return true;
}

// Adaptive buckets (two levels).  A bucket of the uniform grid holding at
// least the split count of sites is divided into F x F sub-buckets, F = 2^k
// the smallest power of two (2 <= F <= 16) with 3 F^2 >= its count, about
// three sites per sub-bucket; its sites are stored by sub-bucket, sub-rows
// in order, so the bucket, and every bucket row, stays one range of sorted
// positions.  A site at offset (lx, ly) from its bucket's corner lies in
// sub-bucket (ly F / s, lx F / s).  fdesc[b] is the offset of bucket b's
// F^2 + 1 sub-bucket starts (relative to the bucket's first position) in the
// pool, or -1 for a bucket that is not divided.
__host__ __device__ inline int fine_log2(int count) {
    int k = 1;
    while (k < 4 && 3 * (1 << (2 * k)) < count) k++;
    return k;
}
// pool entries for n sites: a divided bucket of c >= 4 sites takes F^2 + 1
// of them, at most 1.34 c (the largest ratio, 257 / 193, at c = 193)
__host__ __device__ inline long long fine_pool_cap(long long n) { return n + n / 2 + 64; }

// The grid of one cell's set, for the kernels.
struct CellGrid {
    const int *bs;          // the set's bucket starts
    const int *fd;          // the set's sub-bucket descriptors (null: no sub-buckets)
    const int *fp;          // sub-bucket start pool
    int s, m1, m2, W, H;
    int site_base;
};

struct CellParams {
    const int2 *sites;      // original order (device)
    const int2 *sxy;        // sites sorted by set, then bucket
    const int *sid;         // original (batch) index of sorted position
    const int *bstart;      // bucket CSR over all sets
    const SetMeta *sets;    // per-set metadata
    const int *sset;        // set of each site (the same in sorted and original
                            // order, as the sets stay contiguous); null: one set
    int n;                  // sites in the batch
    int target;             // sites wanted in the first candidate disc
    int exact_only;
    int collect_stats;
    int *ecount;            // e_k per original index
    int *dcount;            // Delaunay edges (k, j > k) per original index
    int *loc;               // -1: fixed slot, else offset into spill
    int *slot;              // n * SLOT_CAP labels
    int *spill;             // spill area
    int spill_cap;
    const int *cell_list;   // cells (sorted positions) to process; null: all
    const int *list_count;  // device count of cell_list entries
    int n_list;             // host upper bound of the list length (grid sizing)
    int *deferred;          // cells handed to the next pass
    int *deferred_count;    // device counter of that list
    int *next_cell;         // dynamic schedule: next list entry to take (null: stride)
    float *need_out;        // first pass: per deferred cell (by sorted position) the
                            // squared disc radius its polygon needs, 0 when unknown
    const float *need_in;   // second pass: the same, read by its gather
    int store_poly;         // thread-per-cell passes: a cell whose polygon the certificate
                            // cannot accept leaves its lines in its slot (ecount = -e)
    int seed_poly;          // warp tier: such a polygon's sites join the first candidates
    const int *coarse_sat;  // summed-area tables of the sets' coarse occupancy grids
    const int *fdesc;       // sub-bucket descriptors over all sets (null: none)
    const int *fpool;       // sub-bucket starts
    WsHeader *hdr;
};

__device__ __forceinline__ const SetMeta &set_of(const SetMeta *sets, const int *sset, int i) {
    return sets[sset ? sset[i] : 0];
}

__device__ __forceinline__ CellGrid cell_grid(const CellParams &P, int i) {
    const SetMeta &M = set_of(P.sets, P.sset, i);
    CellGrid g;
    g.bs = P.bstart + M.bucket_base;
    g.fd = P.fdesc ? P.fdesc + M.bucket_base : nullptr;
    g.fp = P.fpool;
    g.s = M.s; g.m1 = M.m1; g.m2 = M.m2; g.W = M.W; g.H = M.H;
    g.site_base = (int)M.site_base;
    return g;
}

// Sites of a set in the coarse cells that meet the rectangle [x0, x1] x
// [y0, y1] (clamped to the set's box), from its summed-area table: at least
// the sites inside the rectangle.
__device__ __forceinline__ int coarse_sites(const int *sat, const SetMeta &M, int x0, int y0, int x1,
                                            int y1) {
    const int G = M.G;
    auto cell = [](int v, int lim, int G) {
        return (int)((unsigned)min(max(v, 0), lim - 1) * (unsigned)G / (unsigned)lim);
    };
    const int a0 = cell(x0, M.W, G), a1 = cell(x1, M.W, G), b0 = cell(y0, M.H, G), b1 = cell(y1, M.H, G);
    const int *S = sat + M.coarse_base;
    auto at = [&](int cx, int cy) { return (cx < 0 || cy < 0) ? 0 : S[cy * G + cx]; };
    return at(a1, b1) - at(a0 - 1, b1) - at(a1, b0 - 1) + at(a0 - 1, b0 - 1);
}

// Resident CTAs of a kernel on the current device (all SMs x CTAs per SM),
// after raising its dynamic shared memory limit to smem.  Computed once per
// device and kernel; later calls make no CUDA call, so builds can be
// captured into a CUDA graph after a first (warm-up) build on the device.
cudaError_t resident_grid(const void *kern, int threads, int smem, int &grid);

// VOR_* status of the error bits of a workspace header (vor_lib.cu)
int status_of_error_bits(unsigned e);

// Launchers (vor_cells.cu)
cudaError_t launch_cells_fast(const CellParams &P, int lanes, cudaStream_t st);
// one thread per cell; pass 1 over all cells, pass 2 over the list
// P.cell_list: first the candidate gather, then the persistent projector
cudaError_t launch_gather_pass(const CellParams &P, int pass, int *gcount, long long *grho2,
                               float2 *gtab, int *glab, cudaStream_t st);
cudaError_t launch_cells_pass(const CellParams &P, int pass, int *gcount, long long *grho2,
                              float2 *gtab, int *glab, int block, cudaStream_t st);
int pass_gather_width();
long long gather_rows(long long n);   // list rows: n rounded up to whole tiles of 32
// one warp per cell over P.cell_list, cells taken from *P.next_cell, with
// the medium capacities (defers to P.deferred)
cudaError_t launch_cells_medium(const CellParams &P, int max_cells, long long n_max, bool single,
                                cudaStream_t st);
int cells_fast_max_smem();
// one block per cell over P.cell_list (vor_cells_coop.cu): shared-memory
// mode (defers to P.deferred) or global-memory mode (slices of the arena,
// each for sets of at most nmax sites)
cudaError_t launch_cells_coop(const CellParams &P, bool global_mode, char *arena, int slices,
                              long long nmax, int max_cells, cudaStream_t st);
long long coop_slice_bytes(long long nmax);

}  // namespace vor
