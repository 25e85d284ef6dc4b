// vor_internal.h -- shared declarations of the library's translation units.
#pragma once

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
};

// per-build counters (vor_stats order)
enum {
    STAT_RAYS = 0, STAT_VTESTS, STAT_EVALS, STAT_EXACT, STAT_ANNULUS, STAT_RERUNS,
    STAT_DEFERRED, STAT_CANDIDATES, STAT_MAXE, STAT_WIDEN, STAT_N = 16
};

// Workspace header (first 256 bytes of the workspace).
struct WsHeader {
    unsigned err;
    int spill_top;
    int ndeferred;          // cells handed from the first to the second pass
    int ndeferred2;         // cells handed to the warp-per-cell pass
    unsigned long long stats[STAT_N];
    int s, m1, m2, m;       // bucket side and grid (chosen on the device)
    long long pad[10];
};
static_assert(sizeof(WsHeader) <= 256, "header");

// Cells a first-pass group stores in fixed slots (larger ones spill).
constexpr int SLOT_CAP = 16;

struct CellParams {
    const int2 *sites;      // original order (device)
    const int2 *sxy;        // sites sorted by bucket
    const int *sid;         // original index of sorted position
    const int *bstart;      // bucket CSR (m1*m2 + 1)
    int n, W, H;
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
    WsHeader *hdr;
};

// Launchers (vor_cells.cu)
cudaError_t launch_cells_fast(const CellParams &P, int lanes, cudaStream_t st);
// one thread per cell; pass 1 over all cells, pass 2 over the list P.cell_list
cudaError_t launch_cells_pass(const CellParams &P, int pass, int *gcount, long long *grho2, int *gpos,
                              cudaStream_t st);
int pass_gather_width();
cudaError_t launch_cells_large(const CellParams &P, int max_cells, cudaStream_t st);
int cells_fast_max_smem();
int cells_large_capacity();

}  // namespace vor
