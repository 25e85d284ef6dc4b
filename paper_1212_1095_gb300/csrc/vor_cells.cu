// vor_cells.cu -- launchers of the projector kernel: lane-count dispatch of
// the multi-lane first pass and the medium tier (one warp per deferred cell).
#include "vor_cells.cuh"

namespace vor {

int cells_fast_max_smem() { return (int)(F_GROUPS * sizeof(FastSmem)); }

cudaError_t launch_cells_fast(const CellParams &P, int lanes, cudaStream_t st) {
    switch (lanes) {
    case 2: return launch_fast_g<2>(P, st);
    case 4: return launch_fast_g<4>(P, st);
    case 8: return launch_fast_g<8>(P, st);
    case 16: return launch_fast_g<16>(P, st);
    case 32: return launch_fast_g<32>(P, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int CMAX, int SMAX, int EMAX, int RMAX, bool ROUTE, bool PAR>
static cudaError_t launch_tier(const CellParams &P, int max_cells, cudaStream_t st) {
    auto kern = cells_kernel<32, CMAX, SMAX, EMAX, RMAX, true, ROUTE, PAR>;
    const int smem = group_smem_bytes<CMAX, SMAX, EMAX>(PAR);
    int grid = 0;
    cudaError_t e = resident_grid((const void *)kern, 32, smem, grid);
    if (e != cudaSuccess) return e;
    if (max_cells < grid) grid = max_cells > 0 ? max_cells : 1;
    kern<<<grid, 32, smem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_cells_medium(const CellParams &P, int max_cells, long long n_max, bool single,
                                cudaStream_t st) {
    // the routing by site count only where a set is large enough for it;
    // the parallel subedges for a single diagram (run_projector)
    const bool route = n_max > 16LL * M_DEFER_SITES;
    if (single)
        return route ? launch_tier<M_CMAX, M_SMAX, M_EMAX, M_RMAX, true, true>(P, max_cells, st)
                     : launch_tier<M_CMAX, M_SMAX, M_EMAX, M_RMAX, false, true>(P, max_cells, st);
    return route ? launch_tier<M_CMAX, M_SMAX, M_EMAX, M_RMAX, true, false>(P, max_cells, st)
                 : launch_tier<M_CMAX, M_SMAX, M_EMAX, M_RMAX, false, false>(P, max_cells, st);
}

}  // namespace vor
