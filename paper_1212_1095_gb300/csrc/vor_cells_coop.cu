// vor_cells_coop.cu -- launchers of the cooperative large-cell tier (one
// block per cell; see vor_cells_coop.cuh).
#include "vor_cells_coop.cuh"

namespace vor {

long long coop_slice_bytes(long long nmax) {
    long long cap, qcap, ecap;
    return coop_slice_caps(nmax, cap, qcap, ecap);
}

cudaError_t launch_cells_coop(const CellParams &P, bool global_mode, char *arena, int slices,
                              long long nmax, int max_cells, cudaStream_t st) {
    long long cap, qcap, ecap;
    const long long slice = coop_slice_caps(nmax, cap, qcap, ecap);
    if (!global_mode) {
        auto kern = coop_cells_kernel<false>;
        const int smem = (int)sizeof(CoopSmem);
        int grid = 0;
        cudaError_t e = resident_grid((const void *)kern, CO_T, smem, grid);
        if (e != cudaSuccess) return e;
        if (max_cells < grid) grid = max_cells > 0 ? max_cells : 1;
        kern<<<grid, CO_T, smem, st>>>(P, arena, slice, cap, qcap, ecap);
    } else {
        int grid = slices;
        if (max_cells < grid) grid = max_cells > 0 ? max_cells : 1;
        if (grid < 1) grid = 1;
        coop_cells_kernel<true><<<grid, CO_T, 0, st>>>(P, arena, slice, cap, qcap, ecap);
    }
    return cudaGetLastError();
}

}  // namespace vor
