// vor_cells_t1.cu -- launchers of the one-thread-per-cell projector passes.
#include "vor_cells_persist.cuh"

namespace vor {

template <int CMAX>
static cudaError_t launch_pass(const CellParams &P, const GatherOut &G, float target, cudaStream_t st) {
    const int total_max = P.cell_list ? P.n_list : P.n;
    gather_kernel<<<(total_max + 255) / 256, 256, 0, st>>>(P, G, target);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto kern = cells_persist_kernel<P_NT, CMAX, P_SMAX, P_EMAX, P_RMAX>;
    const int smem = P_NT * CMAX * (int)sizeof(float4);
    int resident = 0;
    e = resident_grid((const void *)kern, P_NT, smem, resident);
    if (e != cudaSuccess) return e;
    long long want = ((long long)total_max + P_NT - 1) / P_NT;
    long long grid = resident;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, P_NT, smem, st>>>(P, G);
    return cudaGetLastError();
}

cudaError_t launch_cells_pass(const CellParams &P, int pass, int *gcount, long long *grho2, int *gpos,
                              cudaStream_t st) {
    // both passes share one position buffer of n * (P1_CMAX - 4) entries; the
    // second pass lists fewer cells (the deferred ones) with more sites each
    const long long entries = (long long)P.n * (P1_CMAX - 4);
    if (pass == 1) {
        GatherOut G{gcount, grho2, gpos, P1_CMAX - 4, P.n};
        return launch_pass<P1_CMAX>(P, G, (float)P.target, st);
    }
    GatherOut G{gcount, grho2, gpos, P2_CMAX - 4, (int)(entries / (P2_CMAX - 4))};
    return launch_pass<P2_CMAX>(P, G, 2.2f * (float)P.target, st);
}

int pass_gather_width() { return P1_CMAX - 4; }

}  // namespace vor
