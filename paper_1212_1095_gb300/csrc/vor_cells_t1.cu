// vor_cells_t1.cu -- launchers of the one-thread-per-cell projector passes.
#include "vor_cells_persist.cuh"

namespace vor {

static GatherOut gather_out(const CellParams &P, int pass, int *gcount, long long *grho2,
                            float2 *gtab, int *glab) {
    // both passes share lists of gather_rows(n) * (P1_CMAX - 4) entries in
    // tiles of 32 rows; the second pass lists fewer cells (the deferred ones)
    // with more sites each
    const long long entries = gather_rows(P.n) * (P1_CMAX - 4);
    if (pass == 1) return GatherOut{gcount, grho2, gtab, glab, P1_CMAX - 4, P.n};
    return GatherOut{gcount, grho2, gtab, glab, P2_CMAX - 4, (int)(entries / ((P2_CMAX - 4) * 32) * 32)};
}

cudaError_t launch_gather_pass(const CellParams &P, int pass, int *gcount, long long *grho2,
                               float2 *gtab, int *glab, cudaStream_t st) {
    const int total_max = P.cell_list ? P.n_list : P.n;
    const GatherOut G = gather_out(P, pass, gcount, grho2, gtab, glab);
    if (pass == 1 && !P.cell_list)
        gather_strip_kernel<128, P1_CMAX - 4, 1280, 1280, 32><<<(total_max + 127) / 128, 128, 0, st>>>(
            P, G, (float)P.target);
    else if (pass == 1)
        gather_kernel<64, P1_CMAX - 4, true><<<(total_max + 63) / 64, 64, 0, st>>>(P, G, (float)P.target);
    else
        gather_kernel<128, P2_CMAX - 4, false><<<(total_max + 127) / 128, 128, 0, st>>>(P, G, 2.2f * (float)P.target);
    return cudaGetLastError();
}

template <int CMAX>
static cudaError_t launch_persist(const CellParams &P, const GatherOut &G, cudaStream_t st) {
    const int total_max = P.cell_list ? P.n_list : P.n;
    auto kern = cells_persist_kernel<P_NT, CMAX, P_SMAX, P_EMAX, P_RMAX>;
    const int smem = P_NT * CMAX * (int)sizeof(float2);
    int resident = 0;
    cudaError_t e = resident_grid((const void *)kern, P_NT, smem, resident);
    if (e != cudaSuccess) return e;
    long long want = ((long long)total_max + P_NT - 1) / P_NT;
    long long grid = resident;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, P_NT, smem, st>>>(P, G);
    return cudaGetLastError();
}

cudaError_t launch_cells_pass(const CellParams &P, int pass, int *gcount, long long *grho2,
                              float2 *gtab, int *glab, cudaStream_t st) {
    const GatherOut G = gather_out(P, pass, gcount, grho2, gtab, glab);
    return pass == 1 ? launch_persist<P1_CMAX>(P, G, st) : launch_persist<P2_CMAX>(P, G, st);
}

int pass_gather_width() { return P1_CMAX - 4; }
long long gather_rows(long long n) { return (n + 31) / 32 * 32; }

}  // namespace vor
