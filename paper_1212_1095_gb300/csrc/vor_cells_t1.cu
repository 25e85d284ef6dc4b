// vor_cells_t1.cu -- launchers of the one-thread-per-cell projector passes.
#include "vor_cells_persist.cuh"
#include "vor_flower.cuh"

namespace vor {

static GatherOut gather_out(const CellParams &P, int pass, int *gcount, long long *grho2,
                            float2 *gtab, int *glab) {
    // both passes share lists of gather_rows(n) * (P1_CMAX - 4) entries in
    // tiles of 32 rows; the second pass lists fewer cells (the deferred ones)
    // with more sites each
    const long long entries = gather_rows(P.n) * (P1_CMAX - 4);
    if (pass == 1) return GatherOut{gcount, grho2, gtab, glab, P1_CMAX - 4, P.n};
    const int w = pass == 2 ? P2_CMAX - 4 : P3_CMAX - 4;
    return GatherOut{gcount, grho2, gtab, glab, w, (int)(entries / (w * 32) * 32)};
}

cudaError_t launch_gather_pass(const CellParams &P, int pass, int *gcount, long long *grho2,
                               float2 *gtab, int *glab, cudaStream_t st) {
    const int total_max = P.cell_list ? P.n_list : P.n;
    const GatherOut G = gather_out(P, pass, gcount, grho2, gtab, glab);
    // the sub-bucket versions only when the build divided buckets
    const bool fine = P.fdesc != nullptr;
    if (pass == 1 && !P.cell_list) {
        const int blocks = (total_max + 127) / 128;
        if (fine)
            gather_strip_kernel<128, P1_CMAX - 4, 1280, 1280, 32, true><<<blocks, 128, 0, st>>>(
                P, G, (float)P.target);
        else
            gather_strip_kernel<128, P1_CMAX - 4, 1280, 1280, 32, false><<<blocks, 128, 0, st>>>(
                P, G, (float)P.target);
    } else if (pass == 1) {
        const int blocks = (total_max + 63) / 64;
        if (fine)
            gather_kernel<64, P1_CMAX - 4, true, true><<<blocks, 64, 0, st>>>(P, G, (float)P.target);
        else
            gather_kernel<64, P1_CMAX - 4, true, false><<<blocks, 64, 0, st>>>(P, G, (float)P.target);
    } else if (pass == 2) {
        const int blocks = (total_max + 127) / 128;
        if (fine)
            gather_kernel<128, P2_CMAX - 4, false, true><<<blocks, 128, 0, st>>>(P, G, 2.2f * (float)P.target);
        else
            gather_kernel<128, P2_CMAX - 4, false, false><<<blocks, 128, 0, st>>>(P, G, 2.2f * (float)P.target);
    }
    if (pass >= 3) {
        // one warp per cell of the list; a grid of a few warps per SM slot,
        // the rest by grid stride (the list length is known on the device)
        const long long want = ((long long)total_max + FL_WARPS - 1) / FL_WARPS;
        const int grid = (int)(want < 152 * 16 ? (want > 0 ? want : 1) : 152 * 16);
        flower_gather_kernel<P3_CMAX - 4><<<grid, 32 * FL_WARPS, 0, st>>>(P, G);
    }
    return cudaGetLastError();
}

template <int CMAX, int NT>
static cudaError_t launch_persist(const CellParams &P, const GatherOut &G, cudaStream_t st) {
    const int total_max = P.cell_list ? P.n_list : P.n;
    auto kern = cells_persist_kernel<NT, CMAX, P_SMAX, P_EMAX, P_RMAX>;
    const int smem = NT * CMAX * (int)sizeof(float2);
    int resident = 0;
    cudaError_t e = resident_grid((const void *)kern, NT, smem, resident);
    if (e != cudaSuccess) return e;
    long long want = ((long long)total_max + NT - 1) / NT;
    long long grid = resident;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, NT, smem, st>>>(P, G);
    return cudaGetLastError();
}

cudaError_t launch_cells_pass(const CellParams &P, int pass, int *gcount, long long *grho2,
                              float2 *gtab, int *glab, int block, cudaStream_t st) {
    const GatherOut G = gather_out(P, pass, gcount, grho2, gtab, glab);
    if (pass == 1) {
        // the block shape of the first pass (an autotuner choice): the
        // warps' work is independent, a block shares only its launch slot
        if (block == 32) return launch_persist<P1_CMAX, 32>(P, G, st);
        if (block == 128) return launch_persist<P1_CMAX, 128>(P, G, st);
        return launch_persist<P1_CMAX, P_NT>(P, G, st);
    }
    if (pass == 2) return launch_persist<P2_CMAX, P_NT>(P, G, st);
    return launch_persist<P3_CMAX, P_NT>(P, G, st);
}

int pass_gather_width() { return P1_CMAX - 4; }
long long gather_rows(long long n) { return (n + 31) / 32 * 32; }

}  // namespace vor
