// vor_cells_t1.cu -- launcher of the one-thread-per-cell projector kernel.
#include "vor_cells_persist.cuh"

namespace vor {

template <bool WIDEN>
static cudaError_t launch_t(const CellParams &P, cudaStream_t st) {
    auto kern = cells_thread_kernel<T_NT, T_CMAX, T_SMAX, T_EMAX, T_RMAX, WIDEN>;
    const int smem = T_NT * T_CMAX * (int)sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T_NT, smem);
    if (per_sm < 1) per_sm = 1;
    long long want = ((long long)(P.cell_list ? P.n_list : P.n) + T_NT - 1) / T_NT;
    long long grid = (long long)sms * per_sm;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, T_NT, smem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_cells_thread(const CellParams &P, bool widen, cudaStream_t st) {
    return widen ? launch_t<true>(P, st) : launch_t<false>(P, st);
}

cudaError_t launch_cells_first_pass(const CellParams &P, int *gcount, long long *grho2, int *gpos,
                                    cudaStream_t st) {
    GatherOut G{gcount, grho2, gpos};
    gather_kernel<<<(P.n + 255) / 256, 256, 0, st>>>(P, G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto kern = cells_persist_kernel<P_NT, P_CMAX, P_SMAX, P_EMAX, P_RMAX>;
    const int smem = P_NT * P_CMAX * (int)sizeof(float4);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P_NT, smem);
    if (per_sm < 1) per_sm = 1;
    long long want = ((long long)P.n + P_NT - 1) / P_NT;
    long long grid = (long long)sms * per_sm;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, P_NT, smem, st>>>(P, G);
    return cudaGetLastError();
}

int first_pass_gather_width() { return P_GMAX; }

}  // namespace vor
