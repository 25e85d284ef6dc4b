// vor_cells_g8_16.cu -- explicit instantiations of the projector kernel (lanes per cell 8, 16).
#include "vor_cells.cuh"

namespace vor {
template cudaError_t launch_fast_g<8>(const CellParams &, cudaStream_t);
template cudaError_t launch_fast_g<16>(const CellParams &, cudaStream_t);
}  // namespace vor
