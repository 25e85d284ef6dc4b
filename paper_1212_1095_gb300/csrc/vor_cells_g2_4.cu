// vor_cells_g2_4.cu -- explicit instantiations of the projector kernel (lanes per cell 2, 4).
#include "vor_cells.cuh"

namespace vor {
template cudaError_t launch_fast_g<2>(const CellParams &, cudaStream_t);
template cudaError_t launch_fast_g<4>(const CellParams &, cudaStream_t);
}  // namespace vor
