// vor_cells_g32.cu -- explicit instantiations of the projector kernel (lanes per cell 32).
#include "vor_cells.cuh"

namespace vor {
template cudaError_t launch_fast_g<32>(const CellParams &, cudaStream_t);
}  // namespace vor
