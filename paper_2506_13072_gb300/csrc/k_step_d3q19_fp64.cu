// k_step_d3q19_fp64.cu -- D3Q19 step kernels with double storage (one translation
// unit per lattice and storage so that the library compiles in parallel).
#include "fvlb_launch.cuh"

namespace fvlb {
template cudaError_t step_impl<D3Q19, double>(const StepDesc&);
}  // namespace fvlb
