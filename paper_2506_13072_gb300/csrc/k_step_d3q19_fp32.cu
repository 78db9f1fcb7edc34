// k_step_d3q19_fp32.cu -- D3Q19 step kernels with float storage (one translation
// unit per lattice and storage so that the library compiles in parallel).
#include "fvlb_launch.cuh"

namespace fvlb {
template cudaError_t step_impl<D3Q19, float>(const StepDesc&);
}  // namespace fvlb
