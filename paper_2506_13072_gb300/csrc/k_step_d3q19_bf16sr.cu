// k_step_d3q19_bf16sr.cu -- D3Q19 step kernels with bf16_sr storage (one translation
// unit per lattice and storage so that the library compiles in parallel).
#include "fvlb_launch.cuh"

namespace fvlb {
template cudaError_t step_impl<D3Q19, bf16_sr>(const StepDesc&);
}  // namespace fvlb
