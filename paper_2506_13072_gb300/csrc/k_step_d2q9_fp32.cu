// k_step_d2q9_fp32.cu -- D2Q9 step kernels with float storage (one translation
// unit per lattice and storage so that the library compiles in parallel).
#include "fvlb_launch.cuh"

namespace fvlb {
template cudaError_t step_impl<D2Q9, float>(const StepDesc&);
}  // namespace fvlb
