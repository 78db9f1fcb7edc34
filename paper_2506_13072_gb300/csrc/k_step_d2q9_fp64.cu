// k_step_d2q9_fp64.cu -- D2Q9 step kernels with double storage (one translation
// unit per lattice and storage so that the library compiles in parallel).
#include "fvlb_launch.cuh"

namespace fvlb {
template cudaError_t step_impl<D2Q9, double>(const StepDesc&);
}  // namespace fvlb
