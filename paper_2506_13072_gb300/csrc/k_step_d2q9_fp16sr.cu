// k_step_d2q9_fp16sr.cu -- D2Q9 step kernels with half_sr storage (one translation
// unit per lattice and storage so that the library compiles in parallel).
#include "fvlb_launch.cuh"

namespace fvlb {
template cudaError_t step_impl<D2Q9, half_sr>(const StepDesc&);
}  // namespace fvlb
