// k_step_d2q9_bf16.cu -- D2Q9 step kernels with __nv_bfloat16 storage (one translation
// unit per lattice and storage so that the library compiles in parallel).
#include "fvlb_launch.cuh"

namespace fvlb {
template cudaError_t step_impl<D2Q9, __nv_bfloat16>(const StepDesc&);
}  // namespace fvlb
