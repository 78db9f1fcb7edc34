// k_d3q19.cu -- D3Q19 instantiation of the step, initialisation, field and
// diagnostics launchers (one translation unit per lattice so that the two
// lattices compile in parallel).
#include "fvlb_launch.cuh"

namespace fvlb {

FVLB_EXTERN_STEP(D3Q19)

cudaError_t step_d3q19(const StepDesc& d) {
#define CALL(S) step_impl<D3Q19, S>(d)
  FVLB_DISPATCH(d.storage, CALL)
#undef CALL
}

cudaError_t init_d3q19(const InitDesc& d) {
#define CALL(S) init_impl<D3Q19, S>(d)
  FVLB_DISPATCH(d.storage, CALL)
#undef CALL
}

cudaError_t fields_d3q19(const StepDesc& d, int which, double* out) {
#define CALL(S) fields_impl<D3Q19, S>(d, which, out)
  FVLB_DISPATCH(d.storage, CALL)
#undef CALL
}

cudaError_t reduce_d3q19(const StepDesc& d, double* part, double* out) {
#define CALL(S) reduce_impl<D3Q19, S>(d, part, out)
  FVLB_DISPATCH(d.storage, CALL)
#undef CALL
}

cudaError_t conformation_d3q19(const StepDesc& d, double* part, double* out) {
#define CALL(S) conf_impl<D3Q19, S>(d, part, out)
  FVLB_DISPATCH(d.storage, CALL)
#undef CALL
}

cudaError_t repair_d3q19(const StepDesc& d, double eps, unsigned long long* count) {
#define CALL(S) repair_impl<D3Q19, S>(d, eps, count)
  FVLB_DISPATCH(d.storage, CALL)
#undef CALL
}

}  // namespace fvlb
