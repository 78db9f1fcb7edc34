// k_batch_bf16.cu -- batched persistent D2Q9 step kernels with __nv_bfloat16 storage.
#include "fvlb_batch_impl.cuh"

namespace fvlb {
template cudaError_t batch_step_impl<__nv_bfloat16>(const BatchLaunch&);
template int batch_occupancy_impl<__nv_bfloat16>(int);
template void batch_inst_fill_impl<__nv_bfloat16>(void*, int, int, int, long long, double, double, double,
                                       double, int, const double*, double, const void*, long long,
                                       long long, long long);
}  // namespace fvlb
