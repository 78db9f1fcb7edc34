// k_batch_fp32.cu -- batched persistent D2Q9 step kernels with float storage.
#include "fvlb_batch_impl.cuh"

namespace fvlb {
template cudaError_t batch_step_impl<float>(const BatchLaunch&);
template int batch_occupancy_impl<float>(int);
template void batch_inst_fill_impl<float>(void*, int, int, int, long long, double, double, double,
                                       double, int, const double*, double, const void*, long long,
                                       long long, long long);
}  // namespace fvlb
