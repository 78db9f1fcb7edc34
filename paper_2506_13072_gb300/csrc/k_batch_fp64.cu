// k_batch_fp64.cu -- batched persistent D2Q9 step kernels with double storage.
#include "fvlb_batch_impl.cuh"

namespace fvlb {
template cudaError_t batch_step_impl<double>(const BatchLaunch&);
template int batch_occupancy_impl<double>(int);
template void batch_inst_fill_impl<double>(void*, int, int, int, long long, double, double, double,
                                       double, int, const double*, double, const void*, long long,
                                       long long, long long);
}  // namespace fvlb
