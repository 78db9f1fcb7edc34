// reduce_static.cu -- fvlb_reduce_noalloc: the FP64 diagnostics reduction
// with its scratch memory in a file-scope device array, for callers that
// cannot allocate device memory.  The paper has no counterpart; this is a
// property of the library's interface only.
//
// The reduction is the same two-kernel scheme as fvlb_reduce (per-block
// partial sums, then one block reducing the partials in index order); only
// the partials live in `g_reduce_scratch` instead of handle-owned memory.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "fvlb.h"
#include "fvlb_internal.h"
#include "fvlb_launch.cuh"

namespace {

using namespace fvlb;

// Partial sums of one reduction: at most kMaxParts blocks x 8 doubles
// (64 KiB).  Every GPU that loads the library holds this array until the
// process exits.  All calls share it; each call overwrites the partials it
// uses before reading them, so nothing needs clearing, but two calls whose
// kernels overlap on the GPU (different streams without ordering) race.
constexpr int kMaxParts = 1024;
static __device__ __align__(256) double g_reduce_scratch[kMaxParts * 8];

// Device address of g_reduce_scratch, looked up once per device and CUDA
// context.  In host code the name g_reduce_scratch is only a host-side
// stand-in for the symbol, never a device address.  The address belongs to
// the context the module was loaded into: after cudaDeviceReset (or any new
// primary context) the module loads again, possibly elsewhere, so each
// cached address is kept with the context it was looked up in and looked up
// again when the current context differs.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};

// the current driver context (cuCtxGetCurrent through the runtime's
// driver entry point, so the library needs no link against libcuda)
typedef int (*ctx_get_fn)(void**);
void* current_context() {
  static ctx_get_fn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<ctx_get_fn>(p);
    cudaGetLastError();
  });
  void* ctx = nullptr;
  if (fn && fn(&ctx) != 0) ctx = nullptr;
  return ctx;
}

int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_global_error(FVLB_ECUDA, "fvlb_reduce_noalloc: no current CUDA device");
  }
  if (dev < 0 || dev >= kMaxDevices)
    return set_global_error(FVLB_EINVAL, "fvlb_reduce_noalloc: device ordinal out of range");
  void* ctx = current_context();   // null before the runtime made one current
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_reduce_scratch);   // (makes the primary context current)
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return set_global_error(FVLB_ECUDA,
                              "fvlb_reduce_noalloc: cudaGetSymbolAddress of the scratch failed");
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
    g_scratch_ctx[dev] = current_context();
  }
  *out = g_scratch_ptr[dev];
  return FVLB_OK;
}

template <class L, class S>
cudaError_t launch(const Grid& g, double eta_over_lam, const double F[3], const void* f,
                   const void* h, long long N, double* part, int nparts, double* out,
                   cudaStream_t stream) {
  using R = RT<S>;
  Phys<R> ph{};
  ph.eta_over_lam = R(eta_over_lam);
  ph.four_roll = 0;
  for (int a = 0; a < 3; ++a) ph.Fv[a] = R(F ? F[a] : 0.0);
  k_reduce_partial<L, S><<<nparts, kReduceThreads, 0, stream>>>(
      g, ph, static_cast<const S*>(f), static_cast<const S*>(h), part, N);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_final<<<1, kReduceThreads, 0, stream>>>(part, nparts, N, out);
  return cudaGetLastError();
}

template <class L>
cudaError_t dispatch(int storage, const Grid& g, double eol, const double F[3], const void* f,
                     const void* h, long long N, double* part, int nparts, double* out,
                     cudaStream_t st) {
#define CALL(S) launch<L, S>(g, eol, F, f, h, N, part, nparts, out, st)
  FVLB_DISPATCH(storage, CALL)
#undef CALL
}

}  // namespace

extern "C" int fvlb_reduce_noalloc(int lattice, int storage, int nx, int ny, int nz,
                                   const void* f, const void* h, long long pitch,
                                   double eta_p, double lambda, const double F[3],
                                   double* out, void* stream) {
  if (lattice != FVLB_D2Q9 && lattice != FVLB_D3Q19)
    return set_global_error(FVLB_EINVAL, "fvlb_reduce_noalloc: unknown lattice");
  if (storage < FVLB_FP64 || storage > FVLB_BF16_DEV_SR)
    return set_global_error(FVLB_EINVAL, "fvlb_reduce_noalloc: unknown storage");
  if (lattice == FVLB_D2Q9) nz = 1;
  if (nx < 1 || ny < 1 || nz < 1)
    return set_global_error(FVLB_EINVAL, "fvlb_reduce_noalloc: grid sizes must be >= 1");
  const long long N = (long long)nx * ny * nz;
  if (pitch < N)
    return set_global_error(FVLB_EINVAL, "fvlb_reduce_noalloc: pitch smaller than nx*ny*nz");
  if ((long long)lattice * pitch >= (1ll << 32))
    return set_global_error(FVLB_EINVAL, "fvlb_reduce_noalloc: grid too large");
  if (!f || !h || !out)
    return set_global_error(FVLB_EINVAL, "fvlb_reduce_noalloc: NULL buffer");
  if (!(lambda > 0.0) || !(eta_p >= 0.0) || !std::isfinite(lambda) || !std::isfinite(eta_p))
    return set_global_error(FVLB_EINVAL, "fvlb_reduce_noalloc: need lambda > 0, eta_p >= 0");
  const int nparts = reduce_parts(N);
  if (nparts > kMaxParts)
    return set_global_error(FVLB_EINVAL,
                            "fvlb_reduce_noalloc: more partial sums than the static scratch holds");
  double* part = nullptr;
  int r = scratch_for_current_device(&part);
  if (r != FVLB_OK) return r;
  Grid g{nx, ny, nz, 0, pitch};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = lattice == FVLB_D2Q9
                      ? dispatch<D2Q9>(storage, g, eta_p / lambda, F, f, h, N, part, nparts, out, st)
                      : dispatch<D3Q19>(storage, g, eta_p / lambda, F, f, h, N, part, nparts, out, st);
  if (e != cudaSuccess)
    return set_global_error(FVLB_ECUDA, cudaGetErrorString(e));
  return FVLB_OK;
}
