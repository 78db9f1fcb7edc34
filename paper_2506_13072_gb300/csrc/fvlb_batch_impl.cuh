// fvlb_batch_impl.cuh -- templated host launchers of the batched step, one
// translation unit per storage type (k_batch_<storage>.cu).
#pragma once

#include "fvlb_batch.h"
#include "fvlb_launch.cuh"

namespace fvlb {

// Register budgets: GX groups of 32 nodes x 3 components = 96 GX threads,
// MINB blocks per SM.
template <int GX>
struct BatchMinB {
  static constexpr int value = GX == 4 ? 2 : (GX == 2 ? 4 : 8);
};

// dynamic shared memory of the batched kernel's tile (0: static)
template <class S, int GX>
constexpr size_t batch_dyn() {
  return TileCfg<D2Q9, S, GX, 1, false, false, 1>::kDynamicBytes;
}

template <class S, int GX>
cudaError_t batch_launch_gx(const BatchLaunch& d) {
  constexpr int MINB = BatchMinB<GX>::value;
  constexpr int NT = FusedShape<D2Q9, GX, 1, false>::NT;
  constexpr size_t dyn = batch_dyn<S, GX>();
  using X = typename Store<S>::X;
  auto kern = k_step_batched<D2Q9, S, GX, MINB>;
  if constexpr (dyn > 0) {
    const cudaError_t e = allow_dynamic_smem(kern, dyn);
    if (e != cudaSuccess) return e;
  }
  int blocks = d.blocks;
  if (blocks <= 0) {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, dyn);
    blocks = sms * (per > 0 ? per : 1);
  }
  kern<<<blocks, NT, dyn, d.stream>>>(
      static_cast<const BatchInst<S>*>(d.inst), static_cast<const BatchTile*>(d.tiles),
      d.ntiles, static_cast<S*>(d.fA), static_cast<S*>(d.fB), static_cast<S*>(d.hA),
      static_cast<S*>(d.hB), static_cast<X*>(d.chi), d.parity, d.first, d.tstep, d.mchunk);
  return cudaGetLastError();
}

template <class S>
cudaError_t batch_step_impl(const BatchLaunch& d) {
  switch (d.gx) {
    case 1: return batch_launch_gx<S, 1>(d);
    case 2: return batch_launch_gx<S, 2>(d);
    case 4: return batch_launch_gx<S, 4>(d);
    default: return cudaErrorInvalidValue;
  }
}

template <class S, int GX>
int batch_occupancy_gx() {
  auto kern = k_step_batched<D2Q9, S, GX, BatchMinB<GX>::value>;
  constexpr size_t dyn = batch_dyn<S, GX>();
  if constexpr (dyn > 0) {
    if (allow_dynamic_smem(kern, dyn) != cudaSuccess) return 0;
  }
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, FusedShape<D2Q9, GX, 1, false>::NT, dyn);
  return per;
}

template <class S>
int batch_occupancy_impl(int gx) {
  switch (gx) {
    case 1: return batch_occupancy_gx<S, 1>();
    case 2: return batch_occupancy_gx<S, 2>();
    default: return batch_occupancy_gx<S, 4>();
  }
}

template <class S>
void batch_inst_fill_impl(void* dst, int nx, int ny, int walls, long long pitch, double tau_f,
                          double tau_h, double eta_p, double lambda, int force_kind,
                          const double* F0, double omega, const void* tables, long long f_off,
                          long long h_off, long long chi_off) {
  using R = RT<S>;
  BatchInst<S> I{};
  I.g = Grid{nx, ny, 1, walls, pitch};
  StepDesc sd{};
  sd.nx = nx;
  sd.ny = ny;
  sd.nz = 1;
  sd.tau_f = tau_f;
  sd.tau_h = tau_h;
  sd.eta_p = eta_p;
  sd.lambda = lambda;
  sd.four_roll = force_kind == 2;
  sd.amp = F0[0];
  sd.tables = tables;
  for (int a = 0; a < 3; ++a) sd.Fv[a] = force_kind == 1 ? F0[a] : 0.0;
  I.ph = make_phys<R>(sd);
  I.f_off = f_off;
  I.h_off = h_off;
  I.chi_off = chi_off;
  I.cosine = force_kind == 3;
  for (int a = 0; a < 3; ++a) I.F0[a] = F0[a];
  I.omega = omega;
  *static_cast<BatchInst<S>*>(dst) = I;
}

}  // namespace fvlb
