// fvlb_batch.h -- host-side launch interface of the batched persistent step
// (internal; the public interface is the fvlb_batch_* part of fvlb.h).
#pragma once

#include <cuda_runtime.h>

namespace fvlb {

// One launch of k_step_batched<D2Q9, S, gx> over `ntiles` tiles.  `inst` and
// `tiles` are device arrays built by the host (BatchInst<S>, BatchTile);
// blocks = 0 asks for one block per resident slot of the GPU.
struct BatchLaunch {
  int storage;
  int gx;
  const void* inst;
  const void* tiles;
  int ntiles;
  void *fA, *fB, *hA, *hB, *chi;
  int parity, first;
  const long long* tstep;
  int mchunk;
  int blocks;
  cudaStream_t stream;
};

cudaError_t batch_step(const BatchLaunch& d);
cudaError_t batch_advance(long long* t, cudaStream_t stream);
// resident blocks per SM of k_step_batched for (storage, gx)
int batch_occupancy(int storage, int gx);
// size in bytes of BatchInst<S> for the storage, and a host-side builder
size_t batch_inst_size(int storage);
// Fill the BatchInst of instance i into host buffer dst (batch_inst_size
// bytes): grid, physics in the working precision, arena offsets, force.
void batch_inst_fill(int storage, void* dst, int nx, int ny, int walls, long long pitch,
                     double tau_f, double tau_h, double eta_p, double lambda, int force_kind,
                     const double F0[3], double omega, const void* tables, long long f_off,
                     long long h_off, long long chi_off);

}  // namespace fvlb
