// fvlb_internal.h -- host-side descriptors shared by the C-ABI layer and the
// per-lattice kernel launchers.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace fvlb {

enum Storage { kFP64 = 0, kFP32 = 1, kFP16Dev = 2, kBF16Dev = 3, kFP16DevSR = 4, kBF16DevSR = 5 };

// Bytes of one population buffer of a grid.  The 16-bit forms append FP32
// arrays to each buffer (fvlb_lattice.cuh): the velocity U[D][pitch] after
// f[Q][pitch], the rest stress populations h0[C][pitch] after h[C][Q][pitch].
inline bool v2_storage(int storage) { return storage >= kFP16Dev; }
inline size_t elem_bytes(int storage) { return storage == kFP64 ? 8 : (storage == kFP32 ? 4 : 2); }
inline size_t f_buffer_bytes(int storage, int Q, int D, size_t pitch) {
  return elem_bytes(storage) * (size_t)Q * pitch + (v2_storage(storage) ? 4 * (size_t)D * pitch : 0);
}
inline size_t h_buffer_bytes(int storage, int C, int Q, size_t pitch) {
  return elem_bytes(storage) * (size_t)C * Q * pitch + (v2_storage(storage) ? 4 * (size_t)C * pitch : 0);
}
// HBM bytes one node update reads and writes: populations, chi of the
// previous step, and (16-bit forms) U and h0 in place of the 16-bit rest
// stress populations
inline double bytes_per_update(int storage, int Q, int C, int D) {
  const double sb = (double)elem_bytes(storage), xb = storage == kFP64 ? 8.0 : 4.0;
  if (!v2_storage(storage)) return 2.0 * (Q + (double)C * Q) * sb + 2.0 * C * xb;
  return 2.0 * (Q * sb + 4.0 * D + C * (Q - 1) * sb + 4.0 * C) + 2.0 * C * xb;
}

// Precision-agnostic description of one launch; the launcher converts the
// physics to the working precision of the storage type.
struct StepDesc {
  int nx, ny, nz, walls;
  long long N, pitch;
  int storage;
  int variant;          // 0 fused, 1 split
  const void* f_in;
  void* f_out;
  const void* h_in;
  void* h_out;
  void* chi;
  void* ubuf;           // split variant: D * pitch working-precision values
  double tau_f, tau_h, eta_p, lambda;
  int four_roll;
  double Fv[3];         // uniform force of this step (CONST / COSINE)
  double amp;           // FOUR_ROLL amplitude
  const void* tables;   // FOUR_ROLL: sx[nx], cx[nx], sy[ny], cy[ny] in working precision
  int first;
  long long step;       // step count t of this launch
  int sms;
  cudaStream_t stream;
  const void* mlp;      // learned closure: packed weights, or null (analytic chi)
  double cl_tol;        // fallback tolerance of the learned closure
  unsigned long long* cl_count;  // [0] nodes on the network, [1] fallbacks
  int scheme;           // 0 present (f^B), 1 original (stress divergence as a force)
  void* taup;           // original scheme: C * pitch working-precision values
  void* fdiv;           // original scheme, fused variant: D * pitch working-precision values
  int model;            // constitutive model (0 Oldroyd-B, 1 Giesekus, 2 / 3 PTT)
  double mpar;          // its parameter
  unsigned* err;        // device word: bounded waits that ran out (bit 0: staging copies)
};

struct InitDesc {
  int nx, ny, nz;
  long long N, pitch;
  int storage;
  void* f;
  void* h;
  void* chi;
  const double* u0;
  const double* p0;
  const double* A0;
  int sms;
  cudaStream_t stream;
};

// Per-lattice launchers (one translation unit per lattice).
cudaError_t step_d2q9(const StepDesc& d);
cudaError_t step_d3q19(const StepDesc& d);
cudaError_t init_d2q9(const InitDesc& d);
cudaError_t init_d3q19(const InitDesc& d);
// fields: which as in fvlb.h; out is a device FP64 buffer
cudaError_t fields_d2q9(const StepDesc& d, int which, double* out);
cudaError_t fields_d3q19(const StepDesc& d, int which, double* out);
// diagnostics: part has room for reduce_parts(N) * 8 doubles, out for 8
int reduce_parts(long long N);
cudaError_t reduce_d2q9(const StepDesc& d, double* part, double* out);
cudaError_t reduce_d3q19(const StepDesc& d, double* part, double* out);
// conformation check: part as for the diagnostics, out[3] as fvlb_conformation
cudaError_t conformation_d2q9(const StepDesc& d, double* part, double* out);
cudaError_t conformation_d3q19(const StepDesc& d, double* part, double* out);
// high-Wi repair: count (device) receives the number of nodes changed
cudaError_t repair_d2q9(const StepDesc& d, double eps, unsigned long long* count);
cudaError_t repair_d3q19(const StepDesc& d, double eps, unsigned long long* count);
cudaError_t reduce_finalize(const double* part, int nparts, long long N, double* out,
                            cudaStream_t stream);
// record the message returned by fvlb_last_error(NULL); returns code
int set_global_error(int code, const char* msg);
}  // namespace fvlb
#include "fvlb.h"
namespace fvlb {
// the process-wide allocator hooks (NULL: cudaMalloc / cudaFree)
void current_allocator(fvlb_alloc_fn* a, fvlb_free_fn* f, void** ctx);
// the current state of a handle as a launch descriptor (allocating and
// initialising it to rest if needed)
struct StateView {
  int lattice;
  long long N;
  StepDesc desc;
};
int state_view(fvlb_t h, StateView* v);
// the packed inference weights of a network (device) and its lattice
const void* mlp_packed(fvlb_mlp_t m);
int mlp_lattice(fvlb_mlp_t m);

}  // namespace fvlb
