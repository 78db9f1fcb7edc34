// api.cu -- the C ABI declared in include/fvlb.h: handle life cycle, device
// memory through the caller's allocator hooks, stream, the A/B buffer flip
// and the host-side arithmetic of a step's scalar parameters (the uniform
// force F0 cos(omega t) of the step).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fvlb.h"
#include "fvlb_internal.h"
#include "fvlb_kernels.cuh"

using fvlb::StepDesc;

namespace {

fvlb_alloc_fn g_alloc = nullptr;
fvlb_free_fn g_free = nullptr;
void* g_actx = nullptr;
thread_local std::string g_err;

constexpr uint64_t kStateMagic = 0x31424c5646ull;  // "FVLB1"

// 64-byte header of a checkpoint image, followed by f, h and chi as laid out
// on the device (current buffer).
struct StateHeader {
  uint64_t magic;
  int32_t lattice, nx, ny, nz, storage, first;
  int64_t t, pitch;
  int64_t reserved[2];
};
static_assert(sizeof(StateHeader) == 64, "checkpoint header is 64 bytes");

size_t storage_bytes(int storage) { return storage == FVLB_FP64 ? 8 : (storage == FVLB_FP32 ? 4 : 2); }
size_t chi_bytes(int storage) { return storage == FVLB_FP64 ? 8 : 4; }

}  // namespace

struct fvlb_s {
  int lattice = 0, D = 0, Q = 0, C = 0;
  int nx = 0, ny = 0, nz = 1;
  long long N = 0, pitch = 0;
  double tau_s = 0, eta_p = 0, lambda = 0, tau_h = 0.501;
  fvlb_force force{};
  unsigned walls = 0;
  int storage = FVLB_FP64;
  int variant = FVLB_KERNEL_FUSED;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 1;
  bool allocated = false;
  int first = 1;
  long long t = 0;
  int cur = 0;
  void* f[2] = {nullptr, nullptr};
  void* h[2] = {nullptr, nullptr};
  void* chi = nullptr;
  void* ubuf = nullptr;
  void* tables = nullptr;
  double* part = nullptr;   // reduction partials
  double* red = nullptr;    // 8 reduced doubles
  double* fbuf = nullptr;   // field output scratch, N * max(D, C) doubles
  fvlb_mlp_t mlp = nullptr; // learned closure, or null
  double cl_tol = 1e-2;
  unsigned long long* cl_count = nullptr;  // [0] network nodes, [1] fallbacks
  unsigned* dev_err = nullptr;  // bounded device waits that ran out (bit 0: staging copies)
  int scheme = FVLB_SCHEME_PRESENT;
  void* taup = nullptr;     // original scheme: polymer stress working array
  void* fdiv = nullptr;     // original scheme: its divergence (fused variant)
  int model = FVLB_MODEL_OLDROYD_B;
  double mpar = 0.0;        // alpha (Giesekus) or eps (PTT)
  // periodic finiteness check (fvlb_set_check_interval)
  long chk_every = 0;       // steps between checks, 0: off
  double* chk_host = nullptr;  // page-locked copy of the last check's diagnostics
  cudaEvent_t chk_ev = nullptr;
  bool chk_pending = false;
  long long chk_t = 0;      // step count of the pending check
  long long bad_t = -1;     // step count at which a check found non-finite values
  fvlb_alloc_fn alloc = nullptr;
  fvlb_free_fn free_ = nullptr;
  void* actx = nullptr;
  std::vector<void*> owned;
  std::string err;
};

namespace {

// NVTX range over one API call (visible in a profiler timeline; near free
// when no tool is attached)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

int fail(fvlb_t h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_err = msg;
  return code;
}

int cuda_fail(fvlb_t h, cudaError_t e, const char* what) {
  return fail(h, FVLB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(fvlb_t h, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (h->alloc) {
    p = h->alloc(bytes, h->actx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) h->owned.push_back(p);
  return p;
}

void dev_free(fvlb_t h, void* p) {
  if (!p) return;
  auto it = std::find(h->owned.begin(), h->owned.end(), p);
  if (it != h->owned.end()) h->owned.erase(it);
  if (h->free_) h->free_(p, h->actx);
  else cudaFree(p);
}

void free_all(fvlb_t h) {
  std::vector<void*> o = h->owned;
  for (void* p : o) dev_free(h, p);
  h->owned.clear();
  h->f[0] = h->f[1] = h->h[0] = h->h[1] = nullptr;
  h->chi = h->ubuf = h->tables = nullptr;
  h->part = h->red = h->fbuf = nullptr;
  h->cl_count = nullptr;
  h->dev_err = nullptr;
  h->taup = nullptr;
  h->fdiv = nullptr;
  h->allocated = false;
}

StepDesc make_desc(fvlb_t h) {
  StepDesc d{};
  d.nx = h->nx;
  d.ny = h->ny;
  d.nz = h->nz;
  d.walls = (int)h->walls;
  d.N = h->N;
  d.pitch = h->pitch;
  d.storage = h->storage;
  d.variant = h->variant;
  d.f_in = h->f[h->cur];
  d.f_out = h->f[1 - h->cur];
  d.h_in = h->h[h->cur];
  d.h_out = h->h[1 - h->cur];
  d.chi = h->chi;
  d.ubuf = h->ubuf;
  d.tau_f = h->tau_s;
  d.tau_h = h->tau_h;
  d.eta_p = h->eta_p;
  d.lambda = h->lambda;
  d.four_roll = h->force.kind == FVLB_FORCE_FOUR_ROLL;
  d.amp = h->force.F0[0];
  d.tables = h->tables;
  d.first = h->first;
  d.step = h->t;
  d.sms = h->sms;
  d.stream = h->stream;
  d.mlp = h->mlp ? fvlb::mlp_packed(h->mlp) : nullptr;
  d.cl_tol = h->cl_tol;
  d.cl_count = h->cl_count;
  d.scheme = h->scheme;
  d.taup = h->taup;
  d.fdiv = h->fdiv;
  d.model = h->model;
  d.mpar = h->mpar;
  d.err = h->dev_err;
  double c = 0.0;
  if (h->force.kind == FVLB_FORCE_CONST) c = 1.0;
  if (h->force.kind == FVLB_FORCE_COSINE) c = std::cos(h->force.omega * (double)h->t);
  for (int a = 0; a < 3; ++a) d.Fv[a] = (a < h->D) ? h->force.F0[a] * c : 0.0;
  return d;
}

int ensure_state(fvlb_t h, bool init_rest);

int allocate(fvlb_t h) {
  if (h->allocated) return FVLB_OK;
  h->alloc = g_alloc;
  h->free_ = g_free;
  h->actx = g_actx;
  const size_t sb = storage_bytes(h->storage), xb = chi_bytes(h->storage);
  const size_t P = (size_t)h->pitch;
  const size_t rb = h->storage == FVLB_FP64 ? 8 : 4;
  (void)sb;
  for (int b = 0; b < 2; ++b) {
    h->f[b] = dev_alloc(h, fvlb::f_buffer_bytes(h->storage, h->Q, h->D, P));
    h->h[b] = dev_alloc(h, fvlb::h_buffer_bytes(h->storage, h->C, h->Q, P));
  }
  h->chi = dev_alloc(h, xb * h->C * P);
  h->ubuf = dev_alloc(h, rb * h->D * P);
  const int nparts = fvlb::reduce_parts(h->N);
  h->part = static_cast<double*>(dev_alloc(h, sizeof(double) * 8 * (size_t)nparts));
  h->red = static_cast<double*>(dev_alloc(h, sizeof(double) * 8));
  h->cl_count = static_cast<unsigned long long*>(dev_alloc(h, 2 * sizeof(unsigned long long)));
  h->dev_err = static_cast<unsigned*>(dev_alloc(h, sizeof(unsigned)));
  bool ok = h->f[0] && h->f[1] && h->h[0] && h->h[1] && h->chi && h->ubuf && h->part && h->red &&
            h->cl_count && h->dev_err;
  if (ok && cudaMemset(h->cl_count, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) ok = false;
  if (ok && cudaMemset(h->dev_err, 0, sizeof(unsigned)) != cudaSuccess) ok = false;
  // 16-bit forms: the i = 0 slots of the 16-bit stress arrays are never
  // used (the rest populations are FP32); zero them once so that checkpoint
  // images hold no leftover bytes
  if (ok && fvlb::v2_storage(h->storage))
    for (int b = 0; b < 2 && ok; ++b)
      ok = cudaMemset(h->h[b], 0, fvlb::h_buffer_bytes(h->storage, h->C, h->Q, P)) == cudaSuccess;
  if (ok && h->force.kind == FVLB_FORCE_FOUR_ROLL) {
    const int n = 2 * (h->nx + h->ny);
    h->tables = dev_alloc(h, rb * n);
    ok = h->tables != nullptr;
    if (ok) {
      std::vector<double> t(n);
      for (int x = 0; x < h->nx; ++x) {
        t[x] = std::sin(h->force.k * x);
        t[h->nx + x] = std::cos(h->force.k * x);
      }
      for (int y = 0; y < h->ny; ++y) {
        t[2 * h->nx + y] = std::sin(h->force.k * y);
        t[2 * h->nx + h->ny + y] = std::cos(h->force.k * y);
      }
      cudaError_t e;
      if (rb == 8) {
        e = cudaMemcpy(h->tables, t.data(), 8 * n, cudaMemcpyHostToDevice);
      } else {
        std::vector<float> tf(t.begin(), t.end());
        e = cudaMemcpy(h->tables, tf.data(), 4 * n, cudaMemcpyHostToDevice);
      }
      if (e != cudaSuccess) {
        free_all(h);
        return cuda_fail(h, e, "upload of the force tables");
      }
    }
  }
  if (!ok) {
    free_all(h);
    return fail(h, FVLB_ENOMEM, "device allocation failed");
  }
  h->allocated = true;
  return FVLB_OK;
}

int run_init(fvlb_t h, const double* u0, const double* p0, const double* A0) {
  const size_t N = (size_t)h->N;
  const size_t nu = u0 ? N * h->D : 0, np = p0 ? N : 0, nA = A0 ? N * h->C : 0;
  double* tmp = nullptr;
  if (nu + np + nA) {
    tmp = static_cast<double*>(dev_alloc(h, sizeof(double) * (nu + np + nA)));
    if (!tmp) return fail(h, FVLB_ENOMEM, "device allocation of the initial fields failed");
  }
  cudaError_t e = cudaSuccess;
  double* du = tmp;
  double* dp = tmp ? tmp + nu : nullptr;
  double* dA = tmp ? tmp + nu + np : nullptr;
  if (u0) e = cudaMemcpyAsync(du, u0, sizeof(double) * nu, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && p0)
    e = cudaMemcpyAsync(dp, p0, sizeof(double) * np, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && A0)
    e = cudaMemcpyAsync(dA, A0, sizeof(double) * nA, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    fvlb::InitDesc d{};
    d.nx = h->nx;
    d.ny = h->ny;
    d.nz = h->nz;
    d.N = h->N;
    d.pitch = h->pitch;
    d.storage = h->storage;
    d.f = h->f[h->cur];
    d.h = h->h[h->cur];
    d.chi = h->chi;
    d.u0 = u0 ? du : nullptr;
    d.p0 = p0 ? dp : nullptr;
    d.A0 = A0 ? dA : nullptr;
    d.sms = h->sms;
    d.stream = h->stream;
    e = h->lattice == FVLB_D2Q9 ? fvlb::init_d2q9(d) : fvlb::init_d3q19(d);
  }
  // a new state: forget the time-outs of the old one
  if (e == cudaSuccess && h->dev_err) e = cudaMemsetAsync(h->dev_err, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (tmp) dev_free(h, tmp);
  if (e != cudaSuccess) return cuda_fail(h, e, "initialisation");
  h->first = 1;
  h->t = 0;
  return FVLB_OK;
}

int ensure_state(fvlb_t h, bool init_rest) {
  if (h->allocated) return FVLB_OK;
  int r = allocate(h);
  if (r != FVLB_OK) return r;
  if (init_rest) return run_init(h, nullptr, nullptr, nullptr);
  return FVLB_OK;
}

int comps(fvlb_t h, int which) {
  switch (which) {
    case FVLB_FIELD_U: return h->D;
    case FVLB_FIELD_P: return 1;
    case FVLB_FIELD_A:
    case FVLB_FIELD_TAU_P: return h->C;
    default: return 0;
  }
}

size_t state_bytes(fvlb_t h) {
  const size_t P = (size_t)h->pitch;
  return sizeof(StateHeader) + fvlb::f_buffer_bytes(h->storage, h->Q, h->D, P) +
         fvlb::h_buffer_bytes(h->storage, h->C, h->Q, P) + chi_bytes(h->storage) * (size_t)h->C * P;
}

}  // namespace

namespace fvlb {

int state_view(fvlb_t h, StateView* v) {
  if (!h || !v) return FVLB_EINVAL;
  int r = ensure_state(h, true);
  if (r != FVLB_OK) return r;
  v->lattice = h->lattice;
  v->N = h->N;
  v->desc = make_desc(h);
  return FVLB_OK;
}

int set_global_error(int code, const char* msg) {
  g_err = msg;
  return code;
}

void current_allocator(fvlb_alloc_fn* a, fvlb_free_fn* f, void** ctx) {
  *a = g_alloc;
  *f = g_free;
  *ctx = g_actx;
}

int reduce_parts(long long N) {
  const long long want = (N + kReduceThreads - 1) / kReduceThreads;
  return (int)std::max<long long>(1, std::min<long long>(want, 1024));
}

cudaError_t reduce_finalize(const double* part, int nparts, long long N, double* out,
                            cudaStream_t stream) {
  k_reduce_final<<<1, kReduceThreads, 0, stream>>>(part, nparts, N, out);
  return cudaGetLastError();
}

}  // namespace fvlb

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

static int check_poll(fvlb_t h, bool wait);

int fvlb_set_allocator(fvlb_alloc_fn alloc_fn, fvlb_free_fn free_fn, void* ctx) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr))
    return fail(nullptr, FVLB_EINVAL, "fvlb_set_allocator: give both hooks or neither");
  g_alloc = alloc_fn;
  g_free = free_fn;
  g_actx = alloc_fn ? ctx : nullptr;
  return FVLB_OK;
}

int fvlb_create(fvlb_t* out, int lattice, int nx, int ny, int nz, double tau_s,
                double eta_p, double lambda, const fvlb_force* force) {
  if (!out) return fail(nullptr, FVLB_EINVAL, "fvlb_create: out is NULL");
  *out = nullptr;
  if (lattice != FVLB_D2Q9 && lattice != FVLB_D3Q19)
    return fail(nullptr, FVLB_EINVAL, "fvlb_create: lattice must be FVLB_D2Q9 or FVLB_D3Q19");
  if (lattice == FVLB_D2Q9) nz = 1;
  if (nx < 1 || ny < 1 || nz < 1)
    return fail(nullptr, FVLB_EINVAL, "fvlb_create: grid sizes must be >= 1");
  // population arrays are addressed with 32-bit element offsets: Q * pitch
  // must stay below 2^32 (about 226 M sites for D3Q19, 477 M for D2Q9)
  if ((long long)lattice * (((long long)nx * ny * nz + 63) / 64 * 64) >= (1ll << 32))
    return fail(nullptr, FVLB_EINVAL, "fvlb_create: grid too large for one handle");
  if (!(tau_s > 0.5) || !std::isfinite(tau_s))
    return fail(nullptr, FVLB_EINVAL, "fvlb_create: tau_s must be > 0.5");
  if (!(lambda > 0.0) || !std::isfinite(lambda))
    return fail(nullptr, FVLB_EINVAL, "fvlb_create: lambda must be > 0");
  if (!(eta_p >= 0.0) || !std::isfinite(eta_p))
    return fail(nullptr, FVLB_EINVAL, "fvlb_create: eta_p must be >= 0");
  if (force) {
    if (force->kind < FVLB_FORCE_NONE || force->kind > FVLB_FORCE_COSINE)
      return fail(nullptr, FVLB_EINVAL, "fvlb_create: unknown force kind");
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(force->F0[a]))
        return fail(nullptr, FVLB_EINVAL, "fvlb_create: non-finite force amplitude");
    if (!std::isfinite(force->k) || !std::isfinite(force->omega))
      return fail(nullptr, FVLB_EINVAL, "fvlb_create: non-finite force parameter");
  }
  fvlb_s* h = new (std::nothrow) fvlb_s();
  if (!h) return fail(nullptr, FVLB_ENOMEM, "fvlb_create: out of host memory");
  h->lattice = lattice;
  h->D = lattice == FVLB_D2Q9 ? 2 : 3;
  h->Q = lattice;
  h->C = lattice == FVLB_D2Q9 ? 3 : 6;
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->N = (long long)nx * ny * nz;
  h->pitch = (h->N + 63) / 64 * 64;
  h->tau_s = tau_s;
  h->eta_p = eta_p;
  h->lambda = lambda;
  if (force) h->force = *force;
  else h->force.kind = FVLB_FORCE_NONE;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    delete h;
    cudaGetLastError();
    return fail(nullptr, FVLB_ECUDA, std::string("fvlb_create: no usable CUDA device: ") +
                                         cudaGetErrorString(e));
  }
  *out = h;
  return FVLB_OK;
}

int fvlb_set_walls(fvlb_t h, unsigned mask) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  if (h->allocated) return fail(h, FVLB_ESTATE, "fvlb_set_walls: state already allocated");
  const int n[3] = {h->nx, h->ny, h->nz};
  if (mask >> h->D) return fail(h, FVLB_EINVAL, "fvlb_set_walls: wall on a missing axis");
  for (int a = 0; a < h->D; ++a)
    if (((mask >> a) & 1u) && n[a] < (h->scheme == FVLB_SCHEME_ORIGINAL ? 3 : 2))
      return fail(h, FVLB_EINVAL,
                  "fvlb_set_walls: a walled axis needs >= 2 nodes (>= 3 with the original scheme)");
  h->walls = mask;
  return FVLB_OK;
}

int fvlb_set_scheme(fvlb_t h, int scheme) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  if (scheme != FVLB_SCHEME_PRESENT && scheme != FVLB_SCHEME_ORIGINAL)
    return fail(h, FVLB_EINVAL, "fvlb_set_scheme: unknown scheme");
  if (scheme == FVLB_SCHEME_ORIGINAL) {
    const int n[3] = {h->nx, h->ny, h->nz};
    for (int a = 0; a < h->D; ++a)
      if (((h->walls >> a) & 1u) && n[a] < 3)
        return fail(h, FVLB_EINVAL,
                    "fvlb_set_scheme: the original scheme needs >= 3 nodes across a wall");
    if (h->mlp)
      return fail(h, FVLB_EINVAL, "fvlb_set_scheme: a learned closure is attached");
  }
  h->scheme = scheme;
  return FVLB_OK;
}

int fvlb_set_model(fvlb_t h, int model, double param) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  if (model < FVLB_MODEL_OLDROYD_B || model > FVLB_MODEL_PTT_EXP)
    return fail(h, FVLB_EINVAL, "fvlb_set_model: unknown model");
  if (!(param >= 0.0) || !std::isfinite(param))
    return fail(h, FVLB_EINVAL, "fvlb_set_model: the parameter must be finite and >= 0");
  if (model == FVLB_MODEL_GIESEKUS && param > 1.0)
    return fail(h, FVLB_EINVAL, "fvlb_set_model: the Giesekus mobility must be <= 1");
  if (model != FVLB_MODEL_OLDROYD_B && h->mlp)
    return fail(h, FVLB_EINVAL, "fvlb_set_model: a learned closure is attached");
  h->model = model;
  h->mpar = model == FVLB_MODEL_OLDROYD_B ? 0.0 : param;
  return FVLB_OK;
}

int fvlb_set_precision(fvlb_t h, int storage) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  if (storage < FVLB_FP64 || storage > FVLB_BF16_DEV_SR)
    return fail(h, FVLB_EINVAL, "fvlb_set_precision: unknown storage");
  if (h->allocated) return fail(h, FVLB_ESTATE, "fvlb_set_precision: state already allocated");
  h->storage = storage;
  return FVLB_OK;
}

int fvlb_set_kernel(fvlb_t h, int variant) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  if (variant != FVLB_KERNEL_FUSED && variant != FVLB_KERNEL_SPLIT)
    return fail(h, FVLB_EINVAL, "fvlb_set_kernel: unknown variant");
  if (h->mlp && variant != FVLB_KERNEL_FUSED)
    return fail(h, FVLB_EINVAL, "fvlb_set_kernel: the learned closure needs the fused kernel");
  h->variant = variant;
  return FVLB_OK;
}

int fvlb_set_stream(fvlb_t h, void* stream) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  h->stream = static_cast<cudaStream_t>(stream);
  return FVLB_OK;
}

int fvlb_init_fields(fvlb_t h, const double* u0, const double* p0, const double* A0) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  Range range("fvlb_init_fields");
  int r = ensure_state(h, false);
  if (r != FVLB_OK) return r;
  r = check_poll(h, true);   // a new state: earlier check results no longer apply
  if (r != FVLB_OK) return r;
  h->bad_t = -1;
  return run_init(h, u0, p0, A0);
}

// the original scheme's polymer stress array (C * pitch working-precision
// values) and its divergence (D * pitch), allocated on first need through
// the allocator hooks
static int ensure_taup(fvlb_t h) {
  if (h->scheme != FVLB_SCHEME_ORIGINAL) return FVLB_OK;
  const size_t rb = h->storage == FVLB_FP64 ? 8 : 4;
  if (!h->taup) h->taup = dev_alloc(h, rb * (size_t)h->C * (size_t)h->pitch);
  if (!h->taup) return fail(h, FVLB_ENOMEM, "device allocation of the stress array failed");
  if (!h->fdiv) h->fdiv = dev_alloc(h, rb * (size_t)h->D * (size_t)h->pitch);
  if (!h->fdiv) return fail(h, FVLB_ENOMEM, "device allocation of the stress divergence failed");
  return FVLB_OK;
}

// The periodic finiteness check: collect the result of the pending check
// (waiting for it if `wait`), recording the step of a failure.
static int check_poll(fvlb_t h, bool wait) {
  if (!h->chk_pending) return FVLB_OK;
  cudaError_t e = wait ? cudaEventSynchronize(h->chk_ev) : cudaEventQuery(h->chk_ev);
  if (e == cudaErrorNotReady) return FVLB_OK;
  if (e != cudaSuccess) return cuda_fail(h, e, "finiteness check");
  h->chk_pending = false;
  if (h->chk_host[6] > 0 && h->bad_t < 0) h->bad_t = h->chk_t;
  return FVLB_OK;
}

// The device's record of bounded waits that ran out (set by a step kernel
// whose staged copies did not arrive within its time limit; the state is
// then invalid until the fields are initialised again).  Synchronous.
static int wait_check(fvlb_t h) {
  if (!h->dev_err) return FVLB_OK;
  unsigned v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, h->dev_err, sizeof v, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "device wait record");
  if (v) return fail(h, FVLB_ETIMEOUT, "a step kernel's staged copies did not arrive in time; the state is invalid");
  return FVLB_OK;
}

static int unstable_fail(fvlb_t h) {
  return fail(h, FVLB_EUNSTABLE,
              ("non-finite values in the state (periodic check at step " +
               std::to_string(h->bad_t) + ")").c_str());
}

// Enqueue the diagnostics of the current state and a copy of them to
// page-locked host memory, marked by an event (no host wait).
static int check_enqueue(fvlb_t h) {
  StepDesc d = make_desc(h);
  cudaError_t e = h->lattice == FVLB_D2Q9 ? fvlb::reduce_d2q9(d, h->part, h->red)
                                          : fvlb::reduce_d3q19(d, h->part, h->red);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->chk_host, h->red, sizeof(double) * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(h->chk_ev, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "finiteness check");
  h->chk_pending = true;
  h->chk_t = h->t;
  return FVLB_OK;
}

int fvlb_step(fvlb_t h, long n) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  if (n < 0) return fail(h, FVLB_EINVAL, "fvlb_step: n must be >= 0");
  Range range("fvlb_step");
  int r = ensure_state(h, true);
  if (r != FVLB_OK) return r;
  r = ensure_taup(h);
  if (r != FVLB_OK) return r;
  if (h->chk_every) {
    r = check_poll(h, false);
    if (r != FVLB_OK) return r;
    if (h->bad_t >= 0) return unstable_fail(h);
  }
  for (long k = 0; k < n; ++k) {
    StepDesc d = make_desc(h);
    cudaError_t e = h->lattice == FVLB_D2Q9 ? fvlb::step_d2q9(d) : fvlb::step_d3q19(d);
    if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_step: launch");
    h->cur = 1 - h->cur;
    h->first = 0;
    h->t += 1;
    if (h->chk_every && h->t % h->chk_every == 0) {
      r = check_poll(h, false);
      if (r != FVLB_OK) return r;
      if (h->bad_t >= 0) return unstable_fail(h);
      if (!h->chk_pending) {   // one check in flight at a time
        r = check_enqueue(h);
        if (r != FVLB_OK) return r;
      }
    }
  }
  return FVLB_OK;
}

int fvlb_set_check_interval(fvlb_t h, long every) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  if (every < 0) return fail(h, FVLB_EINVAL, "fvlb_set_check_interval: every must be >= 0");
  if (every) {
    cudaError_t e = cudaSuccess;
    if (!h->chk_host) e = cudaMallocHost(reinterpret_cast<void**>(&h->chk_host), sizeof(double) * 8);
    if (e == cudaSuccess && !h->chk_ev) e = cudaEventCreateWithFlags(&h->chk_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_set_check_interval");
  }
  if (!every) {
    int r = check_poll(h, true);
    if (r != FVLB_OK) return r;
  }
  h->chk_every = every;
  return FVLB_OK;
}

int fvlb_status(fvlb_t h, int wait) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  int r = check_poll(h, wait != 0);
  if (r != FVLB_OK) return r;
  if (wait) {
    r = wait_check(h);
    if (r != FVLB_OK) return r;
  }
  if (h->bad_t >= 0) return unstable_fail(h);
  return FVLB_OK;
}

int fvlb_fields(fvlb_t h, int which, double* host_out, size_t count) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  Range range("fvlb_fields");
  const int nc = comps(h, which);
  if (nc == 0) return fail(h, FVLB_EINVAL, "fvlb_fields: unknown field");
  if (!host_out) return fail(h, FVLB_EINVAL, "fvlb_fields: host_out is NULL");
  const size_t need = (size_t)h->N * nc;
  if (count < need) return fail(h, FVLB_EINVAL, "fvlb_fields: buffer too small");
  int r = ensure_state(h, true);
  if (r != FVLB_OK) return r;
  r = ensure_taup(h);
  if (r != FVLB_OK) return r;
  if (!h->fbuf) {
    h->fbuf = static_cast<double*>(dev_alloc(h, sizeof(double) * (size_t)h->N * std::max(h->D, h->C)));
    if (!h->fbuf) return fail(h, FVLB_ENOMEM, "fvlb_fields: device allocation failed");
  }
  StepDesc d = make_desc(h);
  cudaError_t e = h->lattice == FVLB_D2Q9 ? fvlb::fields_d2q9(d, which, h->fbuf)
                                          : fvlb::fields_d3q19(d, which, h->fbuf);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_out, h->fbuf, sizeof(double) * need, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_fields");
  return wait_check(h);
}

int fvlb_reduce(fvlb_t h, double out[8]) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  Range range("fvlb_reduce");
  if (!out) return fail(h, FVLB_EINVAL, "fvlb_reduce: out is NULL");
  int r = ensure_state(h, true);
  if (r != FVLB_OK) return r;
  r = ensure_taup(h);
  if (r != FVLB_OK) return r;
  StepDesc d = make_desc(h);
  cudaError_t e = h->lattice == FVLB_D2Q9 ? fvlb::reduce_d2q9(d, h->part, h->red)
                                          : fvlb::reduce_d3q19(d, h->part, h->red);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, h->red, sizeof(double) * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_reduce");
  r = wait_check(h);
  if (r != FVLB_OK) return r;
  if (out[6] > 0) return fail(h, FVLB_EUNSTABLE, "fvlb_reduce: non-finite values in the state");
  return FVLB_OK;
}

int fvlb_conformation(fvlb_t h, double out[3]) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  Range range("fvlb_conformation");
  if (!out) return fail(h, FVLB_EINVAL, "fvlb_conformation: out is NULL");
  int r = ensure_state(h, true);
  if (r != FVLB_OK) return r;
  StepDesc d = make_desc(h);
  cudaError_t e = h->lattice == FVLB_D2Q9 ? fvlb::conformation_d2q9(d, h->part, h->red)
                                          : fvlb::conformation_d3q19(d, h->part, h->red);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, h->red, sizeof(double) * 3, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_conformation");
  return FVLB_OK;
}

int fvlb_repair_conformation(fvlb_t h, double eps, long long* repaired) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  Range range("fvlb_repair_conformation");
  if (!(eps > 0.0) || !std::isfinite(eps))
    return fail(h, FVLB_EINVAL, "fvlb_repair_conformation: eps must be finite and > 0");
  int r = ensure_state(h, true);
  if (r != FVLB_OK) return r;
  StepDesc d = make_desc(h);
  // the count reuses the handle's reduction output (8 doubles)
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(h->red);
  cudaError_t e = h->lattice == FVLB_D2Q9 ? fvlb::repair_d2q9(d, eps, cnt)
                                          : fvlb::repair_d3q19(d, eps, cnt);
  unsigned long long host = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, cnt, sizeof(host), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_repair_conformation");
  if (repaired) *repaired = (long long)host;
  return FVLB_OK;
}

int fvlb_set_closure(fvlb_t h, fvlb_mlp_t m, double tol) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  if (m && fvlb::mlp_lattice(m) != h->lattice)
    return fail(h, FVLB_EINVAL, "fvlb_set_closure: network and grid lattices differ");
  if (m && h->storage != FVLB_FP32)
    return fail(h, FVLB_EINVAL, "fvlb_set_closure: the learned closure runs with FP32 storage");
  if (m && !(tol >= 0.0)) return fail(h, FVLB_EINVAL, "fvlb_set_closure: tol must be >= 0");
  if (m && h->variant != FVLB_KERNEL_FUSED)
    return fail(h, FVLB_EINVAL, "fvlb_set_closure: the learned closure needs the fused kernel");
  if (m && h->scheme != FVLB_SCHEME_PRESENT)
    return fail(h, FVLB_EINVAL, "fvlb_set_closure: the learned closure replaces the present scheme's source");
  if (m && h->model != FVLB_MODEL_OLDROYD_B)
    return fail(h, FVLB_EINVAL, "fvlb_set_closure: the learned closure stands for the Oldroyd-B source");
  int r = ensure_state(h, true);
  if (r != FVLB_OK) return r;
  h->mlp = m;
  h->cl_tol = tol;
  cudaError_t e = cudaMemsetAsync(h->cl_count, 0, 2 * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_set_closure");
  return FVLB_OK;
}

int fvlb_closure_stats(fvlb_t h, long long* network_nodes, long long* fallback_nodes) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  if (!h->allocated) {
    if (network_nodes) *network_nodes = 0;
    if (fallback_nodes) *fallback_nodes = 0;
    return FVLB_OK;
  }
  unsigned long long c[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(c, h->cl_count, sizeof(c), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_closure_stats");
  if (network_nodes) *network_nodes = (long long)c[0];
  if (fallback_nodes) *fallback_nodes = (long long)c[1];
  return FVLB_OK;
}

int fvlb_synchronize(fvlb_t h) {
  if (!h) return fail(nullptr, FVLB_EINVAL, "NULL handle");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_synchronize");
  return FVLB_OK;
}

int fvlb_get_time(fvlb_t h, long* t) {
  if (!h || !t) return fail(h, FVLB_EINVAL, "fvlb_get_time: NULL argument");
  *t = (long)h->t;
  return FVLB_OK;
}

int fvlb_state_size(fvlb_t h, size_t* bytes) {
  if (!h || !bytes) return fail(h, FVLB_EINVAL, "fvlb_state_size: NULL argument");
  *bytes = state_bytes(h);
  return FVLB_OK;
}

int fvlb_save_state(fvlb_t h, void* host_buf, size_t bytes) {
  if (!h || !host_buf) return fail(h, FVLB_EINVAL, "fvlb_save_state: NULL argument");
  if (bytes < state_bytes(h)) return fail(h, FVLB_EINVAL, "fvlb_save_state: buffer too small");
  int r = ensure_state(h, true);
  if (r != FVLB_OK) return r;
  StateHeader hd{kStateMagic, h->lattice, h->nx, h->ny, h->nz, h->storage, h->first, h->t, h->pitch, {0, 0}};
  char* p = static_cast<char*>(host_buf);
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  const size_t P = (size_t)h->pitch;
  const size_t bf = fvlb::f_buffer_bytes(h->storage, h->Q, h->D, P),
               bh = fvlb::h_buffer_bytes(h->storage, h->C, h->Q, P),
               bc = chi_bytes(h->storage) * h->C * P;
  cudaError_t e = cudaMemcpyAsync(p, h->f[h->cur], bf, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p + bf, h->h[h->cur], bh, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p + bf + bh, h->chi, bc, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_save_state");
  return FVLB_OK;
}

int fvlb_load_state(fvlb_t h, const void* host_buf, size_t bytes) {
  if (!h || !host_buf) return fail(h, FVLB_EINVAL, "fvlb_load_state: NULL argument");
  if (bytes != state_bytes(h)) return fail(h, FVLB_EINVAL, "fvlb_load_state: size mismatch");
  StateHeader hd;
  std::memcpy(&hd, host_buf, sizeof(hd));
  if (hd.magic != kStateMagic || hd.lattice != h->lattice || hd.nx != h->nx || hd.ny != h->ny ||
      hd.nz != h->nz || hd.storage != h->storage || hd.pitch != h->pitch)
    return fail(h, FVLB_EINVAL, "fvlb_load_state: header does not match this handle");
  int r = ensure_state(h, false);
  if (r != FVLB_OK) return r;
  r = check_poll(h, true);   // a new state: earlier check results no longer apply
  if (r != FVLB_OK) return r;
  h->bad_t = -1;
  const char* p = static_cast<const char*>(host_buf) + sizeof(hd);
  const size_t P = (size_t)h->pitch;
  const size_t bf = fvlb::f_buffer_bytes(h->storage, h->Q, h->D, P),
               bh = fvlb::h_buffer_bytes(h->storage, h->C, h->Q, P),
               bc = chi_bytes(h->storage) * h->C * P;
  cudaError_t e = cudaMemcpyAsync(h->f[h->cur], p, bf, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h[h->cur], p + bf, bh, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->chi, p + bf + bh, bc, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && h->dev_err) e = cudaMemsetAsync(h->dev_err, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fvlb_load_state");
  h->first = hd.first;
  h->t = hd.t;
  return FVLB_OK;
}

int fvlb_bytes_per_update(fvlb_t h, double* bytes) {
  if (!h || !bytes) return fail(h, FVLB_EINVAL, "fvlb_bytes_per_update: NULL argument");
  *bytes = fvlb::bytes_per_update(h->storage, h->Q, h->C, h->D);
  return FVLB_OK;
}

const char* fvlb_last_error(fvlb_t h) {
  if (h) return h->err.c_str();
  return g_err.c_str();
}

int fvlb_destroy(fvlb_t h) {
  if (!h) return FVLB_OK;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  if (h->chk_ev) cudaEventDestroy(h->chk_ev);
  if (h->chk_host) cudaFreeHost(h->chk_host);
  delete h;
  return FVLB_OK;
}

}  // extern "C"
