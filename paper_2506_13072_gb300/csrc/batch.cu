// batch.cu -- C ABI of the batched persistent step (fvlb_batch_* in fvlb.h):
// many independent D2Q9 grids of uneven size and parameters advanced by one
// kernel launch per step, the steps replayed from a captured CUDA graph, and
// the tile shape chosen by timing the candidates on the batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fvlb.h"
#include "fvlb_batch_impl.cuh"

namespace fvlb {
#define FVLB_EXTERN_BATCH(S)                                                             \
  extern template cudaError_t batch_step_impl<S>(const BatchLaunch&);                    \
  extern template int batch_occupancy_impl<S>(int);                                      \
  extern template void batch_inst_fill_impl<S>(void*, int, int, int, long long, double,  \
                                               double, double, double, int, const double*, \
                                               double, const void*, long long, long long,  \
                                               long long);
FVLB_EXTERN_BATCH(double)
FVLB_EXTERN_BATCH(float)
FVLB_EXTERN_BATCH(__half)
FVLB_EXTERN_BATCH(__nv_bfloat16)
#undef FVLB_EXTERN_BATCH

cudaError_t batch_step(const BatchLaunch& d) {
  switch (d.storage) {
    case kFP64: return batch_step_impl<double>(d);
    case kFP32: return batch_step_impl<float>(d);
    case kFP16Dev: return batch_step_impl<__half>(d);
    case kBF16Dev: return batch_step_impl<__nv_bfloat16>(d);
    default: return cudaErrorInvalidValue;
  }
}

int batch_occupancy(int storage, int gx) {
  switch (storage) {
    case kFP64: return batch_occupancy_impl<double>(gx);
    case kFP32: return batch_occupancy_impl<float>(gx);
    case kFP16Dev: return batch_occupancy_impl<__half>(gx);
    default: return batch_occupancy_impl<__nv_bfloat16>(gx);
  }
}

size_t batch_inst_size(int storage) {
  switch (storage) {
    case kFP64: return sizeof(BatchInst<double>);
    case kFP32: return sizeof(BatchInst<float>);
    case kFP16Dev: return sizeof(BatchInst<__half>);
    default: return sizeof(BatchInst<__nv_bfloat16>);
  }
}

void batch_inst_fill(int storage, void* dst, int nx, int ny, int walls, long long pitch,
                     double tau_f, double tau_h, double eta_p, double lambda, int force_kind,
                     const double F0[3], double omega, const void* tables, long long f_off,
                     long long h_off, long long chi_off) {
#define FILL(S)                                                                             \
  batch_inst_fill_impl<S>(dst, nx, ny, walls, pitch, tau_f, tau_h, eta_p, lambda, force_kind, \
                          F0, omega, tables, f_off, h_off, chi_off)
  switch (storage) {
    case kFP64: FILL(double); break;
    case kFP32: FILL(float); break;
    case kFP16Dev: FILL(__half); break;
    default: FILL(__nv_bfloat16); break;
  }
#undef FILL
}

cudaError_t batch_advance(long long* t, cudaStream_t stream) {
  k_advance_step<<<1, 1, 0, stream>>>(t);
  return cudaGetLastError();
}

}  // namespace fvlb

using namespace fvlb;

namespace {

constexpr int kQ = 9, kC = 3, kD = 2;
// tile shapes the autotuner times: 32 GX nodes along x, mchunk rows
constexpr int kGx[] = {1, 2, 4};
constexpr int kChunk[] = {8, 16, 32};

size_t sbytes(int storage) { return storage == FVLB_FP64 ? 8 : (storage == FVLB_FP32 ? 4 : 2); }
size_t xbytes(int storage) { return storage == FVLB_FP64 ? 8 : 4; }

}  // namespace

struct fvlb_batch_s {
  int storage = FVLB_FP32;
  int count = 0;
  std::vector<fvlb_instance> spec;
  std::vector<long long> N, pitch, f_off, h_off, chi_off, tab_off;
  long long f_total = 0, h_total = 0, chi_total = 0, tab_total = 0, Nmax = 0, sites = 0;
  void *fA = nullptr, *fB = nullptr, *hA = nullptr, *hB = nullptr, *chi = nullptr;
  void* tables = nullptr;
  void* inst = nullptr;
  void* tiles = nullptr;
  int tiles_cap = 0;
  long long* tdev = nullptr;
  double* fbuf = nullptr;
  int parity = 0, first = 1;
  long long t = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int gx = 4, mchunk = 16, ntiles = 0, blocks = 0;
  bool tuned = false;
  double tuned_ms = 0.0;
  cudaGraphExec_t graph = nullptr;
  int graph_parity = -1;
  fvlb_alloc_fn alloc = nullptr;
  fvlb_free_fn free_ = nullptr;
  void* actx = nullptr;
  std::vector<void*> owned;
  std::string err;
};

namespace {

int bfail(fvlb_batch_t b, int code, const std::string& msg) {
  if (b) b->err = msg;
  else set_global_error(code, msg.c_str());
  return code;
}

void* balloc(fvlb_batch_t b, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (b->alloc) p = b->alloc(bytes, b->actx);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) b->owned.push_back(p);
  return p;
}

void bfree_all(fvlb_batch_t b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  for (void* p : b->owned) {
    if (b->free_) b->free_(p, b->actx);
    else cudaFree(p);
  }
  b->owned.clear();
}

// tile list of a shape: every instance's x tiles and row chunks, largest
// instances first
std::vector<BatchTile> make_tiles(fvlb_batch_t b, int gx, int mchunk) {
  std::vector<int> order(b->count);
  for (int i = 0; i < b->count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->N[a] > b->N[c]; });
  std::vector<BatchTile> tl;
  const int txs = 32 * gx;
  for (int i : order) {
    const int bxn = (b->spec[i].nx + txs - 1) / txs;
    const int bzn = (b->spec[i].ny + mchunk - 1) / mchunk;
    for (int bz = 0; bz < bzn; ++bz)
      for (int bx = 0; bx < bxn; ++bx) tl.push_back(BatchTile{i, bx, bz});
  }
  return tl;
}

int upload_tiles(fvlb_batch_t b, int gx, int mchunk) {
  std::vector<BatchTile> tl = make_tiles(b, gx, mchunk);
  if ((int)tl.size() > b->tiles_cap) return bfail(b, FVLB_ENOMEM, "tile list larger than reserved");
  cudaError_t e = cudaMemcpyAsync(b->tiles, tl.data(), tl.size() * sizeof(BatchTile),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, FVLB_ECUDA, std::string("tile upload: ") + cudaGetErrorString(e));
  b->gx = gx;
  b->mchunk = mchunk;
  b->ntiles = (int)tl.size();
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per = batch_occupancy(b->storage, gx);
  b->blocks = sms * (per > 0 ? per : 1);
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return FVLB_OK;
}

BatchLaunch make_launch(fvlb_batch_t b) {
  BatchLaunch d{};
  d.storage = b->storage;
  d.gx = b->gx;
  d.inst = b->inst;
  d.tiles = b->tiles;
  d.ntiles = b->ntiles;
  d.fA = b->fA;
  d.fB = b->fB;
  d.hA = b->hA;
  d.hB = b->hB;
  d.chi = b->chi;
  d.parity = b->parity;
  d.first = b->first;
  d.tstep = b->tdev;
  d.mchunk = b->mchunk;
  d.blocks = b->blocks;
  d.stream = b->stream;
  return d;
}

// one step launched directly (first step, odd remainders, tuning)
int direct_step(fvlb_batch_t b) {
  BatchLaunch d = make_launch(b);
  cudaError_t e = batch_step(d);
  if (e == cudaSuccess) e = batch_advance(b->tdev, b->stream);
  if (e != cudaSuccess) return bfail(b, FVLB_ECUDA, std::string("batched step: ") + cudaGetErrorString(e));
  b->parity ^= 1;
  b->first = 0;
  b->t += 1;
  return FVLB_OK;
}

// two steps (parity p, then 1 - p) captured once into a graph
int build_graph(fvlb_batch_t b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(b, FVLB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  for (int q = 0; q < 2; ++q) {
    BatchLaunch d = make_launch(b);
    d.parity = b->parity ^ q;
    d.first = 0;
    if (e == cudaSuccess) e = batch_step(d);
    if (e == cudaSuccess) e = batch_advance(b->tdev, b->stream);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return bfail(b, FVLB_ECUDA, std::string("graph build: ") + cudaGetErrorString(e));
  }
  b->graph_parity = b->parity;
  return FVLB_OK;
}

// time each candidate shape over two real steps (the update of every node
// is identical whatever the shape, so tuning steps are ordinary steps)
int autotune(fvlb_batch_t b) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  int bgx = b->gx, bch = b->mchunk;
  for (int gx : kGx)
    for (int ch : kChunk) {
      int r = upload_tiles(b, gx, ch);
      if (r != FVLB_OK) return r;
      cudaEventRecord(e0, b->stream);
      for (int q = 0; q < 2; ++q) {
        r = direct_step(b);
        if (r != FVLB_OK) return r;
      }
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bgx = gx;
        bch = ch;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tuned = true;
  b->tuned_ms = best / 2.0;
  return upload_tiles(b, bgx, bch);
}

int init_instance(fvlb_batch_t b, int i, const double* u0, const double* p0, const double* A0) {
  const size_t N = (size_t)b->N[i];
  const size_t nu = u0 ? N * kD : 0, np = p0 ? N : 0, nA = A0 ? N * kC : 0;
  double* tmp = b->fbuf;  // N_max * 6 doubles of scratch
  cudaError_t e = cudaSuccess;
  if (u0) e = cudaMemcpyAsync(tmp, u0, sizeof(double) * nu, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && p0)
    e = cudaMemcpyAsync(tmp + nu, p0, sizeof(double) * np, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && A0)
    e = cudaMemcpyAsync(tmp + nu + np, A0, sizeof(double) * nA, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) {
    InitDesc d{};
    d.nx = b->spec[i].nx;
    d.ny = b->spec[i].ny;
    d.nz = 1;
    d.N = b->N[i];
    d.pitch = b->pitch[i];
    d.storage = b->storage;
    const size_t sb = sbytes(b->storage), xb = xbytes(b->storage);
    char* fcur = static_cast<char*>(b->parity ? b->fB : b->fA);
    char* hcur = static_cast<char*>(b->parity ? b->hB : b->hA);
    d.f = fcur + sb * b->f_off[i];
    d.h = hcur + sb * b->h_off[i];
    d.chi = static_cast<char*>(b->chi) + xb * b->chi_off[i];
    d.u0 = u0 ? tmp : nullptr;
    d.p0 = p0 ? tmp + nu : nullptr;
    d.A0 = A0 ? tmp + nu + np : nullptr;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    d.sms = sms;
    d.stream = b->stream;
    e = init_d2q9(d);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, FVLB_ECUDA, std::string("batch init: ") + cudaGetErrorString(e));
  return FVLB_OK;
}

}  // namespace

extern "C" {

int fvlb_batch_create(fvlb_batch_t* out, int lattice, int count, const fvlb_instance* specs,
                      int storage) {
  if (!out) return set_global_error(FVLB_EINVAL, "fvlb_batch_create: out is NULL");
  *out = nullptr;
  if (lattice != FVLB_D2Q9)
    return set_global_error(FVLB_EINVAL, "fvlb_batch_create: batches are D2Q9");
  if (count < 1 || !specs) return set_global_error(FVLB_EINVAL, "fvlb_batch_create: no instances");
  if (storage < FVLB_FP64 || storage > FVLB_BF16_DEV)
    return set_global_error(FVLB_EINVAL, "fvlb_batch_create: storage must be FP64, FP32, FP16_DEV or BF16_DEV");
  for (int i = 0; i < count; ++i) {
    const fvlb_instance& s = specs[i];
    if (s.nx < 1 || s.ny < 1 || !(s.tau_s > 0.5) || !(s.lambda > 0) || !(s.eta_p >= 0) ||
        !std::isfinite(s.tau_s) || !std::isfinite(s.lambda) || !std::isfinite(s.eta_p))
      return set_global_error(FVLB_EINVAL, "fvlb_batch_create: invalid instance parameters");
    if (s.force.kind < FVLB_FORCE_NONE || s.force.kind > FVLB_FORCE_COSINE)
      return set_global_error(FVLB_EINVAL, "fvlb_batch_create: unknown force kind");
    if ((s.walls >> 2) || ((s.walls & 1) && s.nx < 2) || ((s.walls & 2) && s.ny < 2))
      return set_global_error(FVLB_EINVAL, "fvlb_batch_create: invalid walls");
    if ((long long)kQ * (((long long)s.nx * s.ny + 63) / 64 * 64) >= (1ll << 32))
      return set_global_error(FVLB_EINVAL, "fvlb_batch_create: instance too large");
  }
  fvlb_batch_s* b = new (std::nothrow) fvlb_batch_s();
  if (!b) return set_global_error(FVLB_ENOMEM, "fvlb_batch_create: out of host memory");
  b->storage = storage;
  b->count = count;
  b->spec.assign(specs, specs + count);
  current_allocator(&b->alloc, &b->free_, &b->actx);
  for (int i = 0; i < count; ++i) {
    const long long N = (long long)specs[i].nx * specs[i].ny;
    const long long P = (N + 63) / 64 * 64;
    b->N.push_back(N);
    b->pitch.push_back(P);
    b->f_off.push_back(b->f_total);
    b->h_off.push_back(b->h_total);
    b->chi_off.push_back(b->chi_total);
    b->tab_off.push_back(b->tab_total);
    // (16-bit forms: each grid's buffers end with its FP32 arrays, U[D][P]
    // and h0[C][P], counted here in 2-byte elements)
    const long long ext = fvlb::v2_storage(storage) ? 2 : 0;
    b->f_total += kQ * P + ext * kD * P;
    b->h_total += (long long)kC * kQ * P + ext * kC * P;
    b->chi_total += kC * P;
    if (specs[i].force.kind == FVLB_FORCE_FOUR_ROLL) b->tab_total += 2 * (specs[i].nx + specs[i].ny);
    b->Nmax = std::max(b->Nmax, N);
    b->sites += N;
  }
  const size_t sb = sbytes(storage), xb = xbytes(storage), rb = storage == FVLB_FP64 ? 8 : 4;
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return set_global_error(FVLB_ECUDA, "fvlb_batch_create: stream creation failed");
  }
  b->own_stream = true;
  b->fA = balloc(b, sb * b->f_total);
  b->fB = balloc(b, sb * b->f_total);
  b->hA = balloc(b, sb * b->h_total);
  b->hB = balloc(b, sb * b->h_total);
  b->chi = balloc(b, xb * b->chi_total);
  b->tables = b->tab_total ? balloc(b, rb * b->tab_total) : nullptr;
  b->inst = balloc(b, batch_inst_size(storage) * count);
  // the finest shape (32 nodes x 8 rows) has the most tiles
  b->tiles_cap = (int)make_tiles(b, 1, 8).size();
  b->tiles = balloc(b, sizeof(BatchTile) * b->tiles_cap);
  b->tdev = static_cast<long long*>(balloc(b, sizeof(long long)));
  b->fbuf = static_cast<double*>(balloc(b, sizeof(double) * 6 * b->Nmax));
  if (!b->fA || !b->fB || !b->hA || !b->hB || !b->chi || !b->inst || !b->tiles || !b->tdev ||
      !b->fbuf || (b->tab_total && !b->tables)) {
    bfree_all(b);
    cudaStreamDestroy(b->stream);
    delete b;
    return set_global_error(FVLB_ENOMEM, "fvlb_batch_create: device allocation failed");
  }
  // per-instance descriptors and four-roll tables
  std::vector<char> inst(batch_inst_size(storage) * count);
  std::vector<double> tab(b->tab_total);
  for (int i = 0; i < count; ++i) {
    const fvlb_instance& s = specs[i];
    const void* tptr = nullptr;
    if (s.force.kind == FVLB_FORCE_FOUR_ROLL) {
      double* t = tab.data() + b->tab_off[i];
      for (int x = 0; x < s.nx; ++x) {
        t[x] = std::sin(s.force.k * x);
        t[s.nx + x] = std::cos(s.force.k * x);
      }
      for (int y = 0; y < s.ny; ++y) {
        t[2 * s.nx + y] = std::sin(s.force.k * y);
        t[2 * s.nx + s.ny + y] = std::cos(s.force.k * y);
      }
      tptr = static_cast<char*>(b->tables) + rb * b->tab_off[i];
    }
    batch_inst_fill(storage, inst.data() + batch_inst_size(storage) * i, s.nx, s.ny, (int)s.walls,
                    b->pitch[i], s.tau_s, 0.501, s.eta_p, s.lambda, s.force.kind, s.force.F0,
                    s.force.omega, tptr, b->f_off[i], b->h_off[i], b->chi_off[i]);
  }
  e = cudaMemcpy(b->inst, inst.data(), inst.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && b->tab_total) {
    if (rb == 8) {
      e = cudaMemcpy(b->tables, tab.data(), 8 * tab.size(), cudaMemcpyHostToDevice);
    } else {
      std::vector<float> tf(tab.begin(), tab.end());
      e = cudaMemcpy(b->tables, tf.data(), 4 * tf.size(), cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) e = cudaMemset(b->tdev, 0, sizeof(long long));
  if (e != cudaSuccess) {
    bfree_all(b);
    cudaStreamDestroy(b->stream);
    delete b;
    return set_global_error(FVLB_ECUDA, "fvlb_batch_create: upload failed");
  }
  int r = upload_tiles(b, 4, 16);
  for (int i = 0; r == FVLB_OK && i < count; ++i) r = init_instance(b, i, nullptr, nullptr, nullptr);
  if (r != FVLB_OK) {
    std::string msg = b->err;
    bfree_all(b);
    cudaStreamDestroy(b->stream);
    delete b;
    return set_global_error(r, msg.c_str());
  }
  *out = b;
  return FVLB_OK;
}

int fvlb_batch_set_stream(fvlb_batch_t b, void* stream) {
  if (!b) return set_global_error(FVLB_EINVAL, "NULL batch");
  if (!stream) return bfail(b, FVLB_EINVAL, "fvlb_batch_set_stream: a capturable (non-NULL) stream is needed");
  cudaStreamSynchronize(b->stream);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->own_stream = false;
  b->stream = static_cast<cudaStream_t>(stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  return FVLB_OK;
}

int fvlb_batch_init_fields(fvlb_batch_t b, int index, const double* u0, const double* p0,
                           const double* A0) {
  if (!b) return set_global_error(FVLB_EINVAL, "NULL batch");
  if (index < 0 || index >= b->count) return bfail(b, FVLB_EINVAL, "fvlb_batch_init_fields: bad index");
  if (b->t != 0) return bfail(b, FVLB_ESTATE, "fvlb_batch_init_fields: the batch has already stepped");
  return init_instance(b, index, u0, p0, A0);
}

int fvlb_batch_step(fvlb_batch_t b, long n) {
  nvtxRangePushA("fvlb_batch_step");   // one range over the whole call (graph replays)
  struct Pop { ~Pop() { nvtxRangePop(); } } pop;
  if (!b) return set_global_error(FVLB_EINVAL, "NULL batch");
  if (n < 0) return bfail(b, FVLB_EINVAL, "fvlb_batch_step: n must be >= 0");
  int r = FVLB_OK;
  if (n > 0 && b->first) {
    r = direct_step(b);
    --n;
  }
  const long ntune = 2L * (sizeof(kGx) / sizeof(int)) * (sizeof(kChunk) / sizeof(int));
  if (r == FVLB_OK && !b->tuned && n >= ntune) {
    r = autotune(b);
    n -= ntune;
  }
  while (r == FVLB_OK && n > 0) {
    if (n >= 2 && b->tuned) {
      if (!b->graph || b->graph_parity != b->parity) r = build_graph(b);
      if (r != FVLB_OK) break;
      cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
      if (e != cudaSuccess) return bfail(b, FVLB_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
      b->t += 2;
      n -= 2;
    } else {
      r = direct_step(b);
      --n;
    }
  }
  return r;
}

int fvlb_batch_fields(fvlb_batch_t b, int index, int which, double* host_out, size_t count) {
  if (!b) return set_global_error(FVLB_EINVAL, "NULL batch");
  if (index < 0 || index >= b->count) return bfail(b, FVLB_EINVAL, "fvlb_batch_fields: bad index");
  const int nc = which == FVLB_FIELD_U ? kD : (which == FVLB_FIELD_P ? 1 : (which == FVLB_FIELD_A || which == FVLB_FIELD_TAU_P ? kC : 0));
  if (nc == 0) return bfail(b, FVLB_EINVAL, "fvlb_batch_fields: unknown field");
  if (!host_out || count < (size_t)b->N[index] * nc) return bfail(b, FVLB_EINVAL, "fvlb_batch_fields: buffer too small");
  const fvlb_instance& s = b->spec[index];
  const size_t sb = sbytes(b->storage), xb = xbytes(b->storage), rb = b->storage == FVLB_FP64 ? 8 : 4;
  StepDesc d{};
  d.nx = s.nx;
  d.ny = s.ny;
  d.nz = 1;
  d.walls = (int)s.walls;
  d.N = b->N[index];
  d.pitch = b->pitch[index];
  d.storage = b->storage;
  d.f_in = static_cast<char*>(b->parity ? b->fB : b->fA) + sb * b->f_off[index];
  d.h_in = static_cast<char*>(b->parity ? b->hB : b->hA) + sb * b->h_off[index];
  d.chi = static_cast<char*>(b->chi) + xb * b->chi_off[index];
  d.tau_f = s.tau_s;
  d.tau_h = 0.501;
  d.eta_p = s.eta_p;
  d.lambda = s.lambda;
  d.four_roll = s.force.kind == FVLB_FORCE_FOUR_ROLL;
  d.amp = s.force.F0[0];
  d.tables = d.four_roll ? static_cast<char*>(b->tables) + rb * b->tab_off[index] : nullptr;
  const double c = s.force.kind == FVLB_FORCE_CONST ? 1.0
                   : s.force.kind == FVLB_FORCE_COSINE ? std::cos(s.force.omega * (double)b->t) : 0.0;
  for (int a = 0; a < 3; ++a) d.Fv[a] = a < kD ? s.force.F0[a] * c : 0.0;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  d.sms = sms;
  d.stream = b->stream;
  cudaError_t e = fields_d2q9(d, which, b->fbuf);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_out, b->fbuf, sizeof(double) * b->N[index] * nc, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, FVLB_ECUDA, std::string("fvlb_batch_fields: ") + cudaGetErrorString(e));
  return FVLB_OK;
}

int fvlb_batch_info(fvlb_batch_t b, long long* sites, double* bytes_per_update, int* gx,
                    int* rows, double* tuned_ms_per_step) {
  if (!b) return set_global_error(FVLB_EINVAL, "NULL batch");
  if (sites) *sites = b->sites;
  if (bytes_per_update)
    *bytes_per_update = fvlb::bytes_per_update(b->storage, kQ, kC, kD);
  if (gx) *gx = b->gx;
  if (rows) *rows = b->mchunk;
  if (tuned_ms_per_step) *tuned_ms_per_step = b->tuned ? b->tuned_ms : 0.0;
  return FVLB_OK;
}

int fvlb_batch_synchronize(fvlb_batch_t b) {
  if (!b) return set_global_error(FVLB_EINVAL, "NULL batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, FVLB_ECUDA, std::string("fvlb_batch_synchronize: ") + cudaGetErrorString(e));
  return FVLB_OK;
}

int fvlb_batch_get_time(fvlb_batch_t b, long* t) {
  if (!b || !t) return set_global_error(FVLB_EINVAL, "fvlb_batch_get_time: NULL argument");
  *t = (long)b->t;
  return FVLB_OK;
}

const char* fvlb_batch_last_error(fvlb_batch_t b) {
  if (!b) return fvlb_last_error(nullptr);
  return b->err.c_str();
}

int fvlb_batch_destroy(fvlb_batch_t b) {
  if (!b) return FVLB_OK;
  cudaStreamSynchronize(b->stream);
  bfree_all(b);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return FVLB_OK;
}

}  // extern "C"
