// mlp.cu -- the learned stress closure: training-pair collection from the
// plain method's state, GPU training of the network (hand-written forward,
// backward and Adam kernels), FP16 packing, tensor-core inference, and the
// fvlb_mlp_* C ABI.  Applying the network inside the step is in
// k_step_fused (fvlb_set_closure).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "fvlb.h"
#include "fvlb_internal.h"
#include "fvlb_launch.cuh"
#include "fvlb_mlp.cuh"

namespace fvlb {

// ---------------------------------------------------------------------------
// Training pairs from the current state of a grid (the plain method).
// For every stride-th node s: x = (lambda grad u, A - I, [dt/lambda]) and
// target y = lambda chi, with grad u and chi exactly as the step forms them.
// ---------------------------------------------------------------------------
template <class L, class S>
__device__ void node_velocity(const Grid& g, const Phys<RT<S>>& ph, const S* __restrict__ f,
                              int x, int y, int z, RT<S> (&u)[L::D]) {
  using R = RT<S>;
  const long long s = ((long long)z * g.ny + y) * g.nx + x;
  R fv[L::Q];
  load_f<L, S>(f, g.pitch, s, fv);
  R F[3];
  body_force<L, R>(ph, x, y, F);
  velocity<L, R>(fv, F, u);
}

template <class L, class S>
__global__ void k_closure_pairs(Grid g, Phys<RT<S>> ph, const S* __restrict__ f,
                                const S* __restrict__ h, long long N, long long stride,
                                long long npairs, float* __restrict__ X, float* __restrict__ T,
                                double lam) {
  using R = RT<S>;
  constexpr int D = L::D, Q = L::Q, C = L::C;
  constexpr int IN = MlpDims<D>::IN, OUT = MlpDims<D>::OUT;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < npairs;
       j += (long long)gridDim.x * blockDim.x) {
    const long long s = (j * stride) % N;
    const int p[3] = {(int)(s % g.nx), (int)((s / g.nx) % g.ny), (int)(s / ((long long)g.nx * g.ny))};
    const int n[3] = {g.nx, g.ny, g.nz};
    R u[D];
    node_velocity<L, S>(g, ph, f, p[0], p[1], p[2], u);
    R gr[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int qp[3] = {p[0], p[1], p[2]}, qm[3] = {p[0], p[1], p[2]};
      qp[a] = (p[a] + 1) % n[a];
      qm[a] = (p[a] - 1 + n[a]) % n[a];
      R up[D], um[D];
      node_velocity<L, S>(g, ph, f, qp[0], qp[1], qp[2], up);
      node_velocity<L, S>(g, ph, f, qm[0], qm[1], qm[2], um);
      const bool wall = (g.walls >> a) & 1;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        R d = R(0.5) * (up[b] - um[b]);
        if (wall && p[a] == 0) d = u[b] + up[b] * R(1.0 / 3.0);
        if (wall && p[a] == n[a] - 1) d = -(u[b] + um[b] * R(1.0 / 3.0));
        gr[a][b] = d;
      }
    }
    R Ad[C], A[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
      R a = R(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) a += load_h<L, S>(h, g.pitch, s, k, i);
      Ad[k] = a;
      A[k] = a + (diag<L>(k) ? R(1) : R(0));
    }
    R chi[C];
    chi_tensor<L, R>(A, Ad, gr, ph, chi);
    float* xr = X + j * IN;
    int q = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) xr[q++] = float(lam * double(gr[a][b]));
#pragma unroll
    for (int k = 0; k < C; ++k) xr[q++] = float(Ad[k]);
    if (D == 2) xr[q++] = float(1.0 / lam);
    float* tr = T + j * OUT;
#pragma unroll
    for (int k = 0; k < C; ++k) tr[k] = float(lam * double(chi[k]));
  }
}

// ---------------------------------------------------------------------------
// Training: per-sample forward and backward (one thread per sample, 64
// samples per block), then per-block weight gradients by fixed-order sums
// over the block's samples (deterministic), written as partials.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gelu_acc(float z, float* dz) {
  const float c = 0.7978845608028654f;
  const float u = c * (z + 0.044715f * z * z * z);
  const float th = tanhf(u);
  if (dz) *dz = 0.5f * (1.0f + th) + 0.5f * z * (1.0f - th * th) * c * (1.0f + 3.0f * 0.044715f * z * z);
  return 0.5f * z * (1.0f + th);
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  return hash32(x);
}

constexpr int kTB = 64;  // samples per training block

template <int IN, int OUT>
__global__ void __launch_bounds__(kTB)
    k_mlp_grad(const float* __restrict__ prm, const float* __restrict__ X,
               const float* __restrict__ T, long long count, long long n, int sample_seed,
               long long batch_base, float delta2, float* __restrict__ part,
               float* __restrict__ part_loss) {
  using PP = MlpParams<IN, OUT>;
  constexpr int H = kMlpH;
  extern __shared__ float sm[];
  float* W = sm;                          // PP::N
  float* xs = W + PP::N;                  // [kTB][IN]
  float* z1 = xs + kTB * IN;              // [kTB][H+1]  (z1, then dz1)
  float* h1 = z1 + kTB * (H + 1);         // [kTB][H+1]
  float* z2 = h1 + kTB * (H + 1);         // [kTB][H+1]  (z2, then dz2)
  float* h2 = z2 + kTB * (H + 1);         // [kTB][H+1]
  float* dy = h2 + kTB * (H + 1);         // [kTB][OUT]
  constexpr int LD = H + 1;
  const int tid = threadIdx.x;
  for (int i = tid; i < PP::N; i += kTB) W[i] = prm[i];
  const long long gi = batch_base + blockIdx.x * (long long)kTB + tid;
  const bool valid = gi < batch_base + n;
  long long src = 0;
  if (valid) {
    src = sample_seed >= 0
              ? (long long)(((uint64_t)mix32((uint32_t)gi * 0x9e3779b9u ^ mix32((uint32_t)sample_seed)) *
                             (uint64_t)count) >> 32)
              : gi;
  }
  for (int k = 0; k < IN; ++k) xs[tid * IN + k] = valid ? X[src * IN + k] : 0.f;
  __syncthreads();
  // forward
  float loss = 0.f;
  for (int j = 0; j < H; ++j) {
    float a = W[PP::B1 + j];
    for (int k = 0; k < IN; ++k) a += W[PP::W1 + j * IN + k] * xs[tid * IN + k];
    z1[tid * LD + j] = a;
    h1[tid * LD + j] = gelu_acc(a, nullptr);
  }
  for (int j = 0; j < H; ++j) {
    float a = W[PP::B2 + j];
    for (int k = 0; k < H; ++k) a += W[PP::W2 + j * H + k] * h1[tid * LD + k];
    z2[tid * LD + j] = a;
    h2[tid * LD + j] = gelu_acc(a, nullptr);
  }
  // sample weight: 1, or 1 / (mean_o t_o^2 + delta^2) for the relative loss
  float wgt = 1.f;
  if (delta2 > 0.f && valid) {
    float tt = 0.f;
    for (int o = 0; o < OUT; ++o) tt += T[src * OUT + o] * T[src * OUT + o];
    wgt = 1.f / (tt / float(OUT) + delta2);
  }
  const float scale = 2.0f * wgt / (float(n) * float(OUT));
  for (int o = 0; o < OUT; ++o) {
    float y = W[PP::B3 + o];
    for (int k = 0; k < H; ++k) y += W[PP::W3 + o * H + k] * h2[tid * LD + k];
    const float r = valid ? y - T[src * OUT + o] : 0.f;
    loss += wgt * r * r;
    dy[tid * OUT + o] = scale * r;
  }
  // backward through layer 3 and GELU: dz2 (stored over z2)
  for (int i = 0; i < H; ++i) {
    float d = 0.f;
    for (int o = 0; o < OUT; ++o) d += W[PP::W3 + o * H + i] * dy[tid * OUT + o];
    float dg;
    gelu_acc(z2[tid * LD + i], &dg);
    z2[tid * LD + i] = d * dg;
  }
  // through layer 2: dz1 (stored over z1)
  for (int k = 0; k < H; ++k) {
    float d = 0.f;
    for (int i = 0; i < H; ++i) d += W[PP::W2 + i * H + k] * z2[tid * LD + i];
    float dg;
    gelu_acc(z1[tid * LD + k], &dg);
    z1[tid * LD + k] = d * dg;
  }
  __syncthreads();
  // block partial gradients, fixed summation order over samples
  float* out = part + (long long)blockIdx.x * PP::N;
  for (int e = tid; e < PP::N; e += kTB) {
    float acc = 0.f;
    if (e < PP::B1) {  // W1[j][k] = sum_s dz1[s][j] x[s][k]
      const int j = e / IN, k = e % IN;
      for (int s = 0; s < kTB; ++s) acc += z1[s * LD + j] * xs[s * IN + k];
    } else if (e < PP::W2) {
      const int j = e - PP::B1;
      for (int s = 0; s < kTB; ++s) acc += z1[s * LD + j];
    } else if (e < PP::B2) {  // W2[i][k] = sum_s dz2[s][i] h1[s][k]
      const int i = (e - PP::W2) / H, k = (e - PP::W2) % H;
      for (int s = 0; s < kTB; ++s) acc += z2[s * LD + i] * h1[s * LD + k];
    } else if (e < PP::W3) {
      const int i = e - PP::B2;
      for (int s = 0; s < kTB; ++s) acc += z2[s * LD + i];
    } else if (e < PP::B3) {  // W3[o][i] = sum_s dy[s][o] h2[s][i]
      const int o = (e - PP::W3) / H, i = (e - PP::W3) % H;
      for (int s = 0; s < kTB; ++s) acc += dy[s * OUT + o] * h2[s * LD + i];
    } else {
      const int o = e - PP::B3;
      for (int s = 0; s < kTB; ++s) acc += dy[s * OUT + o];
    }
    out[e] = acc;
  }
  // block loss, fixed order
  __shared__ float sl[kTB];
  sl[tid] = loss;
  __syncthreads();
  if (tid == 0) {
    float a = 0.f;
    for (int s = 0; s < kTB; ++s) a += sl[s];
    part_loss[blockIdx.x] = a;
  }
}

// Sum the block partials (fixed order) into grad[] (and the loss); if adam,
// apply one Adam step to the FP32 master parameters.
__global__ void k_mlp_update(float* __restrict__ prm, float* __restrict__ mo,
                             float* __restrict__ ve, const float* __restrict__ part,
                             const float* __restrict__ part_loss, int nblocks, int nparam,
                             float* __restrict__ grad, double* __restrict__ loss, double loss_scale,
                             int adam, float lr, float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) {
    double a = 0.0;
    for (int b = 0; b < nblocks; ++b) a += part_loss[b];
    *loss = a * loss_scale;
  }
  if (p >= nparam) return;
  float g = 0.f;
  for (int b = 0; b < nblocks; ++b) g += part[(long long)b * nparam + p];
  if (grad) grad[p] = g;
  if (adam) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float m = b1 * mo[p] + (1.f - b1) * g;
    const float v = b2 * ve[p] + (1.f - b2) * g * g;
    mo[p] = m;
    ve[p] = v;
    prm[p] -= lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
  }
}

// FP32 master parameters -> packed FP16 inference weights
template <int IN, int OUT>
__global__ void k_mlp_pack(const float* __restrict__ prm, MlpPacked* __restrict__ P) {
  using PP = MlpParams<IN, OUT>;
  constexpr int H = kMlpH;
  for (int e = threadIdx.x; e < H * 24; e += blockDim.x) {
    const int n = e / 24, k = e % 24;
    P->W1[n][k] = __float2half_rn(k < IN ? prm[PP::W1 + n * IN + k] : 0.f);
  }
  for (int e = threadIdx.x; e < H * 72; e += blockDim.x) {
    const int n = e / 72, k = e % 72;
    P->W2[n][k] = __float2half_rn(k < H ? prm[PP::W2 + n * H + k] : 0.f);
  }
  for (int e = threadIdx.x; e < 8 * 72; e += blockDim.x) {
    const int n = e / 72, k = e % 72;
    P->W3[n][k] = __float2half_rn(n < OUT && k < H ? prm[PP::W3 + n * H + k] : 0.f);
  }
  for (int e = threadIdx.x; e < H; e += blockDim.x) {
    P->b1[e] = prm[PP::B1 + e];
    P->b2[e] = prm[PP::B2 + e];
  }
  for (int e = threadIdx.x; e < 8; e += blockDim.x) P->b3[e] = e < OUT ? prm[PP::B3 + e] : 0.f;
}

// Tensor-core inference of n samples (32 per warp).
template <int IN, int OUT>
__global__ void __launch_bounds__(128) k_mlp_infer(const MlpPacked* __restrict__ Pg,
                                                   const float* __restrict__ X, long long n,
                                                   float* __restrict__ Y) {
  __shared__ MlpPacked P;
  __shared__ __half xs[4][32][24];
  __shared__ float ys[4][32][8];
  mlp_load(P, Pg);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long base = (blockIdx.x * 4LL + w) * 32; base < n; base += gridDim.x * 128LL) {
    const long long r = base + lane;
    for (int k = 0; k < 24; ++k)
      xs[w][lane][k] = __float2half_rn(r < n && k < IN ? X[r * IN + k] : 0.f);
    __syncwarp();
    mlp_warp(P, xs[w], ys[w]);
    __syncwarp();
    if (r < n)
      for (int o = 0; o < OUT; ++o) Y[r * OUT + o] = ys[w][lane][o];
    __syncwarp();
  }
}

}  // namespace fvlb

// ===========================================================================
// C ABI
// ===========================================================================
using namespace fvlb;

struct fvlb_mlp_s {
  int lattice = 9, D = 2, IN = 8, OUT = 3, NP = 0;
  long long cap = 0, count = 0;
  float *prm = nullptr, *mo = nullptr, *ve = nullptr, *grad = nullptr;
  float *X = nullptr, *T = nullptr;
  float *part = nullptr, *part_loss = nullptr;
  int max_blocks = 0;
  double* loss = nullptr;
  MlpPacked* packed = nullptr;
  long long adam_t = 0;
  double delta = 0.0;       // relative-loss floor (0: plain mean squared error)
  cudaStream_t stream = nullptr;
  fvlb_alloc_fn alloc = nullptr;
  fvlb_free_fn free_ = nullptr;
  void* actx = nullptr;
  std::vector<void*> owned;
  std::string err;
};

namespace {

int mfail(fvlb_mlp_t m, int code, const std::string& msg) {
  if (m) m->err = msg;
  else set_global_error(code, msg.c_str());
  return code;
}

void* malloc_dev(fvlb_mlp_t m, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (m->alloc) p = m->alloc(bytes, m->actx);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) m->owned.push_back(p);
  return p;
}

size_t train_smem(int IN, int OUT, int NP) {
  return sizeof(float) * ((size_t)NP + kTB * IN + 4 * kTB * (kMlpH + 1) + kTB * OUT);
}

cudaError_t launch_grad(fvlb_mlp_t m, const float* X, const float* T, long long count,
                        long long n, int seed, long long base, int nblocks) {
  const float d2 = float(m->delta * m->delta);
  const size_t sm = train_smem(m->IN, m->OUT, m->NP);
  if (m->D == 2) {
    cudaFuncSetAttribute(k_mlp_grad<8, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_mlp_grad<8, 3><<<nblocks, kTB, sm, m->stream>>>(m->prm, X, T, count, n, seed, base, d2,
                                                      m->part, m->part_loss);
  } else {
    cudaFuncSetAttribute(k_mlp_grad<15, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_mlp_grad<15, 6><<<nblocks, kTB, sm, m->stream>>>(m->prm, X, T, count, n, seed, base, d2,
                                                       m->part, m->part_loss);
  }
  return cudaGetLastError();
}

cudaError_t repack(fvlb_mlp_t m) {
  if (m->D == 2) k_mlp_pack<8, 3><<<1, 256, 0, m->stream>>>(m->prm, m->packed);
  else k_mlp_pack<15, 6><<<1, 256, 0, m->stream>>>(m->prm, m->packed);
  return cudaGetLastError();
}

uint32_t host_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

}  // namespace

namespace fvlb {
const void* mlp_packed(fvlb_mlp_t m) { return m ? m->packed : nullptr; }
int mlp_lattice(fvlb_mlp_t m) { return m ? m->lattice : 0; }
}  // namespace fvlb

extern "C" {

int fvlb_mlp_create(fvlb_mlp_t* out, int lattice, long capacity, unsigned seed) {
  if (!out) return set_global_error(FVLB_EINVAL, "fvlb_mlp_create: out is NULL");
  *out = nullptr;
  if (lattice != FVLB_D2Q9 && lattice != FVLB_D3Q19)
    return set_global_error(FVLB_EINVAL, "fvlb_mlp_create: unknown lattice");
  if (capacity < 1) return set_global_error(FVLB_EINVAL, "fvlb_mlp_create: capacity must be >= 1");
  fvlb_mlp_s* m = new (std::nothrow) fvlb_mlp_s();
  if (!m) return set_global_error(FVLB_ENOMEM, "fvlb_mlp_create: out of host memory");
  m->lattice = lattice;
  m->D = lattice == FVLB_D2Q9 ? 2 : 3;
  m->IN = m->D == 2 ? 8 : 15;
  m->OUT = m->D == 2 ? 3 : 6;
  m->NP = m->D == 2 ? MlpParams<8, 3>::N : MlpParams<15, 6>::N;
  m->cap = capacity;
  m->max_blocks = 4096;
  current_allocator(&m->alloc, &m->free_, &m->actx);
  cudaError_t e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete m;
    return set_global_error(FVLB_ECUDA, "fvlb_mlp_create: stream creation failed");
  }
  m->prm = static_cast<float*>(malloc_dev(m, sizeof(float) * m->NP));
  m->mo = static_cast<float*>(malloc_dev(m, sizeof(float) * m->NP));
  m->ve = static_cast<float*>(malloc_dev(m, sizeof(float) * m->NP));
  m->grad = static_cast<float*>(malloc_dev(m, sizeof(float) * m->NP));
  m->X = static_cast<float*>(malloc_dev(m, sizeof(float) * m->IN * capacity));
  m->T = static_cast<float*>(malloc_dev(m, sizeof(float) * m->OUT * capacity));
  m->part = static_cast<float*>(malloc_dev(m, sizeof(float) * m->NP * (size_t)m->max_blocks));
  m->part_loss = static_cast<float*>(malloc_dev(m, sizeof(float) * m->max_blocks));
  m->loss = static_cast<double*>(malloc_dev(m, sizeof(double)));
  m->packed = static_cast<MlpPacked*>(malloc_dev(m, sizeof(MlpPacked)));
  if (!m->prm || !m->mo || !m->ve || !m->grad || !m->X || !m->T || !m->part || !m->part_loss ||
      !m->loss || !m->packed) {
    fvlb_mlp_destroy(m);
    return set_global_error(FVLB_ENOMEM, "fvlb_mlp_create: device allocation failed");
  }
  // He initialisation from a counter-based hash (Box-Muller), biases zero
  std::vector<float> p(m->NP, 0.f);
  const int H = kMlpH;
  auto normal = [&](uint32_t i) {
    const uint32_t a = host_hash(seed * 0x9e3779b9u ^ (2 * i + 1));
    const uint32_t b = host_hash(seed * 0x85ebca6bu ^ (2 * i + 2));
    const double u1 = (a + 1.0) / 4294967297.0, u2 = b / 4294967296.0;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  const int w1 = 0, w2 = H * m->IN + H, w3 = w2 + H * H + H;
  for (int i = 0; i < H * m->IN; ++i) p[w1 + i] = float(normal(i) * std::sqrt(2.0 / m->IN));
  for (int i = 0; i < H * H; ++i) p[w2 + i] = float(normal(100000 + i) * std::sqrt(2.0 / H));
  for (int i = 0; i < m->OUT * H; ++i) p[w3 + i] = float(normal(200000 + i) * std::sqrt(1.0 / H));
  e = cudaMemcpy(m->prm, p.data(), sizeof(float) * m->NP, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->mo, 0, sizeof(float) * m->NP);
  if (e == cudaSuccess) e = cudaMemset(m->ve, 0, sizeof(float) * m->NP);
  if (e == cudaSuccess) e = repack(m);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    fvlb_mlp_destroy(m);
    return set_global_error(FVLB_ECUDA, "fvlb_mlp_create: initialisation failed");
  }
  *out = m;
  return FVLB_OK;
}

int fvlb_mlp_num_params(fvlb_mlp_t m, size_t* n) {
  if (!m || !n) return mfail(m, FVLB_EINVAL, "fvlb_mlp_num_params: NULL argument");
  *n = (size_t)m->NP;
  return FVLB_OK;
}

int fvlb_mlp_get_params(fvlb_mlp_t m, float* host, size_t count) {
  if (!m || !host || count < (size_t)m->NP) return mfail(m, FVLB_EINVAL, "fvlb_mlp_get_params: bad buffer");
  cudaError_t e = cudaMemcpyAsync(host, m->prm, sizeof(float) * m->NP, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mfail(m, FVLB_ECUDA, cudaGetErrorString(e));
  return FVLB_OK;
}

int fvlb_mlp_set_params(fvlb_mlp_t m, const float* host, size_t count) {
  if (!m || !host || count != (size_t)m->NP) return mfail(m, FVLB_EINVAL, "fvlb_mlp_set_params: bad buffer");
  cudaError_t e = cudaMemcpyAsync(m->prm, host, sizeof(float) * m->NP, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = repack(m);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mfail(m, FVLB_ECUDA, cudaGetErrorString(e));
  return FVLB_OK;
}

int fvlb_mlp_collect(fvlb_mlp_t m, fvlb_t h, long stride) {
  if (!m || !h) return mfail(m, FVLB_EINVAL, "fvlb_mlp_collect: NULL argument");
  if (stride < 1) return mfail(m, FVLB_EINVAL, "fvlb_mlp_collect: stride must be >= 1");
  StateView v;
  int r = state_view(h, &v);
  if (r != FVLB_OK) return mfail(m, r, "fvlb_mlp_collect: no state");
  if (v.lattice != m->lattice) return mfail(m, FVLB_EINVAL, "fvlb_mlp_collect: lattice mismatch");
  const long long want = (v.N + stride - 1) / stride;
  const long long n = std::min<long long>(want, m->cap - m->count);
  if (n <= 0) return FVLB_OK;
  StepDesc d = v.desc;
  const int threads = 128;
  const int blocks = (int)std::min<long long>((n + threads - 1) / threads, 4096);
  float* X = m->X + m->count * m->IN;
  float* T = m->T + m->count * m->OUT;
  Grid g{d.nx, d.ny, m->D == 3 ? d.nz : 1, d.walls, d.pitch};
  cudaError_t e = cudaSuccess;
#define PAIRS(L, S)                                                                          \
  {                                                                                          \
    using R = RT<S>;                                                                         \
    Phys<R> ph = make_phys<R>(d);                                                            \
    k_closure_pairs<L, S><<<blocks, threads, 0, d.stream>>>(                                 \
        g, ph, static_cast<const S*>(d.f_in), static_cast<const S*>(d.h_in), d.N, stride, n, X, \
        T, d.lambda);                                                                        \
    e = cudaGetLastError();                                                                  \
  }
  if (d.storage == kFP64) {
    if (m->D == 2) PAIRS(D2Q9, double) else PAIRS(D3Q19, double)
  } else if (d.storage == kFP32) {
    if (m->D == 2) PAIRS(D2Q9, float) else PAIRS(D3Q19, float)
  } else {
    return mfail(m, FVLB_EINVAL, "fvlb_mlp_collect: collect from an FP64 or FP32 state");
  }
#undef PAIRS
  if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
  if (e != cudaSuccess) return mfail(m, FVLB_ECUDA, std::string("fvlb_mlp_collect: ") + cudaGetErrorString(e));
  m->count += n;
  return FVLB_OK;
}

int fvlb_mlp_set_loss(fvlb_mlp_t m, double delta) {
  if (!m) return set_global_error(FVLB_EINVAL, "NULL mlp");
  if (!(delta >= 0.0) || !std::isfinite(delta)) return mfail(m, FVLB_EINVAL, "fvlb_mlp_set_loss: delta must be >= 0");
  m->delta = delta;
  return FVLB_OK;
}

int fvlb_mlp_count(fvlb_mlp_t m, long* count) {
  if (!m || !count) return mfail(m, FVLB_EINVAL, "fvlb_mlp_count: NULL argument");
  *count = (long)m->count;
  return FVLB_OK;
}

int fvlb_mlp_get_pairs(fvlb_mlp_t m, float* x, float* t, long n) {
  if (!m || !x || !t || n < 0 || n > m->count) return mfail(m, FVLB_EINVAL, "fvlb_mlp_get_pairs: bad arguments");
  cudaError_t e = cudaMemcpyAsync(x, m->X, sizeof(float) * m->IN * n, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t, m->T, sizeof(float) * m->OUT * n, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mfail(m, FVLB_ECUDA, cudaGetErrorString(e));
  return FVLB_OK;
}

int fvlb_mlp_train(fvlb_mlp_t m, long steps, int batch, double lr, double* last_loss) {
  if (!m) return set_global_error(FVLB_EINVAL, "NULL mlp");
  if (steps < 0 || batch < kTB || batch % kTB || batch / kTB > m->max_blocks || !(lr > 0))
    return mfail(m, FVLB_EINVAL, "fvlb_mlp_train: batch must be a multiple of 64 (<= 262144), lr > 0");
  if (m->count < 1) return mfail(m, FVLB_ESTATE, "fvlb_mlp_train: no training pairs");
  const int nblocks = batch / kTB;
  cudaError_t e = cudaSuccess;
  for (long s = 0; s < steps && e == cudaSuccess; ++s) {
    m->adam_t += 1;
    e = launch_grad(m, m->X, m->T, m->count, batch, (int)(m->adam_t & 0x7fffffff), 0, nblocks);
    if (e != cudaSuccess) break;
    const float bc1 = 1.f - std::pow(0.9f, (float)m->adam_t), bc2 = 1.f - std::pow(0.999f, (float)m->adam_t);
    k_mlp_update<<<(m->NP + 255) / 256, 256, 0, m->stream>>>(
        m->prm, m->mo, m->ve, m->part, m->part_loss, nblocks, m->NP, nullptr, m->loss,
        1.0 / ((double)batch * m->OUT), 1, (float)lr, bc1, bc2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = repack(m);
  if (e == cudaSuccess && last_loss)
    e = cudaMemcpyAsync(last_loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mfail(m, FVLB_ECUDA, std::string("fvlb_mlp_train: ") + cudaGetErrorString(e));
  return FVLB_OK;
}

int fvlb_mlp_grad(fvlb_mlp_t m, const float* x, const float* t, long n, float* grad, double* loss) {
  if (!m || !x || !t || !grad || n < 1) return mfail(m, FVLB_EINVAL, "fvlb_mlp_grad: bad arguments");
  const int nblocks = (int)((n + kTB - 1) / kTB);
  if (nblocks > m->max_blocks) return mfail(m, FVLB_EINVAL, "fvlb_mlp_grad: too many samples");
  // stage the samples in the training buffers' tail-free front (copies)
  float *dx = nullptr, *dt = nullptr;
  dx = static_cast<float*>(malloc_dev(m, sizeof(float) * m->IN * n));
  dt = static_cast<float*>(malloc_dev(m, sizeof(float) * m->OUT * n));
  if (!dx || !dt) return mfail(m, FVLB_ENOMEM, "fvlb_mlp_grad: device allocation failed");
  cudaError_t e = cudaMemcpyAsync(dx, x, sizeof(float) * m->IN * n, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dt, t, sizeof(float) * m->OUT * n, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = launch_grad(m, dx, dt, n, n, -1, 0, nblocks);
  if (e == cudaSuccess) {
    k_mlp_update<<<(m->NP + 255) / 256, 256, 0, m->stream>>>(
        m->prm, m->mo, m->ve, m->part, m->part_loss, nblocks, m->NP, m->grad, m->loss,
        1.0 / ((double)n * m->OUT), 0, 0.f, 1.f, 1.f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->NP, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  // release the staging buffers
  for (void* p : {static_cast<void*>(dx), static_cast<void*>(dt)}) {
    m->owned.erase(std::find(m->owned.begin(), m->owned.end(), p));
    if (m->free_) m->free_(p, m->actx);
    else cudaFree(p);
  }
  if (e != cudaSuccess) return mfail(m, FVLB_ECUDA, std::string("fvlb_mlp_grad: ") + cudaGetErrorString(e));
  return FVLB_OK;
}

int fvlb_mlp_infer(fvlb_mlp_t m, const float* x, long n, float* y) {
  if (!m || !x || !y || n < 1) return mfail(m, FVLB_EINVAL, "fvlb_mlp_infer: bad arguments");
  float* dx = static_cast<float*>(malloc_dev(m, sizeof(float) * m->IN * n));
  float* dy = static_cast<float*>(malloc_dev(m, sizeof(float) * m->OUT * n));
  if (!dx || !dy) return mfail(m, FVLB_ENOMEM, "fvlb_mlp_infer: device allocation failed");
  cudaError_t e = cudaMemcpyAsync(dx, x, sizeof(float) * m->IN * n, cudaMemcpyHostToDevice, m->stream);
  const int blocks = (int)std::min<long long>((n + 127) / 128, 4096);
  if (e == cudaSuccess) {
    if (m->D == 2) k_mlp_infer<8, 3><<<blocks, 128, 0, m->stream>>>(m->packed, dx, n, dy);
    else k_mlp_infer<15, 6><<<blocks, 128, 0, m->stream>>>(m->packed, dx, n, dy);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(y, dy, sizeof(float) * m->OUT * n, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  for (void* p : {static_cast<void*>(dx), static_cast<void*>(dy)}) {
    m->owned.erase(std::find(m->owned.begin(), m->owned.end(), p));
    if (m->free_) m->free_(p, m->actx);
    else cudaFree(p);
  }
  if (e != cudaSuccess) return mfail(m, FVLB_ECUDA, std::string("fvlb_mlp_infer: ") + cudaGetErrorString(e));
  return FVLB_OK;
}

const char* fvlb_mlp_last_error(fvlb_mlp_t m) {
  if (!m) return fvlb_last_error(nullptr);
  return m->err.c_str();
}

int fvlb_mlp_destroy(fvlb_mlp_t m) {
  if (!m) return FVLB_OK;
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (void* p : m->owned) {
    if (m->free_) m->free_(p, m->actx);
    else cudaFree(p);
  }
  m->owned.clear();
  if (m->stream) cudaStreamDestroy(m->stream);
  delete m;
  return FVLB_OK;
}

}  // extern "C"
