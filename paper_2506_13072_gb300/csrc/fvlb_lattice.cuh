// fvlb_lattice.cuh -- lattice traits, storage traits and the per-site algebra
// of the fluctuating lattice Boltzmann step (arXiv 2506.13072, Sec. 2.2-2.3),
// written for the CUDA kernels of this library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace fvlb {

// ---------------------------------------------------------------------------
// Lattices.  Velocities in the paper's order: D2Q9 Sec. 2.2, D3Q19
// Appendix A.  Weights: Sec. 2.2 (D2Q9); 1/3, 1/18, 1/36 (D3Q19, fixed by
// 4th-order isotropy with c_s^2 = 1/3).  Symmetric tensor components are
// stored compactly: 2D (xx, xy, yy), 3D (xx, yy, zz, xy, xz, yz).
// All accessors are constexpr so that unrolled loops fold them away.
// ---------------------------------------------------------------------------
struct D2Q9 {
  static constexpr int D = 2, Q = 9, C = 3;
  __host__ __device__ static constexpr int cx(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
  }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i < 5 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5);
  }
  // compact component k -> (a, b)
  __host__ __device__ static constexpr int ca(int k) { return k == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int cb(int k) { return k == 0 ? 0 : 1; }
};

struct D3Q19 {
  static constexpr int D = 3, Q = 19, C = 6;
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  // pairs (1,2) (3,4) ... (17,18) are opposite
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
  }
  __host__ __device__ static constexpr int ca(int k) {
    return k < 3 ? k : (k == 5 ? 1 : 0);
  }
  __host__ __device__ static constexpr int cb(int k) {
    return k < 3 ? k : (k == 3 ? 1 : 2);
  }
};

template <class L>
__host__ __device__ constexpr int cc(int i, int a) {
  return a == 0 ? L::cx(i) : (a == 1 ? L::cy(i) : L::cz(i));
}

// compact index of (a, b)
template <class L>
__host__ __device__ constexpr int sym(int a, int b) {
  if (L::D == 2) {
    return (a == 0 && b == 0) ? 0 : ((a == 1 && b == 1) ? 2 : 1);
  } else {
    if (a == b) return a;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
  }
}

// ---------------------------------------------------------------------------
// Storage traits: how a population is held in HBM and in which precision the
// site arithmetic runs.  Every form holds f (whose rest equilibrium is 0) and
// the stress populations as deviations from the rest equilibrium
// (h_ab,i - w_i delta_ab).
// ---------------------------------------------------------------------------
// 16-bit re-read through L2 only; volatile so that it is not merged with the
// first read of the same population.
__device__ __forceinline__ unsigned short ld_l2_u16(const void* p) {
  unsigned short v;
  asm volatile("ld.global.cg.u16 %0, [%1];" : "=h"(v) : "l"(p));
  return v;
}

template <class S>
struct Store;

// a + v for a 16-bit v, converted (exactly) and added in one mixed-precision
// instruction: the same result as converting first and adding in FP32
__device__ __forceinline__ float add_f16(float a, unsigned short v) {
  float d;
  asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(v), "f"(a));
  return d;
}
__device__ __forceinline__ float add_bf16(float a, unsigned short v) {
  float d;
  asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(v), "f"(a));
  return d;
}
// v * w + a for 16-bit v and w, likewise (the product is exact in FP32)
__device__ __forceinline__ float fma_f16(unsigned short v, unsigned short w, float a) {
  float d;
  asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(v), "h"(w), "f"(a));
  return d;
}
// v - a for a 16-bit v, likewise
__device__ __forceinline__ float sub_f16(unsigned short v, float a) {
  float d;
  asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(v), "f"(a));
  return d;
}
__device__ __forceinline__ float sub_bf16(unsigned short v, float a) {
  float d;
  asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(v), "f"(a));
  return d;
}

template <>
struct Store<double> {
  using R = double;     // arithmetic
  using X = double;     // chi of the previous step
  static constexpr bool V2 = false;  // no reference-based 16-bit layout (see below)
  __device__ static __forceinline__ double ld(const double* p) { return __ldg(p); }
  __device__ static __forceinline__ double cvt(double v) { return v; }
  __device__ static __forceinline__ double acc(double a, double v) { return a + v; }
  static constexpr bool sr = false;
  __device__ static __forceinline__ void st(double* p, double v, uint32_t) { *p = v; }
  __device__ static __forceinline__ double ld_l2(const double* p) {
    double v;
    asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
  }
};

template <>
struct Store<float> {
  using R = float;
  using X = float;
  static constexpr bool V2 = false;
  __device__ static __forceinline__ float ld(const float* p) { return __ldg(p); }
  __device__ static __forceinline__ float cvt(float v) { return v; }
  __device__ static __forceinline__ float acc(float a, float v) { return a + v; }
  static constexpr bool sr = false;
  __device__ static __forceinline__ void st(float* p, float v, uint32_t) { *p = v; }
  __device__ static __forceinline__ float ld_l2(const float* p) {
    float v;
    asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
  }
};

template <>
struct Store<__half> {
  using R = float;
  using X = float;
  static constexpr bool V2 = true;
  static constexpr float KF = 4096.0f;       // flow-population scale (2^12)
  static constexpr bool sr = false;
  __device__ static __forceinline__ float ld(const __half* p) {
    return __half2float(__ldg(p));
  }
  __device__ static __forceinline__ float cvt(__half v) { return __half2float(v); }
  __device__ static __forceinline__ float cvtb(unsigned short b) { return __half2float(__ushort_as_half(b)); }
  __device__ static __forceinline__ float accb(float a, unsigned short b) { return add_f16(a, b); }
  __device__ static __forceinline__ float subb(unsigned short b, float a) { return sub_f16(b, a); }
  __device__ static __forceinline__ float acc(float a, __half v) { return add_f16(a, __half_as_ushort(v)); }
  __device__ static __forceinline__ void st(__half* p, float v, uint32_t) {
    *p = __float2half_rn(v);
  }
  // store, and return the stored value
  __device__ static __forceinline__ float st_r(__half* p, float v, uint32_t) {
    const __half q = __float2half_rn(v);
    *p = q;
    return __half2float(q);
  }
  // v / KF + e (2^-12 is the FP16 number 0x0C00)
  __device__ static __forceinline__ float dev_add(__half v, float e) {
    return fma_f16(__half_as_ushort(v), 0x0C00, e);
  }
  // store, and return the stored value minus v (its rounding error)
  __device__ static __forceinline__ float st_d(__half* p, float v, uint32_t) {
    const __half q = __float2half_rn(v);
    *p = q;
    return sub_f16(__half_as_ushort(q), v);
  }
  __device__ static __forceinline__ float ld_l2(const __half* p) {
    return __half2float(__ushort_as_half(ld_l2_u16(p)));
  }
};

template <>
struct Store<__nv_bfloat16> {
  using R = float;
  using X = float;
  static constexpr bool V2 = true;
  static constexpr float KF = 1.0f;          // (no subnormal range to avoid)
  static constexpr bool sr = false;
  __device__ static __forceinline__ float ld(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
  }
  __device__ static __forceinline__ float cvt(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __forceinline__ float cvtb(unsigned short b) { return __uint_as_float((uint32_t)b << 16); }
  __device__ static __forceinline__ float accb(float a, unsigned short b) { return add_bf16(a, b); }
  __device__ static __forceinline__ float subb(unsigned short b, float a) { return sub_bf16(b, a); }
  __device__ static __forceinline__ float acc(float a, __nv_bfloat16 v) { return add_bf16(a, __bfloat16_as_ushort(v)); }
  __device__ static __forceinline__ void st(__nv_bfloat16* p, float v, uint32_t) {
    *p = __float2bfloat16_rn(v);
  }
  __device__ static __forceinline__ float st_r(__nv_bfloat16* p, float v, uint32_t) {
    const __nv_bfloat16 q = __float2bfloat16_rn(v);
    *p = q;
    return __bfloat162float(q);
  }
  __device__ static __forceinline__ float dev_add(__nv_bfloat16 v, float e) {  // KF = 1
    return add_bf16(e, __bfloat16_as_ushort(v));
  }
  __device__ static __forceinline__ float st_d(__nv_bfloat16* p, float v, uint32_t) {
    const __nv_bfloat16 q = __float2bfloat16_rn(v);
    *p = q;
    return sub_bf16(__bfloat16_as_ushort(q), v);
  }
  __device__ static __forceinline__ float ld_l2(const __nv_bfloat16* p) {
    return __uint_as_float((uint32_t)ld_l2_u16(p) << 16);
  }
};

// 16-bit forms with stochastic rounding: the value is rounded up or down to
// a neighbouring representable number with probabilities proportional to
// its distance from each, so the rounding error has zero mean and does not
// accumulate coherently over steps.  Same bits in memory as __half /
// __nv_bfloat16.
struct half_sr {
  unsigned short b;
};
struct bf16_sr {
  unsigned short b;
};

static_assert(Store<__half>::KF == 4096.0f, "dev_add takes 1 / KF as the FP16 number 0x0C00 (2^-12)");

template <>
struct Store<half_sr> {
  using R = float;
  using X = float;
  static constexpr bool V2 = true;
  static constexpr float KF = 4096.0f;
  static constexpr bool sr = true;
  __device__ static __forceinline__ float ld(const half_sr* p) {
    return __half2float(__ushort_as_half(__ldg(&p->b)));
  }
  __device__ static __forceinline__ float cvt(half_sr v) {
    return __half2float(__ushort_as_half(v.b));
  }
  __device__ static __forceinline__ float cvtb(unsigned short b) { return __half2float(__ushort_as_half(b)); }
  __device__ static __forceinline__ float accb(float a, unsigned short b) { return add_f16(a, b); }
  __device__ static __forceinline__ float subb(unsigned short b, float a) { return sub_f16(b, a); }
  __device__ static __forceinline__ float acc(float a, half_sr v) { return add_f16(a, v.b); }
  // r: 32 random bits.  Add r * ulp(|v|) in magnitude, then truncate.
  __device__ static __forceinline__ __half round(float v, uint32_t r) {
    const uint32_t bits = __float_as_uint(v);
    int e = (int)((bits >> 23) & 0xffu) - 127;  // binade of |v|
    e = e < -14 ? -14 : e;                      // half subnormals share one ulp
    const float ulp = __uint_as_float((uint32_t)(e - 10 + 127) << 23);
    const float jit = __uint2float_rz(r >> 8) * (1.0f / 16777216.0f) * ulp;
    const float w = v + copysignf(jit, v);
    return __float2half_rz(w);
  }
  __device__ static __forceinline__ void st(half_sr* p, float v, uint32_t r) {
    p->b = __half_as_ushort(round(v, r));
  }
  __device__ static __forceinline__ float st_r(half_sr* p, float v, uint32_t r) {
    const __half q = round(v, r);
    p->b = __half_as_ushort(q);
    return __half2float(q);
  }
  __device__ static __forceinline__ float dev_add(half_sr v, float e) {
    return fma_f16(v.b, 0x0C00, e);
  }
  __device__ static __forceinline__ float st_d(half_sr* p, float v, uint32_t r) {
    const __half q = round(v, r);
    p->b = __half_as_ushort(q);
    return sub_f16(__half_as_ushort(q), v);
  }
  __device__ static __forceinline__ float ld_l2(const half_sr* p) {
    return __half2float(__ushort_as_half(ld_l2_u16(p)));
  }
};

template <>
struct Store<bf16_sr> {
  using R = float;
  using X = float;
  static constexpr bool V2 = true;
  static constexpr float KF = 1.0f;
  static constexpr bool sr = true;
  __device__ static __forceinline__ float ld(const bf16_sr* p) {
    return __uint_as_float((uint32_t)__ldg(&p->b) << 16);
  }
  __device__ static __forceinline__ float cvt(bf16_sr v) { return __uint_as_float((uint32_t)v.b << 16); }
  __device__ static __forceinline__ float cvtb(unsigned short b) { return __uint_as_float((uint32_t)b << 16); }
  __device__ static __forceinline__ float accb(float a, unsigned short b) { return add_bf16(a, b); }
  __device__ static __forceinline__ float subb(unsigned short b, float a) { return sub_bf16(b, a); }
  __device__ static __forceinline__ float acc(float a, bf16_sr v) { return add_bf16(a, v.b); }
  // add 16 random bits below the kept 16 and truncate (sign-magnitude, so the
  // rounding is unbiased in magnitude and hence in value)
  __device__ static __forceinline__ void st(bf16_sr* p, float v, uint32_t r) {
    const uint32_t bits = __float_as_uint(v);
    const uint32_t exp = bits & 0x7f800000u;
    const uint32_t out = exp == 0x7f800000u ? bits : bits + (r >> 16);
    p->b = (unsigned short)(out >> 16);
  }
  __device__ static __forceinline__ float st_r(bf16_sr* p, float v, uint32_t r) {
    const uint32_t bits = __float_as_uint(v);
    const uint32_t exp = bits & 0x7f800000u;
    const uint32_t out = (exp == 0x7f800000u ? bits : bits + (r >> 16)) & 0xffff0000u;
    p->b = (unsigned short)(out >> 16);
    return __uint_as_float(out);
  }
  __device__ static __forceinline__ float dev_add(bf16_sr v, float e) {  // KF = 1
    return add_bf16(e, v.b);
  }
  __device__ static __forceinline__ float st_d(bf16_sr* p, float v, uint32_t r) {
    return st_r(p, v, r) - v;
  }
  __device__ static __forceinline__ float ld_l2(const bf16_sr* p) {
    return __uint_as_float((uint32_t)ld_l2_u16(p) << 16);
  }
};

// Random bits for stochastic rounding: one counter-based hash per site and
// step (the "lowbias32" integer hash of C. Wellons), then a 32-bit linear
// congruential sequence (Numerical Recipes constants) whose high bits feed
// one store each.
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ uint32_t lcg_next(uint32_t& r) {
  r = r * 1664525u + 1013904223u;
  return r;
}

// ---------------------------------------------------------------------------
// Launch-time description of a grid and of the physics of a step.
// ---------------------------------------------------------------------------
struct Grid {
  int nx, ny, nz;     // nz = 1 in 2D
  int walls;          // bit a: halfway bounce-back walls on axis a
  long long pitch;    // elements between consecutive population arrays
};

template <class R>
struct Phys {
  R inv_tau_f;        // 1 / tau_f
  R tau_f;
  R inv_tau_h;        // 1 / tau_h
  R kh;               // 1 - 1 / (2 tau_h)
  R kf;               // 1 - 1 / (2 tau_f)
  R eta_over_lam;     // eta_p / lambda
  R inv_lam;          // 1 / lambda
  int four_roll;      // 1: F = amp (sx cy, -cx sy); 0: F = Fv
  R Fv[3];
  R amp;
  const R* sx;        // sin(k x), x < nx
  const R* cxs;       // cos(k x)
  const R* sy;        // sin(k y), y < ny
  const R* cys;       // cos(k y)
  int first;          // first step: chi of the previous step := chi
  uint32_t step;      // step counter (stochastic-rounding stream)
  unsigned* err;      // bounded device waits that ran out (bit 0: staging copies), or null
  R lam;              // lambda
  const void* mlp;    // learned closure: packed network weights (or null)
  float cl_tol2;      // squared fallback tolerance of the learned closure
  unsigned long long* cl_count;  // [0] nodes on the network, [1] fallbacks
  int model;          // constitutive model: 0 Oldroyd-B, 1 Giesekus, 2 / 3 PTT
  R mpar;             // its parameter: alpha (Giesekus) or eps (PTT)
  const R* fdiv;      // fused step of the original scheme: div tau_p [D][pitch],
                      // added to the body force (null for the present scheme)
};

template <class S>
struct Bufs {
  using X = typename Store<S>::X;
  const S* __restrict__ f_in;
  S* __restrict__ f_out;
  const S* __restrict__ h_in;
  S* __restrict__ h_out;
  X* __restrict__ chi;  // [C][pitch], read and rewritten in place
};

// ---------------------------------------------------------------------------
// Layout of the 16-bit forms (Store<S>::V2).  Rounding a population to 16
// bits every step biases slowly evolving flows: the per-step change of a
// population can be as small as its rounding error, which then accumulates
// coherently.  So:
//  - the flow populations are stored scaled, s_i = KF (f_i - e_i(U)), as
//    deviations from the velocity part of the equilibrium,
//    e_i(U) = w_i (3 c_i.U + 4.5 (c_i.U)^2 - 1.5 U.U), at the velocity U
//    that their destination node had in the step that wrote them (a node
//    pushing f_i to x + c_i takes U = u(x + c_i) from its velocity ring);
//    U[D][pitch] (FP32) follows f[Q][pitch] in the same buffer, written by
//    each node for its own populations of the next step;
//  - the stress populations h'_{k,i} (i >= 1) are 16-bit; the rest
//    population of each component is FP32, h0[C][pitch] following
//    h[C][Q][pitch] (whose i = 0 slots are unused), and takes up the
//    rounding residual of the component's other populations at every
//    store, so the stored populations of a node carry no rounding bias in
//    their sum.
// ---------------------------------------------------------------------------
template <class S>
struct V2Layout {
  static constexpr bool on = Store<S>::V2;
};

// 3 w_i as the coefficient of the first-order terms (c_i.u, c_i.F) of the
// flow equilibrium and the Guo forcing, chosen so that the lattice's second
// moment sum_i (3 w_i) c_ia c_ib = delta_ab holds exactly in R.  With each
// 3 w_i rounded on its own, FP32 gives (1 + 7.45e-9) delta_ab in both
// lattices, so every collision adds that fraction of rho u and F to the
// momentum, which over 10^4-10^5 steps of a channel flow was the largest
// FP32 error against FP64.  One class of directions (axis or diagonal)
// takes the rounded value, the other the remainder, whichever of the two
// is exact in R; FP64 keeps the plain 3 w_i.
template <class L>
__host__ __device__ constexpr int n_diag_x() { return L::D == 2 ? 4 : 8; }
template <class L, class R>
__host__ __device__ constexpr double w3(int i) {
  if (i == 0) return 0.0;
  if (std::is_same<R, double>::value) return 3.0 * L::w(i);
  const bool axis = cc<L>(i, 0) * cc<L>(i, 0) + cc<L>(i, 1) * cc<L>(i, 1) +
                        cc<L>(i, 2) * cc<L>(i, 2) == 1;
  double a = (double)(R)(3.0 * L::w(1));
  double d = (1.0 - 2.0 * a) / n_diag_x<L>();
  if ((double)(R)d != d) {
    d = (double)(R)(3.0 * L::w(L::Q - 1));
    a = (1.0 - n_diag_x<L>() * d) / 2.0;
  }
  return axis ? a : d;
}
template <class L, class R>
__host__ __device__ constexpr bool w3_exact() {
  const double a = w3<L, R>(1), d = w3<L, R>(L::Q - 1);
  return (double)(R)a == a && (double)(R)d == d && 2.0 * a + n_diag_x<L>() * d == 1.0;
}
static_assert(w3_exact<D2Q9, float>() && w3_exact<D3Q19, float>(),
              "first-order coefficients must carry the exact second moment in FP32");

// velocity part of f^eq: e_i(u) = w_i (3 c.u + 4.5 (c.u)^2 - 1.5 u.u), with
// w3<L, R>(i) for 3 w_i (so that sum_i c_i e_i(u) = u holds in R)
template <class L, class R>
__device__ __forceinline__ R feq_u(int i, const R (&u)[L::D]) {
  R cu = R(0), uu = R(0);
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    const int c = cc<L>(i, a);
    if (c == 1) cu += u[a];
    if (c == -1) cu -= u[a];
    uu += u[a] * u[a];
  }
  return R(w3<L, R>(i)) * cu + R(L::w(i)) * (R(4.5) * cu * cu - R(1.5) * uu);
}

// Sum of the weights as rounded to the working precision R, minus one
// (exact in double: the rounded weights have few enough bits).  FP32:
// 7.45e-9 (D2Q9), 1.49e-8 (D3Q19).  A collision whose equilibrium part is
// w_i alpha moves the zeroth moment by alpha times this at every step; the
// stress collisions take it back out of their rest population.
template <class L, class R>
__host__ __device__ constexpr double weight_sum_excess() {
  double s = 0.0;
  for (int i = 0; i < L::Q; ++i) s += (double)(R)L::w(i);
  return s - 1.0;
}

// Pressure part of the flow equilibrium, lam_i p (lam_0 = 3 (w_0 - 1),
// lam_i = 3 w_i), with p = c_s^2 / (1 - w_0) S and S the bracket of the
// pressure formula (Sec. 2.2, Appendix B).  The next step's S sums the
// non-rest populations, so the equilibrium gives S back times
// (sum_{i>=1} lam_i) / (3 (1 - w_0)), which with FP32 constants is 1 + 4.3e-8
// (D2Q9) or 1 + 3.0e-8 (D3Q19): a gain on the pressure at every collision.
// In FP32 the part is formed as nu_i T with nu_i = w_i / w_1 (1 on the
// axes, 1/4 (D2Q9) or 1/2 (D3Q19) on the diagonals, nu_0 = -K) and
// T = S / K, K = (1 - w_0) / w_1 (5, 12), by a correctly rounded division:
// every nu_i is exact and sum_{i>=1} nu_i = K, so nothing is gained or lost
// beyond unbiased rounding.  FP64 keeps lam_i and p.
// (the ratios are multiples of 1/4; rounding removes the FP64 quotients' error)
__host__ __device__ constexpr double quarter(double x) {
  return (double)(long long)(x * 4.0 + (x >= 0.0 ? 0.5 : -0.5)) / 4.0;
}
template <class L, class R>
__host__ __device__ constexpr double p_coef(int i) {
  if (std::is_same<R, double>::value) return i == 0 ? (L::w(0) - 1.0) * 3.0 : L::w(i) * 3.0;
  return quarter(i == 0 ? (L::w(0) - 1.0) / L::w(1) : L::w(i) / L::w(1));
}
template <class L, class R>
__device__ __forceinline__ R p_part(R S) {
  if constexpr (std::is_same<R, double>::value) return R(1.0 / (3.0 * (1.0 - L::w(0)))) * S;
  else return S / R(-p_coef<L, R>(0));
}
// the same from p itself (initial state): p / (3 w_1)
template <class L, class R>
__device__ __forceinline__ R p_part_of_p(R p) {
  if constexpr (std::is_same<R, double>::value) return p;
  else return p / R(quarter(1.0 / (3.0 * L::w(1))));
}
// p from the pressure variable (in FP64, for output)
template <class L, class R>
__device__ __forceinline__ double p_of_part(R t) {
  if constexpr (std::is_same<R, double>::value) return t;
  else return double(t) * quarter(1.0 / (3.0 * L::w(1)));
}
template <class L, class R>
__host__ __device__ constexpr bool p_coef_exact() {
  double k = 0.0;
  for (int i = 1; i < L::Q; ++i) {
    if ((double)(R)p_coef<L, R>(i) != p_coef<L, R>(i)) return false;
    k += p_coef<L, R>(i);
  }
  return k == -p_coef<L, R>(0) && (double)(R)k == k;
}
static_assert(p_coef_exact<D2Q9, float>() && p_coef_exact<D3Q19, float>(),
              "pressure coefficients must be exact in FP32 and sum to K");

// the same with |u|^2 given
template <class L, class R>
__device__ __forceinline__ R feq_u(int i, const R (&u)[L::D], R uu) {
  R cu = R(0);
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    const int c = cc<L>(i, a);
    if (c == 1) cu += u[a];
    if (c == -1) cu -= u[a];
  }
  return R(w3<L, R>(i)) * cu + R(L::w(i)) * (R(4.5) * cu * cu - R(1.5) * uu);
}

// The FP32 arrays that follow the 16-bit populations: U[D][pitch] after
// f[Q][pitch], h0[C][pitch] after h[C][Q][pitch] (pitch is a multiple of 64
// elements, so they start 128-byte aligned).
template <class L, class T>
__device__ __forceinline__ auto f_ext(T* f, long long pitch) {
  using F = typename std::conditional<std::is_const<T>::value, const float, float>::type;
  return reinterpret_cast<F*>(f + (long long)L::Q * pitch);
}
template <class L, class T>
__device__ __forceinline__ auto h_ext(T* h, long long pitch) {
  using F = typename std::conditional<std::is_const<T>::value, const float, float>::type;
  return reinterpret_cast<F*>(h + (long long)L::C * L::Q * pitch);
}

// ---------------------------------------------------------------------------
// Per-site algebra.
// ---------------------------------------------------------------------------

// Body force at (x, y); 3D forces do not depend on z.
template <class L, class R>
__device__ __forceinline__ void body_force(const Phys<R>& ph, int x, int y,
                                           R F[3]) {
  if (ph.four_roll) {
    F[0] = ph.amp * __ldg(ph.sx + x) * __ldg(ph.cys + y);
    F[1] = -ph.amp * __ldg(ph.cxs + x) * __ldg(ph.sy + y);
    F[2] = R(0);
  } else {
    F[0] = ph.Fv[0];
    F[1] = ph.Fv[1];
    F[2] = ph.Fv[2];
  }
}

// u = sum_{i != 0} c_i f_i + F / 2   (Sec. 2.2)
template <class L, class R>
__device__ __forceinline__ void velocity(const R (&f)[L::Q], const R F[3],
                                         R (&u)[L::D]) {
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    R m = R(0);
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
      const int c = cc<L>(i, a);
      if (c == 1) m += f[i];
      else if (c == -1) m -= f[i];
    }
    u[a] = m + R(0.5) * F[a];
  }
}

// f^B for a symmetric polymer stress (compact components t[C]).  This is
// the least-norm solution of the three moment constraints of Sec. 2.2
// (sum f^B = 0, sum c f^B = 0, sum c c f^B = -tau_p / tau_f), written per
// direction class; it equals the pseudo-inverse matrices of Appendix A.
template <class L, class R>
__device__ __forceinline__ R fB_dir(int i, const R (&t)[L::C], R inv_tau_f) {
  if (L::D == 2) {
    const R a = t[0], s = t[1], b = t[2];
    const int x = L::cx(i), y = L::cy(i);
    R v;
    if (i == 0) v = (a + b) * R(1.0 / 3.0);
    else if (y == 0) v = (R(2) * b - a) * R(1.0 / 6.0);
    else if (x == 0) v = (R(2) * a - b) * R(1.0 / 6.0);
    else v = -(R(3 * x * y) * s + R(2) * (a + b)) * R(1.0 / 12.0);
    return v * inv_tau_f;
  } else {
    const int c0 = L::cx(i), c1 = L::cy(i), c2 = L::cz(i);
    const int n = c0 * c0 + c1 * c1 + c2 * c2;
    R v;
    if (n == 0) {
      v = (t[0] + t[1] + t[2]) * R(5.0 / 21.0);
    } else if (n == 1) {
      const int a = c0 != 0 ? 0 : (c1 != 0 ? 1 : 2);
      const R taa = t[a];
      const R rest = t[0] + t[1] + t[2] - taa;
      v = -taa * R(1.0 / 42.0) + rest * R(1.0 / 7.0);
    } else {
      const int g = c0 == 0 ? 0 : (c1 == 0 ? 1 : 2);  // axis normal to the plane
      const int a = g == 0 ? 1 : 0, b = g == 2 ? 1 : 2;
      const R sab = t[sym<L>(a, b)];
      const int cab = cc<L>(i, a) * cc<L>(i, b);
      v = -(t[a] + t[b]) * R(5.0 / 42.0) + t[g] * R(1.0 / 21.0) -
          R(0.25) * R(cab) * sab;
    }
    return v * inv_tau_f;
  }
}

// (grad u)_{ab} = d_a u_b, chi = -(A - I)/lambda + A.grad u + (grad u)^T.A
// in compact components (Sec. 2.3); Ad = A - I.
__device__ __forceinline__ float rexp(float x) { return expf(x); }
__device__ __forceinline__ double rexp(double x) { return exp(x); }

// Relaxation part P of the stress source chi = -P / lambda + A.grad u +
// (grad u)^T.A (Sec. 2.3), component k, from M = A - I (Ad): the paper's
// Oldroyd-B model P = M, or one of the models it names beside it (Sec. 1):
// Giesekus P = M + alpha M.M, linear PTT P = (1 + eps tr M) M, exponential
// PTT P = exp(eps tr M) M (no slip parameter).  In 2D M has no z entries.
template <class L, class R>
__device__ __forceinline__ R relax_part(int k, const R (&Ad)[L::C], int model, R par) {
  const R m = Ad[k];
  if (model == 0) return m;
  if (model == 1) {
    const int a = L::ca(k), b = L::cb(k);
    R mm = R(0);
#pragma unroll
    for (int g = 0; g < L::D; ++g) mm += Ad[sym<L>(a, g)] * Ad[sym<L>(g, b)];
    return m + par * mm;
  }
  R tr = R(0);
#pragma unroll
  for (int g = 0; g < L::D; ++g) tr += Ad[sym<L>(g, g)];
  return (model == 2 ? R(1) + par * tr : rexp(par * tr)) * m;
}

template <class L, class R>
__device__ __forceinline__ void chi_tensor(const R (&A)[L::C], const R (&Ad)[L::C],
                                           const R (&g)[L::D][L::D], const Phys<R>& ph,
                                           R (&chi)[L::C]) {
#pragma unroll
  for (int k = 0; k < L::C; ++k) {
    const int a = L::ca(k), b = L::cb(k);
    R v = -relax_part<L, R>(k, Ad, ph.model, ph.mpar) * ph.inv_lam;
#pragma unroll
    for (int q = 0; q < L::D; ++q) {
      v += A[sym<L>(a, q)] * g[q][b] + g[q][a] * A[sym<L>(q, b)];
    }
    chi[k] = v;
  }
}

}  // namespace fvlb
