// fvlb_mlp.cuh -- the learned stress closure's network on the GPU.
//
// A small MLP maps a node's lambda-scaled local state to its lambda-scaled
// stress source (Sec. 2.3, chi = -(A - I)/lambda + A.grad u + (grad u)^T.A):
//   x = (lambda d_a u_b  [D x D, row-major], A - I [C compact], dt/lambda [2D])
//   y = lambda chi [C compact]
// IN -> 64 -> 64 -> OUT (D2Q9: 8 -> 3, D3Q19: 15 -> 6), GELU in its tanh
// form.  Training keeps FP32 master weights (per-sample forward/backward on
// CUDA cores, deterministic block reductions, Adam); inference packs the
// weights to FP16 and runs each layer of 32 nodes on the tensor cores with
// mma.sync m16n8k16 (FP16 operands, FP32 accumulation), the GELU of each
// pair of hidden units in packed FP16 arithmetic (half the instructions of
// two FP32 evaluations; the activations are FP16 operands of the next
// layer in any case).  The products are
// 16 x 16 x 64 and 16 x 64 x 64 per warp (two warps per 32-node group, one
// m16 tile each), fused into the collision of the nodes the group already
// holds; the register-level mma keeps them there (a tcgen05 tile would need
// the operands staged through shared memory and tensor memory for a 16-row
// product).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace fvlb {

constexpr int kMlpH = 64;

template <int D>
struct MlpDims;
template <>
struct MlpDims<2> {
  static constexpr int IN = 8, OUT = 3;
};
template <>
struct MlpDims<3> {
  static constexpr int IN = 15, OUT = 6;
};

// number of FP32 parameters: W1[H][IN] b1[H] W2[H][H] b2[H] W3[OUT][H] b3[OUT]
template <int IN, int OUT>
struct MlpParams {
  static constexpr int W1 = 0;
  static constexpr int B1 = W1 + kMlpH * IN;
  static constexpr int W2 = B1 + kMlpH;
  static constexpr int B2 = W2 + kMlpH * kMlpH;
  static constexpr int W3 = B2 + kMlpH;
  static constexpr int B3 = W3 + OUT * kMlpH;
  static constexpr int N = B3 + OUT;
};

// Packed inference weights (FP16 rows padded so that the 32-bit fragment
// loads of a warp hit 32 distinct shared-memory banks) and FP32 biases.
struct __align__(16) MlpPacked {
  __half W1[kMlpH][24];  // [n][k], k < 16 (inputs zero-padded to 16)
  __half W2[kMlpH][72];  // [n][k], k < 64
  __half W3[8][72];      // [n][k], n < OUT (rows beyond OUT are zero)
  float b1[kMlpH], b2[kMlpH], b3[8];
};

__device__ __forceinline__ uint32_t h2_bits(__half2 v) { return *reinterpret_cast<uint32_t*>(&v); }

__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
  return h2_bits(__floats2half2_rn(lo, hi));
}

// GELU in its tanh form, 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))),
// of the pair (lo, hi), in packed FP16; returns the packed FP16 results.
// Beyond |z| ~ 256 the cube overflows to +-inf, whose tanh is +-1, so the
// result is z or 0 as GELU's limits are.
__device__ __forceinline__ uint32_t gelu_f16x2(float lo, float hi) {
  const __half2 z = __floats2half2_rn(lo, hi);
  const __half2 z2 = __hmul2(z, z);
  const __half2 in = __hfma2(__hmul2(__float2half2_rn(0.044715f), z2), z, z);
  const __half2 arg = __hmul2(__float2half2_rn(0.7978845608028654f), in);
  uint32_t t;
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(h2_bits(arg)));
  const __half2 hz = __hmul2(__float2half2_rn(0.5f), z);
  return h2_bits(__hfma2(hz, *reinterpret_cast<const __half2*>(&t), hz));
}

__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                          uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t lds32(const __half* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// One warp: Y[r][0..7] = MLP(X[r][0..15]) for the 16 rows r of m-tile mt
// (rows 16 mt .. 16 mt + 15).  X and Y are shared-memory staging rows; P
// the packed weights.
// Fragment layout of mma.m16n8k16 (g = lane / 4, t = lane % 4):
//   A: a0 (g, 2t..2t+1) a1 (g+8, 2t..) a2 (g, 2t+8..) a3 (g+8, 2t+8..)
//   B: b0 (k = 2t..2t+1, n = g)  b1 (k = 2t+8.., n = g)
//   C: c0,c1 (g, 2t..2t+1)  c2,c3 (g+8, 2t..2t+1)
// The accumulators of two adjacent n8 tiles form the A fragment of the
// next layer's k16 tile, so hidden activations never leave registers; the
// layers are interleaved so that only one layer-1 output (16 registers of
// packed FP16) and one pair of layer-2 tiles are live at a time.
__device__ __forceinline__ void mlp_tile(const MlpPacked& P, const __half (*X)[24],
                                         float (*Y)[8], int mt) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = mt * 16 + g, r1 = r0 + 8;
  uint32_t a[4] = {lds32(&X[r0][2 * t]), lds32(&X[r1][2 * t]), lds32(&X[r0][2 * t + 8]),
                   lds32(&X[r1][2 * t + 8])};
  // layer 1: 16 -> 64, packed k-tile by k-tile into layer 2's A fragments
  uint32_t a2[4][4];
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    float h0[4], h1[4];
    {
      const float c0 = P.b1[2 * kt * 8 + 2 * t], c1 = P.b1[2 * kt * 8 + 2 * t + 1];
      h0[0] = c0; h0[1] = c1; h0[2] = c0; h0[3] = c1;
      const float d0 = P.b1[(2 * kt + 1) * 8 + 2 * t], d1 = P.b1[(2 * kt + 1) * 8 + 2 * t + 1];
      h1[0] = d0; h1[1] = d1; h1[2] = d0; h1[3] = d1;
    }
    mma_16816(h0, a, lds32(&P.W1[2 * kt * 8 + g][2 * t]), lds32(&P.W1[2 * kt * 8 + g][2 * t + 8]));
    mma_16816(h1, a, lds32(&P.W1[(2 * kt + 1) * 8 + g][2 * t]),
              lds32(&P.W1[(2 * kt + 1) * 8 + g][2 * t + 8]));
    a2[kt][0] = gelu_f16x2(h0[0], h0[1]);
    a2[kt][1] = gelu_f16x2(h0[2], h0[3]);
    a2[kt][2] = gelu_f16x2(h1[0], h1[1]);
    a2[kt][3] = gelu_f16x2(h1[2], h1[3]);
  }
  // layers 2 (64 -> 64) and 3 (64 -> 8, OUT used): each pair of layer-2
  // n-tiles is one layer-3 k-tile, accumulated as soon as it is ready
  float y[4];
  y[0] = P.b3[2 * t]; y[1] = P.b3[2 * t + 1]; y[2] = y[0]; y[3] = y[1];
#pragma unroll
  for (int k3 = 0; k3 < 4; ++k3) {
    float h0[4], h1[4];
    {
      const float c0 = P.b2[2 * k3 * 8 + 2 * t], c1 = P.b2[2 * k3 * 8 + 2 * t + 1];
      h0[0] = c0; h0[1] = c1; h0[2] = c0; h0[3] = c1;
      const float d0 = P.b2[(2 * k3 + 1) * 8 + 2 * t], d1 = P.b2[(2 * k3 + 1) * 8 + 2 * t + 1];
      h1[0] = d0; h1[1] = d1; h1[2] = d0; h1[3] = d1;
    }
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      mma_16816(h0, a2[kt], lds32(&P.W2[2 * k3 * 8 + g][kt * 16 + 2 * t]),
                lds32(&P.W2[2 * k3 * 8 + g][kt * 16 + 2 * t + 8]));
      mma_16816(h1, a2[kt], lds32(&P.W2[(2 * k3 + 1) * 8 + g][kt * 16 + 2 * t]),
                lds32(&P.W2[(2 * k3 + 1) * 8 + g][kt * 16 + 2 * t + 8]));
    }
    const uint32_t a3[4] = {gelu_f16x2(h0[0], h0[1]), gelu_f16x2(h0[2], h0[3]),
                            gelu_f16x2(h1[0], h1[1]), gelu_f16x2(h1[2], h1[3])};
    mma_16816(y, a3, lds32(&P.W3[g][k3 * 16 + 2 * t]), lds32(&P.W3[g][k3 * 16 + 2 * t + 8]));
  }
  Y[r0][2 * t] = y[0];
  Y[r0][2 * t + 1] = y[1];
  Y[r1][2 * t] = y[2];
  Y[r1][2 * t + 1] = y[3];
}

// Both m-tiles of 32 rows (one warp).
__device__ __forceinline__ void mlp_warp(const MlpPacked& P, const __half (*X)[24],
                                         float (*Y)[8]) {
  mlp_tile(P, X, Y, 0);
  mlp_tile(P, X, Y, 1);
}

// Cooperative copy of the packed weights into shared memory.
__device__ __forceinline__ void mlp_load(MlpPacked& dst, const MlpPacked* __restrict__ src) {
  const int n = (int)(sizeof(MlpPacked) / 16);
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&dst);
  for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = __ldg(s + i);
}

}  // namespace fvlb
