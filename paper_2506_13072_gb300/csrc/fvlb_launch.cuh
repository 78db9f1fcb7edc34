// fvlb_launch.cuh -- host-side launch logic, templated on the lattice; each
// lattice's translation unit instantiates it once.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "fvlb_internal.h"
#include "fvlb_kernels.cuh"

namespace fvlb {

// Tile shapes of the fused step: GX x TY groups of 32 x-consecutive nodes
// (a warp spans x, so every population load and store is one coalesced
// 128-byte line, shifted by at most one element for the pushes), C threads
// per node, optional fill warps (FW); MINB is the number of resident blocks
// per SM the register allocation must allow.  The shapes below were the
// fastest of those measured on GB300 (256^3 D3Q19, 2048^2 D2Q9).
// Launch-shape overrides from the environment, for tuning sweeps.
inline int tune_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoi(v) : dflt;
}

template <class R>
Phys<R> make_phys(const StepDesc& d) {
  Phys<R> p;
  p.tau_f = R(d.tau_f);
  p.inv_tau_f = R(1.0 / d.tau_f);
  p.inv_tau_h = R(1.0 / d.tau_h);
  p.kh = R(1.0 - 0.5 / d.tau_h);
  p.kf = R(1.0 - 0.5 / d.tau_f);
  p.eta_over_lam = R(d.eta_p / d.lambda);
  p.inv_lam = R(1.0 / d.lambda);
  p.four_roll = d.four_roll;
  p.Fv[0] = R(d.Fv[0]);
  p.Fv[1] = R(d.Fv[1]);
  p.Fv[2] = R(d.Fv[2]);
  p.amp = R(d.amp);
  const R* t = static_cast<const R*>(d.tables);
  p.sx = t;
  p.cxs = t ? t + d.nx : nullptr;
  p.sy = t ? t + 2 * d.nx : nullptr;
  p.cys = t ? t + 2 * d.nx + d.ny : nullptr;
  p.first = d.first;
  p.step = (uint32_t)d.step;
  p.lam = R(d.lambda);
  p.mlp = d.mlp;
  p.cl_tol2 = float(d.cl_tol * d.cl_tol);
  p.cl_count = d.cl_count;
  p.model = d.model;
  p.mpar = R(d.mpar);
  p.fdiv = nullptr;
  p.err = d.err;
  return p;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library does not link the driver API); null when it is unavailable
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// One tiled map without swizzle or interleave; dims[0] runs over the nodes
// of a population array, strides are the byte strides of dims 1 ...
inline bool encode_map(CUtensorMap* m, CUtensorMapDataType t, int rank, const void* base,
                       const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box) {
  const auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, t, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tensor maps of a fused launch whose warps stage rows of BX nodes
// (StageMaps in fvlb_kernels.cuh); `on` = 0 (the kernel's cp.async
// staging) when a row start cannot lie on a 16-byte boundary, a buffer is
// not 16-byte aligned, an encoding fails, or FVLB_STAGE_TMA=0.
template <class L, class S>
StageMaps stage_maps(const StepDesc& d, int BX) {
  StageMaps m;
  std::memset(&m, 0, sizeof m);
  constexpr int Q = L::Q, C = L::C, D = L::D;
  constexpr int NJ = (Q - C) / C + 1;
  constexpr cuuint64_t es = sizeof(S);
  if (tune_int("FVLB_STAGE_TMA", 1) == 0) return m;
  if (((cuuint64_t)d.nx * es) % 16 != 0 || ((cuuint64_t)d.pitch * es) % 16 != 0) return m;
  auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  if (!aligned(d.f_in) || !aligned(d.h_in) || !aligned(d.chi)) return m;
  const CUtensorMapDataType t =
      es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  const CUtensorMapDataType tf = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint64_t P = (cuuint64_t)d.pitch;
  const cuuint32_t bx = (cuuint32_t)BX;
  bool ok = true;
  {
    const cuuint64_t dims[2] = {P, (cuuint64_t)C * Q}, st[1] = {P * es};
    const cuuint32_t box[2] = {bx, (cuuint32_t)Q};
    ok = ok && encode_map(&m.h, t, 2, d.h_in, dims, st, box);
  }
  {
    const cuuint64_t dims[3] = {P, (cuuint64_t)C, (cuuint64_t)NJ}, st[2] = {P * es, C * P * es};
    const cuuint32_t box[3] = {bx, 1, (cuuint32_t)NJ};
    ok = ok && encode_map(&m.f3, t, 3, d.f_in, dims, st, box);
  }
  if (Split<L>::nf(0) > NJ) {
    const cuuint64_t dims[2] = {P, (cuuint64_t)NJ + 1}, st[1] = {C * P * es};
    const cuuint32_t box[2] = {bx, (cuuint32_t)NJ + 1};
    ok = ok && encode_map(&m.f4, t, 2, d.f_in, dims, st, box);
  }
  {
    static_assert(sizeof(typename Store<S>::X) == 4, "chi is staged as 4-byte values");
    const cuuint64_t dims[2] = {P, (cuuint64_t)C}, st[1] = {P * 4};
    const cuuint32_t box[2] = {bx, 1};
    ok = ok && encode_map(&m.x, tf, 2, d.chi, dims, st, box);
  }
  if constexpr (Store<S>::V2) {
    const char* h0 = static_cast<const char*>(d.h_in) + es * C * Q * P;
    const char* U = static_cast<const char*>(d.f_in) + es * Q * P;
    if (!aligned(h0) || !aligned(U)) return m;
    {
      const cuuint64_t dims[2] = {P, (cuuint64_t)C}, st[1] = {P * 4};
      const cuuint32_t box[2] = {bx, 1};
      ok = ok && encode_map(&m.e0, tf, 2, h0, dims, st, box);
    }
    {
      const cuuint64_t dims[2] = {P, (cuuint64_t)D}, st[1] = {P * 4};
      const cuuint32_t box[2] = {bx, (cuuint32_t)D};
      ok = ok && encode_map(&m.u, tf, 2, U, dims, st, box);
    }
  }
  m.on = ok ? 1 : 0;
  return m;
}

inline int grid_stride_blocks(long long N, int threads, int sms) {
  const long long want = (N + threads - 1) / threads;
  const long long cap = (long long)std::max(sms, 1) * 16;
  return (int)std::max<long long>(1, std::min(want, cap));
}

// Let kernel `kern` take `bytes` of dynamic shared memory on the current
// device: set once per device and kernel (before its first launch, so also
// before a stream capture that contains one).
template <class K>
cudaError_t allow_dynamic_smem(K* kern, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;  // (kernel, device) set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const std::pair<const void*, int> key{reinterpret_cast<const void*>(kern), dev};
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& d : done)
    if (d == key) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.push_back(key);
  return e;
}

// Launch a fused-step kernel instance; a tile of more than 48 KB of shared
// memory (XN > 1) is given it dynamically.
template <class L, class S, int GX, int TY, int MINB, bool WALLS, bool FW, bool CL, int XN,
          bool ORIG = false>
cudaError_t launch_kernel(dim3 grid, const StepDesc& d, const Grid& g, const Phys<RT<S>>& ph,
                          const Bufs<S>& b, int mchunk, const StageMaps& tm) {
  constexpr int NT = FusedShape<L, GX, TY, FW, XN, fill_warps_max<S, XN>()>::NT;
  constexpr size_t dyn = TileCfg<L, S, GX, TY, FW, CL, XN, MINB>::kDynamicBytes;
  auto kern = k_step_fused<L, S, GX, TY, MINB, WALLS, FW, CL, XN, ORIG>;
  if constexpr (dyn > 0) {
    const cudaError_t e = allow_dynamic_smem(kern, dyn);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, NT, dyn, d.stream>>>(g, ph, b, mchunk, tm);
  return cudaGetLastError();
}

template <class L, class S, int GX, int TY, int MINB, bool FW, int XN = 1, bool ORIG = false>
cudaError_t launch_fused(const StepDesc& d, const Grid& g, const Phys<RT<S>>& ph,
                         const Bufs<S>& b) {
  constexpr int TXS = GX * 32 * XN;
  const int bx = (d.nx + TXS - 1) / TXS;
  const int by = L::D == 3 ? (d.ny + TY - 1) / TY : 1;
  const int nm = L::D == 3 ? g.nz : d.ny;
  // chunks along the march axis: enough blocks for several waves, but at
  // least `min_chunk` planes so the two halo planes stay a small overhead
  const int waves = tune_int("FVLB_WAVES", L::D == 2 ? 4 : 16);
  const int min_chunk = tune_int("FVLB_MIN_CHUNK", 8);
  const long long target = (long long)std::max(d.sms, 1) * MINB * waves;
  int nchunk = (int)std::max<long long>(1, target / std::max(1, bx * by));
  int mchunk = std::max(min_chunk, (nm + nchunk - 1) / nchunk);
  mchunk = std::min(mchunk, nm);
  nchunk = (nm + mchunk - 1) / mchunk;
  dim3 grid(bx, by, nchunk);
  StageMaps tm;
  std::memset(&tm, 0, sizeof tm);
  if constexpr (TileCfg<L, S, GX, TY, FW, false, XN, MINB>::PF) tm = stage_maps<L, S>(d, 32 * XN);
  if constexpr (std::is_same<S, float>::value && XN == 1 && !ORIG && (L::D == 3 || !FW)) {
    if (d.mlp) {  // learned closure (FP32 storage only); two blocks per SM
      if (d.walls) return launch_kernel<L, S, GX, TY, 2, true, FW, true, 1>(grid, d, g, ph, b, mchunk, tm);
      return launch_kernel<L, S, GX, TY, 2, false, FW, true, 1>(grid, d, g, ph, b, mchunk, tm);
    }
  }
  if (d.walls)
    return launch_kernel<L, S, GX, TY, MINB, true, FW, false, XN, ORIG>(grid, d, g, ph, b, mchunk, tm);
  return launch_kernel<L, S, GX, TY, MINB, false, FW, false, XN, ORIG>(grid, d, g, ph, b, mchunk, tm);
}

// The fused step in the shape measured fastest on GB300 (256^3 D3Q19, 2048^2
// D2Q9): 2D four 32-node groups x 3 components + 5 (FP32) or 4 (16-bit) halo
// fill warps (544 / 512 threads, 2 blocks per SM; FP64 and the learned
// closure without fill warps, 384 threads); 3D FP32 and 16-bit a 64-node row, each of the 6 component warps
// taking its two 32-node halves in turn, + 7 (FP32) or 4 (16-bit) halo fill
// warps (416 / 320 threads, 2 blocks per SM; a 64-register cap for 3 blocks
// per SM measured slower); 3D FP64 and the learned closure one 32-node row
// with 4 fill warps.  ORIG: the original scheme's
// step (div tau_p from ph.fdiv in the body force, f^B off).
template <class L, class S, bool ORIG>
cudaError_t fused_step(const StepDesc& d, const Grid& g, const Phys<RT<S>>& ph,
                       const Bufs<S>& b) {
  constexpr bool wide = sizeof(RT<S>) == 8;
  if constexpr (L::D == 2) {
    // 4 groups x 3 components; FP64 and the learned closure fill the ring
    // in the collision threads, FP32 and 16-bit storage with fill warps
    if constexpr (wide) {
      return launch_fused<L, S, 4, 1, 1, false, 1, ORIG>(d, g, ph, b);
    } else {
      if constexpr (!ORIG) {
        if (d.mlp) return launch_fused<L, S, 4, 1, 2, false, 1>(d, g, ph, b);
      }
      return launch_fused<L, S, 4, 1, 2, true, 1, ORIG>(d, g, ph, b);
    }
  } else {
    if constexpr (wide) return launch_fused<L, S, 1, 1, 1, true, 1, ORIG>(d, g, ph, b);
    else if constexpr (sizeof(S) == 4) {
      if constexpr (!ORIG) {
        if (d.mlp) return launch_fused<L, S, 1, 1, 2, true, 1>(d, g, ph, b);
      }
      return launch_fused<L, S, 1, 1, 2, true, 2, ORIG>(d, g, ph, b);
    } else {
      return launch_fused<L, S, 1, 1, 2, true, 2, ORIG>(d, g, ph, b);
    }
  }
}

template <class L, class S>
cudaError_t step_impl(const StepDesc& d) {
  using R = RT<S>;
  using X = typename Store<S>::X;
  Grid g{d.nx, d.ny, L::D == 3 ? d.nz : 1, d.walls, d.pitch};
  Phys<R> ph = make_phys<R>(d);
  Bufs<S> b{static_cast<const S*>(d.f_in), static_cast<S*>(d.f_out),
            static_cast<const S*>(d.h_in), static_cast<S*>(d.h_out),
            static_cast<X*>(d.chi)};
  if (d.scheme == 1) {
    // the original scheme: the polymer stress of every node, then either its
    // divergence per node and the fused step with it as part of the body
    // force and f^B off (three launches), or the split velocity and
    // collision kernels, which take the divergence themselves
    const int threads = 128;
    const int blocks = grid_stride_blocks(d.N, threads, d.sms);
    R* taup = static_cast<R*>(d.taup);
    k_taup<L, S><<<blocks, threads, 0, d.stream>>>(g, ph, b.h_in, taup, d.N);
    if constexpr (sizeof(S) >= 4) {  // fused form for FP32 and FP64 storage
      if (d.variant == 0 && !d.mlp) {
        R* fdiv = static_cast<R*>(d.fdiv);
        k_fdiv<L, S><<<blocks, threads, 0, d.stream>>>(g, taup, fdiv, d.N);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ph.fdiv = fdiv;
        return fused_step<L, S, true>(d, g, ph, b);
      }
    }
    R* ubuf = static_cast<R*>(d.ubuf);
    k_velocity<L, S, true><<<blocks, threads, 0, d.stream>>>(g, ph, b.f_in, ubuf, taup, d.N);
    k_collide_split<L, S, true, true><<<blocks, threads, 0, d.stream>>>(g, ph, b, ubuf, taup, d.N);
    return cudaGetLastError();
  }
  if (d.variant == 0) {
    return fused_step<L, S, false>(d, g, ph, b);
  } else {
    const int threads = 128;
    const int blocks = grid_stride_blocks(d.N, threads, d.sms);
    R* ubuf = static_cast<R*>(d.ubuf);
    k_velocity<L, S><<<blocks, threads, 0, d.stream>>>(g, ph, b.f_in, ubuf, nullptr, d.N);
    k_collide_split<L, S, true><<<blocks, threads, 0, d.stream>>>(g, ph, b, ubuf, nullptr, d.N);
  }
  return cudaGetLastError();
}

template <class L, class S>
cudaError_t init_impl(const InitDesc& d) {
  Grid g{d.nx, d.ny, L::D == 3 ? d.nz : 1, 0, d.pitch};
  const int threads = 256;
  const int blocks = grid_stride_blocks(d.N, threads, d.sms);
  k_init<L, S><<<blocks, threads, 0, d.stream>>>(
      g, static_cast<S*>(d.f), static_cast<S*>(d.h),
      static_cast<typename Store<S>::X*>(d.chi), d.u0, d.p0, d.A0, d.N);
  return cudaGetLastError();
}

template <class L, class S>
cudaError_t fields_impl(const StepDesc& d, int which, double* out) {
  using R = RT<S>;
  Grid g{d.nx, d.ny, L::D == 3 ? d.nz : 1, d.walls, d.pitch};
  Phys<R> ph = make_phys<R>(d);
  const int threads = 256;
  const int blocks = grid_stride_blocks(d.N, threads, d.sms);
  const S* f = static_cast<const S*>(d.f_in);
  const S* h = static_cast<const S*>(d.h_in);
  if (d.scheme == 1) {
    R* taup = static_cast<R*>(d.taup);
    k_taup<L, S><<<blocks, threads, 0, d.stream>>>(g, ph, h, taup, d.N);
    k_fields<L, S, true><<<blocks, threads, 0, d.stream>>>(g, ph, f, h, which, out, taup, d.N);
  } else {
    k_fields<L, S><<<blocks, threads, 0, d.stream>>>(g, ph, f, h, which, out, nullptr, d.N);
  }
  return cudaGetLastError();
}

template <class L, class S>
cudaError_t reduce_impl(const StepDesc& d, double* part, double* out) {
  using R = RT<S>;
  Grid g{d.nx, d.ny, L::D == 3 ? d.nz : 1, d.walls, d.pitch};
  Phys<R> ph = make_phys<R>(d);
  const int nparts = reduce_parts(d.N);
  const S* f = static_cast<const S*>(d.f_in);
  const S* h = static_cast<const S*>(d.h_in);
  if (d.scheme == 1) {
    R* taup = static_cast<R*>(d.taup);
    k_taup<L, S><<<grid_stride_blocks(d.N, 256, d.sms), 256, 0, d.stream>>>(g, ph, h, taup, d.N);
    k_reduce_partial<L, S, true><<<nparts, kReduceThreads, 0, d.stream>>>(g, ph, f, h, part, d.N,
                                                                          taup);
  } else {
    k_reduce_partial<L, S><<<nparts, kReduceThreads, 0, d.stream>>>(g, ph, f, h, part, d.N);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return reduce_finalize(part, nparts, d.N, out, d.stream);
}

template <class L, class S>
cudaError_t conf_impl(const StepDesc& d, double* part, double* out) {
  Grid g{d.nx, d.ny, L::D == 3 ? d.nz : 1, d.walls, d.pitch};
  const int nparts = reduce_parts(d.N);
  k_conf_partial<L, S><<<nparts, kReduceThreads, 0, d.stream>>>(
      g, static_cast<const S*>(d.h_in), part, d.N);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_conf_final<<<1, kReduceThreads, 0, d.stream>>>(part, nparts, out);
  return cudaGetLastError();
}

template <class L, class S>
cudaError_t repair_impl(const StepDesc& d, double eps, unsigned long long* count) {
  Grid g{d.nx, d.ny, L::D == 3 ? d.nz : 1, d.walls, d.pitch};
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), d.stream);
  if (e != cudaSuccess) return e;
  k_repair<L, S><<<grid_stride_blocks(d.N, kReduceThreads, d.sms), kReduceThreads, 0, d.stream>>>(
      g, static_cast<S*>(const_cast<void*>(d.h_in)), eps, count, d.N);
  return cudaGetLastError();
}

// step_impl is instantiated per (lattice, storage) in its own translation
// unit (k_step_<lattice>_<storage>.cu) so that the library builds in parallel.
#define FVLB_EXTERN_STEP(L)                                                   \
  extern template cudaError_t step_impl<L, double>(const StepDesc&);        \
  extern template cudaError_t step_impl<L, float>(const StepDesc&);         \
  extern template cudaError_t step_impl<L, __half>(const StepDesc&);        \
  extern template cudaError_t step_impl<L, __nv_bfloat16>(const StepDesc&); \
  extern template cudaError_t step_impl<L, half_sr>(const StepDesc&);       \
  extern template cudaError_t step_impl<L, bf16_sr>(const StepDesc&);

#define FVLB_DISPATCH(storage, CALL)                              \
  switch (storage) {                                              \
    case kFP64: return CALL(double);                              \
    case kFP32: return CALL(float);                               \
    case kFP16Dev: return CALL(__half);                           \
    case kBF16Dev: return CALL(__nv_bfloat16);                    \
    case kFP16DevSR: return CALL(half_sr);                        \
    case kBF16DevSR: return CALL(bf16_sr);                        \
    default: return cudaErrorInvalidValue;                        \
  }

}  // namespace fvlb
