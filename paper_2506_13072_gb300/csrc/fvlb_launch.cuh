// fvlb_launch.cuh -- host-side launch logic, templated on the lattice; each
// lattice's translation unit instantiates it once.
#pragma once

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>
#include <cstdlib>
#include <type_traits>

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
  return p;
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
                          const Bufs<S>& b, int mchunk) {
  constexpr int NT = FusedShape<L, GX, TY, FW, XN>::NT;
  constexpr size_t dyn = TileCfg<L, S, GX, TY, FW, CL, XN, MINB>::kDynamicBytes;
  auto kern = k_step_fused<L, S, GX, TY, MINB, WALLS, FW, CL, XN, ORIG>;
  if constexpr (dyn > 0) {
    const cudaError_t e = allow_dynamic_smem(kern, dyn);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, NT, dyn, d.stream>>>(g, ph, b, mchunk);
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
  if constexpr (std::is_same<S, float>::value && XN == 1 && !ORIG) {
    if (d.mlp) {  // learned closure (FP32 storage only); two blocks per SM
      if (d.walls) return launch_kernel<L, S, GX, TY, 2, true, FW, true, 1>(grid, d, g, ph, b, mchunk);
      return launch_kernel<L, S, GX, TY, 2, false, FW, true, 1>(grid, d, g, ph, b, mchunk);
    }
  }
  if (d.walls)
    return launch_kernel<L, S, GX, TY, MINB, true, FW, false, XN, ORIG>(grid, d, g, ph, b, mchunk);
  return launch_kernel<L, S, GX, TY, MINB, false, FW, false, XN, ORIG>(grid, d, g, ph, b, mchunk);
}

// The fused step in the shape measured fastest on GB300 (256^3 D3Q19, 2048^2
// D2Q9): 2D four 32-node groups x 3 components (384 threads, 2 blocks per
// SM); 3D FP32 a 64-node row, each of the 6 component warps taking its two
// 32-node halves in turn, + 4 halo fill warps (320 threads, 2 blocks per SM;
// a 64-register cap for 3 blocks per SM measured slower); 3D 16-bit, FP64
// and the learned closure one 32-node row.  ORIG: the original scheme's
// step (div tau_p from ph.fdiv in the body force, f^B off).
template <class L, class S, bool ORIG>
cudaError_t fused_step(const StepDesc& d, const Grid& g, const Phys<RT<S>>& ph,
                       const Bufs<S>& b) {
  constexpr bool wide = sizeof(RT<S>) == 8;
  if constexpr (L::D == 2) {
    // 4 groups x 3 components, ring filled by the collision threads
    if constexpr (wide) return launch_fused<L, S, 4, 1, 1, false, 1, ORIG>(d, g, ph, b);
    else return launch_fused<L, S, 4, 1, 2, false, 1, ORIG>(d, g, ph, b);
  } else {
    if constexpr (wide) return launch_fused<L, S, 1, 1, 1, true, 1, ORIG>(d, g, ph, b);
    else if constexpr (sizeof(S) == 4) {
      if constexpr (!ORIG) {
        if (d.mlp) return launch_fused<L, S, 1, 1, 2, true, 1>(d, g, ph, b);
      }
      return launch_fused<L, S, 1, 1, 2, true, 2, ORIG>(d, g, ph, b);
    } else {
      return launch_fused<L, S, 1, 1, 2, true, 1, ORIG>(d, g, ph, b);
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
