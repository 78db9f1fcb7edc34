// fvlb_kernels.cuh -- CUDA kernels of one fluctuating-LB time step
// (arXiv 2506.13072, Sec. 2.2 flow LB with f^B and Guo forcing, Sec. 2.3
// conformation LB), plus initialisation, field extraction and the FP64
// diagnostics reduction.
//
// Data layout in HBM (structure of arrays, x fastest, each array padded to
// `pitch` elements):  f[Q][pitch], h[C][Q][pitch], chi[C][pitch].  The state
// is double-buffered (f and h read from one buffer, written to the other);
// chi is read and rewritten in place by its own site only.
//
// A step is "collide, then push": the site reads its own populations
// (coalesced, unshifted), collides, and writes population i to the
// neighbour x + c_i of the other buffer (or, through a halfway-bounce-back
// wall, to its own node in the opposite direction).  The velocity gradient
// in chi needs the same-step velocity of the 2 (2D) or 6 (3D) nearest
// neighbours, which with push streaming are one node away, so a one-node
// velocity halo suffices.
#pragma once

#include <cuda.h>   // CUtensorMap (the type only; maps are encoded on the host)

#include <type_traits>

#include "fvlb_lattice.cuh"
#include "fvlb_mlp.cuh"

namespace fvlb {

template <class S>
using RT = typename Store<S>::R;

// Asynchronous global -> shared copies (cp.async, one element per thread);
// the copies of a thread become visible to it after cp_wait_all.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
  else if constexpr (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
// wait until at most N of this thread's most recent groups are pending
template <int N>
__device__ __forceinline__ void cp_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Bulk tensor copies (TMA) into shared memory, completed on an mbarrier.
// A warp's lane 0 arms the barrier with the byte count of its copies and
// issues them; every lane of the warp waits for the barrier's phase.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make initialised barriers visible to the copy engine
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait for the phase of parity `parity` to complete, for at most about 2 s;
// on time-out record bit 0 in *err (when given) and return false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > 2000000000ull) {
      if (err) atomicOr(err, 1u);
      return false;
    }
  }
  return true;
}
// order this thread's earlier shared-memory accesses before later accesses
// of the copy engine to the same memory
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2),
      "r"(smem_addr(bar))
      : "memory");
}

// Tensor maps of one launch's staged arrays (the fused step's copies of a
// warp's row of nodes into its stage buffer), encoded on the host; `on` = 0:
// the warps copy with cp.async instead.  Dimension 0 is the node index
// within a population array (x fastest, `pitch` long), so a box of BX
// nodes is one warp's row; the arrays must start on 16-byte boundaries and
// a box's first node must lie on one (nx a multiple of 16 / element size).
struct StageMaps {
  CUtensorMap h;    // h[C Q][pitch]; box BX x Q: component k's rows k Q ..
  CUtensorMap f3;   // f as [J][C][pitch]; box BX x 1 x J: rows k + j C, j < J
  CUtensorMap f4;   // D3Q19: f rows 0, C, 2C, 3C as [4][pitch]; box BX x 4
  CUtensorMap x;    // chi[C][pitch]; box BX x 1
  CUtensorMap e0;   // 16-bit forms: FP32 rest stress populations h0[C][pitch]; box BX x 1
  CUtensorMap u;    // 16-bit forms: FP32 velocities U[D][pitch]; box BX x D
  int on;
};

// Make a pointer opaque to the compiler at this point of the program.  Used
// to stop the 114 population addresses of a D3Q19 site from being computed
// once and kept live (in registers) between the two reads of the stress
// populations, which would cap the number of resident warps.
template <class T>
__device__ __forceinline__ T* opaque(T* p) {
  asm volatile("" : "+l"(p));
  return p;
}

// load f_i(s) (16-bit forms: s_i / KF + e_i(U) with the node's stored U)
template <class L, class S>
__device__ __forceinline__ void load_f(const S* __restrict__ f, long long pitch,
                                       long long s, RT<S> (&fv)[L::Q]) {
  using R = RT<S>;
  if constexpr (Store<S>::V2) {
    const float* U = f_ext<L>(f, pitch);
    R u[L::D];
#pragma unroll
    for (int a = 0; a < L::D; ++a) u[a] = U[a * pitch + s];
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      fv[i] = Store<S>::ld(f + i * pitch + s) * R(1.0f / Store<S>::KF) + feq_u<L, R>(i, u);
  } else {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) fv[i] = Store<S>::ld(f + i * pitch + s);
  }
}

// Stress populations are held as deviations from the rest equilibrium,
// h'_{k,i} = h_{k,i} - w_i delta_k (delta_k = 1 on diagonal components), in
// every storage precision: the conformation then enters as A - I = sum_i h'
// without the cancellation of summing h ~ w_i A and subtracting I.
// (16-bit forms: the rest population from its FP32 array)
template <class L, class S>
__device__ __forceinline__ RT<S> load_h(const S* __restrict__ h, long long pitch,
                                        long long s, int k, int i) {
  if constexpr (Store<S>::V2) {
    if (i == 0) return h_ext<L>(h, pitch)[k * pitch + s];
  }
  return Store<S>::ld(h + (long long)(k * L::Q + i) * pitch + s);
}

// second read of a stress population within one site update (served by L2);
// hs points at the site's first population
template <class L, class S>
__device__ __forceinline__ RT<S> reload_h(const S* hs, long long pitch, int k, int i) {
  return Store<S>::ld_l2(hs + (long long)(k * L::Q + i) * pitch);
}

template <class L, class S>
__device__ __forceinline__ void store_h(S* __restrict__ h, long long pitch,
                                        long long s, int k, int i, RT<S> v, uint32_t r) {
  Store<S>::st(h + (long long)(k * L::Q + i) * pitch + s, v, r);
}

template <class L>
__host__ __device__ constexpr bool diag(int k) {
  return L::ca(k) == L::cb(k);
}

// Streaming destination of population i leaving (x, y, z) (node s):
// periodic wrap, or halfway bounce-back to the same node, opposite direction.
template <class L>
__device__ __forceinline__ long long push_dest(const Grid& g, int i, int x, int y,
                                               int z, long long s, int& j) {
  int xd = x + L::cx(i), yd = y + L::cy(i), zd = z + L::cz(i);
  bool bb = false;
  if (L::cx(i) != 0 && (xd < 0 || xd >= g.nx)) {
    if (g.walls & 1) bb = true;
    else xd = xd < 0 ? xd + g.nx : xd - g.nx;
  }
  if (L::cy(i) != 0 && (yd < 0 || yd >= g.ny)) {
    if (g.walls & 2) bb = true;
    else yd = yd < 0 ? yd + g.ny : yd - g.ny;
  }
  if (L::D == 3 && L::cz(i) != 0 && (zd < 0 || zd >= g.nz)) {
    if (g.walls & 4) bb = true;
    else zd = zd < 0 ? zd + g.nz : zd - g.nz;
  }
  if (bb) {
    j = L::opp(i);
    return s;
  }
  j = i;
  return ((long long)zd * g.ny + yd) * g.nx + xd;
}

// p = c_s^2 / (1 - w_0) [sum_{i!=0} f_i + s_0(u) + tau_f F_0 + tau_f f^B_0]
// (Sec. 2.2, Appendix B) with F_0 = -3 w_0 (1 - 1/(2 tau_f)) F.u and
// s_0 = -1.5 w_0 |u|^2; returned as the pressure variable of p_part (p in
// FP64, p / (3 w_1) in FP32).
template <class L, class R>
__device__ __forceinline__ R pressure(const Phys<R>& ph, const R (&f)[L::Q],
                                      const R (&u)[L::D], const R F[3], R fB0) {
  R sum = R(0);
#pragma unroll
  for (int i = 1; i < L::Q; ++i) sum += f[i];
  R uu = R(0), Fu = R(0);
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    uu += u[a] * u[a];
    Fu += F[a] * u[a];
  }
  constexpr double w0 = L::w(0);
  const R s0 = R(-1.5 * w0) * uu;
  const R F0 = R(-3.0 * w0) * ph.kf * Fu;
  return p_part<L, R>(sum + s0 + ph.tau_f * F0 + ph.tau_f * fB0);
}

// ---------------------------------------------------------------------------
// Collide one site and push its populations.  u and gr (d_a u_b) are the
// site's velocity and velocity gradient of this step; f its populations.
// HOLD_H keeps all C*Q stress populations in registers (2D); otherwise the
// conformation is summed in a first pass and each component re-read for its
// collision (3D, where C*Q = 114).
// ORIG: the original scheme the paper compares with (Sec. 1, Tables 1-2):
// no fluctuation term f^B; the caller's F already holds the stress
// divergence, so it enters u, the pressure and the Guo term as a body force.
// ---------------------------------------------------------------------------
template <class L, class S, bool HOLD_H, bool ORIG = false>
__device__ __forceinline__ void collide_site(const Grid& g, const Phys<RT<S>>& ph,
                                             const Bufs<S>& b, long long s, int x,
                                             int y, int z, const RT<S> (&u)[L::D],
                                             const RT<S> (&gr)[L::D][L::D],
                                             const RT<S> (&f)[L::Q], const RT<S> F[3],
                                             const RT<S>* __restrict__ ubuf = nullptr) {
  using R = RT<S>;
  using X = typename Store<S>::X;
  constexpr int D = L::D, Q = L::Q, C = L::C;
  const long long P = g.pitch;
  // stochastic-rounding stream of this site and step (unused otherwise)
  uint32_t rng = Store<S>::sr ? hash32((uint32_t)s * 0x9e3779b9u ^ hash32(ph.step)) : 0u;

  // --- conformation A = I + sum_i h' (Sec. 2.3) --------------------------
  R Ad[C];  // A - I
  R hv[HOLD_H ? C : 1][HOLD_H ? Q : 1];
#pragma unroll
  for (int k = 0; k < C; ++k) {
    // Q loads in flight per component: keeps the register footprint (and so
    // the number of resident warps) bounded when the populations are re-read
    // below instead of held.
    const S* hk = HOLD_H ? b.h_in + s : opaque(b.h_in + s);
    R a = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R v = (Store<S>::V2 && i == 0) ? R(h_ext<L>(b.h_in, P)[k * P + s])
                                           : Store<S>::ld(hk + (long long)(k * Q + i) * P);
      if (HOLD_H) hv[HOLD_H ? k : 0][HOLD_H ? i : 0] = v;
      a += v;
    }
    Ad[k] = a;
  }
  // --- flow collision inputs (Sec. 2.2) ------------------------------------
  // f^B is linear in tau_p = (eta_p/lambda)(A - I): evaluate it on A - I with
  // the factor eta_p / (lambda tau_f) folded in.
  const R kB = ph.eta_over_lam * ph.inv_tau_f;
  R uu = R(0), Fu = R(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    uu += u[a] * u[a];
    Fu += F[a] * u[a];
  }
  const R fB0 = ORIG ? R(0) : fB_dir<L, R>(0, Ad, kB);
  const R p = pressure<L, R>(ph, f, u, F, fB0);

  // --- stress source (Sec. 2.3) ---------------------------------------------
  R src[C];
  {
    R A[C], chi[C];
#pragma unroll
    for (int k = 0; k < C; ++k) A[k] = Ad[k] + (diag<L>(k) ? R(1) : R(0));
    chi_tensor<L, R>(A, Ad, gr, ph, chi);
#pragma unroll
    for (int k = 0; k < C; ++k) {
      R old = R(b.chi[k * P + s]);
      if (ph.first) old = chi[k];
      b.chi[k * P + s] = X(chi[k]);
      // chi_i + 0.5 (chi_i^n - chi_i^{n-1}) = phi_i (1.5 chi - 0.5 chi_old)
      src[k] = R(1.5) * chi[k] - R(0.5) * old;
    }
  }

  // --- collide and push, one direction at a time ----------------------------
  // The destination of direction i is computed once and shared by f_i and
  // the C stress populations h_{k,i}.
  const S* hs = b.h_in + s;
  // 16-bit forms: the rest stress populations (stored last, in FP32, with
  // the rounding residuals of the component's other populations) and this
  // node's velocity for the flow populations it receives next step
  // The rest stress population keeps the node's populations summing to the
  // post-collision zeroth moment (as in the fused step): FP32 storage takes
  // it as that moment minus the other populations' sum; the 16-bit forms
  // take the rounding residuals less the rounded weights' excess
  constexpr bool RS = std::is_same<S, float>::value;
  constexpr double kWx = weight_sum_excess<L, R>();
  R h0post[Store<S>::V2 ? C : 1], hres[(Store<S>::V2 || RS) ? C : 1];
  if constexpr (RS) {
#pragma unroll
    for (int k = 0; k < C; ++k) hres[k] = R(0);
  }
  if constexpr (Store<S>::V2) {
#pragma unroll
    for (int k = 0; k < C; ++k) hres[k] = R(0);
    float* Uo = f_ext<L>(b.f_out, P);
#pragma unroll
    for (int a = 0; a < D; ++a) Uo[a * P + s] = float(u[a]);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (!HOLD_H && i % 3 == 0) hs = opaque(hs);
    R cu = R(0), cF = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int c = cc<L>(i, a);
      if (c == 1) { cu += u[a]; cF += F[a]; }
      if (c == -1) { cu -= u[a]; cF -= F[a]; }
    }
    int j;
    const long long d = push_dest<L>(g, i, x, y, z, s, j);
    const R wi = R(L::w(i));

    // flow: f* = f - (f - f^eq)/tau_f + f^B + F_i (Sec. 2.2)
    const R lam_i = R(p_coef<L, R>(i));
    const R w3i = R(w3<L, R>(i));
    const R feq = lam_i * p + (w3i * cu + wi * (R(4.5) * cu * cu - R(1.5) * uu));
    const R Fi = ph.kf * (w3i * cF + wi * (R(9) * cF * cu - R(3) * Fu));
    const R fBi = ORIG ? R(0) : fB_dir<L, R>(i, Ad, kB);
    const R fpost = f[i] - (f[i] - feq) * ph.inv_tau_f + fBi + Fi;
    if constexpr (Store<S>::V2) {
      // deviation from e_j(u) of the receiving node (velocity of this step)
      R ud[D];
#pragma unroll
      for (int a = 0; a < D; ++a) ud[a] = ubuf[a * P + d];
      Store<S>::st(b.f_out + j * P + d, R(Store<S>::KF) * (fpost - feq_u<L, R>(j, ud)),
                   Store<S>::sr ? lcg_next(rng) : 0u);
    } else {
      Store<S>::st(b.f_out + j * P + d, fpost, Store<S>::sr ? lcg_next(rng) : 0u);
    }

    // stress: h* = h - (h - h^eq)/tau_h + phi_i src, phi_i = w_i [1 + (1 - 1/(2 tau_h)) c.u/c_s^2]
    const R phi = wi * (R(1) + ph.kh * R(3) * cu);
#pragma unroll
    for (int k = 0; k < C; ++k) {
      R hi;
      if (HOLD_H) hi = hv[HOLD_H ? k : 0][HOLD_H ? i : 0];
      else if (Store<S>::V2 && i == 0) hi = R(h_ext<L>(b.h_in, P)[k * P + s]);
      else hi = reload_h<L, S>(hs, P, k, i);
      // h^eq - w_i delta_k = w_i [(A - I)_k + A_k c_i.u / c_s^2]
      const R heq = wi * (Ad[k] + (Ad[k] + (diag<L>(k) ? R(1) : R(0))) * (R(3) * cu));
      const R post = hi - (hi - heq) * ph.inv_tau_h + phi * src[k];
      if constexpr (Store<S>::V2) {
        if (i == 0) {
          // less the weights' excess times the weight-proportional part
          h0post[k] = post - R(kWx) * (ph.inv_tau_h * Ad[k] + src[k]);
        } else {
          S* q = b.h_out + (long long)(k * Q + j) * P + d;
          hres[k] -= Store<S>::st_d(q, post, Store<S>::sr ? lcg_next(rng) : 0u);
        }
      } else if constexpr (RS) {
        if (i != 0) {
          hres[k] += post;
          store_h<L, S>(b.h_out, P, d, k, j, post, 0u);
        }
      } else {
        store_h<L, S>(b.h_out, P, d, k, j, post, Store<S>::sr ? lcg_next(rng) : 0u);
      }
    }
  }
  if constexpr (RS) {
#pragma unroll
    for (int k = 0; k < C; ++k) store_h<L, S>(b.h_out, P, s, k, 0, (Ad[k] + src[k]) - hres[k], 0u);
  }
  if constexpr (Store<S>::V2) {
    float* h0o = h_ext<L>(b.h_out, P);
#pragma unroll
    for (int k = 0; k < C; ++k) h0o[k * P + s] = float(h0post[k] + hres[k]);
  }
}

// ---------------------------------------------------------------------------
// Fused step: one launch per time step, component-parallel.
//
// Tile: a block owns GX x TY groups of 32 consecutive x-nodes (2D: GX groups
// in one row, TY = 1; 3D: GX x TY groups in an x-y tile) and marches along
// the slowest axis (2D: y, 3D: z) over a chunk of `mchunk` planes.
//
// Work split: each node of a plane is updated by C threads, one per
// symmetric stress component k (C = 3 in 2D, 6 in 3D), in C different warps
// of the same group, so a warp reads and writes one component's populations
// h_{k,i} of 32 consecutive nodes (coalesced).  Thread k also collides and
// pushes the flow populations f_i with i = k (mod C).  The nodes' A - I
// components and the partial sums of f entering the pressure are exchanged
// through shared memory.  Holding Q + ceil(Q/C) populations instead of
// Q (1 + C) keeps the register footprint low enough for many resident warps.
//
// Velocity gradient: the same-step velocity of the tile and a one-node halo
// is kept in a four-plane shared-memory ring (planes m-1 .. m+2).  Separate
// fill warps compute it from the populations of plane m+2 while the
// collision warps update plane m, so the fill's memory latency hides behind
// the collision; halo velocities are recomputed from their populations (read
// through L2), so blocks never wait on each other.  Per plane: the collision
// warps' memory phase, barrier, collision phase (with the fill running),
// barrier.
// ---------------------------------------------------------------------------
template <class L>
struct Split {
  // number of flow directions owned by component k
  __host__ __device__ static constexpr int nf(int k) { return (L::Q - k + L::C - 1) / L::C; }
  static constexpr int NFMAX = (L::Q + L::C - 1) / L::C;
};

// Velocity of a ring slot: the D components in one 16-byte (FP32) or
// 32-byte (FP64) record, so a slot is read and written with vector
// shared-memory accesses.
template <class R, int D>
struct alignas(sizeof(R) * (D == 3 ? 4 : 2)) Vel {
  R v[D == 3 ? 4 : 2];
};

// out[0..N) = p[0..N) from shared memory, p 16-byte aligned, in 16- and
// 8-byte pieces.
template <class R, int N>
__device__ __forceinline__ void lds_row(const R* p, R (&out)[N]) {
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int j = 0; j + 4 <= N; j += 4) {
      const float4 t = *reinterpret_cast<const float4*>(p + j);
      out[j] = t.x; out[j + 1] = t.y; out[j + 2] = t.z; out[j + 3] = t.w;
    }
    if constexpr (N % 4 >= 2) {
      const float2 t = *reinterpret_cast<const float2*>(p + N / 4 * 4);
      out[N / 4 * 4] = t.x; out[N / 4 * 4 + 1] = t.y;
    }
    if constexpr (N % 2 == 1) out[N - 1] = p[N - 1];
  } else {
#pragma unroll
    for (int j = 0; j + 2 <= N; j += 2) {
      const double2 t = *reinterpret_cast<const double2*>(p + j);
      out[j] = t.x; out[j + 1] = t.y;
    }
    if constexpr (N % 2 == 1) out[N - 1] = p[N - 1];
  }
}

// Call fn(std::integral_constant<int, k>) for a run-time component index
// k < 6 (the callee ignores k >= its lattice's C).
template <class Fn>
__device__ __forceinline__ void on_component(int k, Fn&& fn) {
  switch (k) {
    case 0: fn(std::integral_constant<int, 0>{}); break;
    case 1: fn(std::integral_constant<int, 1>{}); break;
    case 2: fn(std::integral_constant<int, 2>{}); break;
    case 3: fn(std::integral_constant<int, 3>{}); break;
    case 4: fn(std::integral_constant<int, 4>{}); break;
    default: fn(std::integral_constant<int, 5>{}); break;
  }
}

// FW: dedicated fill warps computing the ring one plane ahead (D3Q19, where
// a halo velocity costs 19 loads), or the ring filled by the first NE
// collision threads in their own memory phase (D2Q9, 9 loads).
// XN: nodes per collision thread along x; a collision warp covers XN rows
// of 32 consecutive nodes of one plane, one after the other (with fill
// warps only).  Up to four fill warps, each thread filling SPF ring slots.
// Most fill warps of a tile.  FP32: one ring slot per fill thread (3D
// 64-node rows 7 warps at 72 registers, measured 3 % faster than 4 warps of
// two slots each at 96; D2Q9 128-node tiles 5 warps at 56 registers, 7 %
// faster than 4); 4 otherwise (the 16-bit forms spill with more).
template <class S, int XN>
__host__ __device__ constexpr int fill_warps_max() {
  return sizeof(S) == 4 ? (XN == 2 ? 7 : 5) : 4;
}

// Fill warps that take x-neighbouring node pairs (see fused_tile).
template <class S, int XN>
__host__ __device__ constexpr bool fill_pairs() {
  return sizeof(S) == 2;
}

template <class L, int GX, int TY, bool FW, int XN = 1, int NFWM = 4>
struct FusedShape {
  static constexpr int NG = GX * TY;              // groups of 32 x XN nodes per plane tile
  static constexpr int NCW = NG * L::C;           // collision warps
  static constexpr int TXS = GX * 32 * XN;        // tile extent along x
  static constexpr int EX = TXS + 2;
  static constexpr int EY = (L::D == 3) ? TY + 2 : 1;
  static constexpr int NE = EX * EY;              // ring slots per plane
  static constexpr int NFW = FW ? ((NE + 31) / 32 < NFWM ? (NE + 31) / 32 : NFWM) : 0;  // fill warps
  static constexpr int SPF = FW ? (NE + NFW * 32 - 1) / (NFW * 32) : 0;  // slots per fill thread
  static constexpr int NT = (NCW + NFW) * 32;     // threads
};

// Shared memory of the learned closure in a tile: the packed network, the
// BF16 input rows and FP32 output rows of each group's warp, and the chosen
// chi of every node.
template <int NG, int C, int NS>
struct ClosureSmem {
  MlpPacked P;
  __half X[NG][32][24];
  float Y[NG][32][8];
  float chi[C][NS];
};
struct NoClosureSmem {
  int unused;
};

// Shared memory of one tile and the choices that depend on its size.
//  - Stage (PF): the next planes' populations of every collision thread
//    (Q stress populations and its flow populations, chi, and the 16-bit
//    forms' FP32 arrays), copied with bulk tensor copies or cp.async: FP32
//    and 16-bit storage.  NST buffers: the copies run NST - 1 planes ahead
//    of the collision (three where the budget allows, else two).
//  - The exchange arrays sAd / sPf are double-buffered by plane parity where
//    the budget allows: plane m + 1 then writes the other copy while slower
//    warps still read plane m's, and one barrier per plane suffices
//    (otherwise a second barrier closes each plane).  Node-major, each
//    node's C values padded to CP for vector loads.
// The budget is the 48 KB of static shared memory for one node per thread;
// with more, the tile lives in dynamic shared memory sized for MINB blocks
// per SM (two: 110 KB; three: 72 KB).
template <class L, class S, int GX, int TY, bool FW, bool CL, int XN, int MINB = 2>
struct TileCfg {
  using R = RT<S>;
  using X = typename Store<S>::X;
  using Sh = FusedShape<L, GX, TY, FW, XN, fill_warps_max<S, XN>()>;
  static constexpr int D = L::D, Q = L::Q, C = L::C;
  static constexpr int NS = Sh::NG * 32 * XN;     // nodes per plane tile
  static constexpr int NFM = Split<L>::NFMAX;
  static constexpr int NPP = Q + NFM;             // staged populations per thread
  static constexpr int BX = 32 * XN;              // stage columns of one warp
  static constexpr int CP = C == 6 ? 8 : 4;
  static constexpr bool PF = sizeof(S) == 4 || sizeof(S) == 2;
  using CLS = typename std::conditional<CL, ClosureSmem<Sh::NG, C, NS>, NoClosureSmem>::type;
  static constexpr size_t kRing = sizeof(Vel<R, D>) * 4 * Sh::NE;
  // 16-bit forms: the FP32 rest stress population of the thread's
  // component and the node's stored velocity U, staged beside the rest
  static constexpr bool V2 = Store<S>::V2;
  static constexpr int NEX = 1 + D;
  // One collision warp's stage buffer: its component's Q stress populations
  // and its NFM flow populations (i = k + j C) of the warp's BX nodes, chi,
  // and (16-bit forms) the FP32 rest population and U; every part starts
  // on a 128-byte boundary, as a bulk tensor copy into it requires.
  struct WStage0 {
    alignas(128) S h[Q][BX];
    alignas(128) S f[NFM][BX];
    alignas(128) X chi[BX];
  };
  struct WStageV2 : WStage0 {
    alignas(128) float ext[NEX][BX];
  };
  using WStage = typename std::conditional<V2, WStageV2, WStage0>::type;
  static constexpr size_t kStage1 = PF ? sizeof(WStage) * Sh::NCW : 0;
  static constexpr size_t kEx1 = 2 * sizeof(R) * CP * NS;
  // dynamic shared memory: several rows per thread, a staged 2D tile, a
  // staged 16-bit tile or a staged tile with the learned closure (whose
  // stages fill the static 48 KB and leave no room for the double-buffered
  // exchange or a third stage)
  static constexpr bool kDynamic = XN > 1 || (PF && (D == 2 || V2 || CL));
  static constexpr size_t kLimit = kDynamic ? (MINB >= 3 ? 72 : 110) * 1024 : 48 * 1024;
  static constexpr int NST =
      (PF && kRing + sizeof(CLS) + 3 * kStage1 + 2 * kEx1 <= kLimit) ? 3 : 2;
  static constexpr int NBUF = (kRing + sizeof(CLS) + NST * kStage1 + 2 * kEx1 <= kLimit) ? 2 : 1;
  using Stage = typename std::conditional<PF, WStage[NST][Sh::NCW], int>::type;
  struct Smem {
    Vel<R, D> ring[4][Sh::NE];                    // velocity of planes m-1 .. m+2
    alignas(16) R sAd[NBUF][NS][CP];              // A - I of the tile nodes
    alignas(16) R sPf[NBUF][NS][CP];              // partial sums of f_{i != 0}
    CLS cls;                                      // learned closure (CL only)
    alignas(128) Stage stage;
    uint64_t bar[PF ? NST : 1][Sh::NCW];          // bulk-copy barriers of the stage buffers
  };
  static constexpr size_t kDynamicBytes = kDynamic ? sizeof(Smem) : 0;
};

// One tile of the fused step: tile (bx, by) of the plane, chunk bz of the
// march axis.  Called by k_step_fused (one tile per block) and by the
// batched persistent kernel (many tiles of many grids per block).
template <class L, class S, int GX, int TY, bool WALLS, bool FW, bool CL = false, int XN = 1,
          bool ORIG = false, int MINB = 2>
__device__ __forceinline__ void fused_tile(const Grid& g, const Phys<RT<S>>& ph,
                                           const Bufs<S>& b, int mchunk, int bx, int by,
                                           int bz, const StageMaps* tm = nullptr) {
  using R = RT<S>;
  using X = typename Store<S>::X;
  using Sh = FusedShape<L, GX, TY, FW, XN, fill_warps_max<S, XN>()>;
  using Cfg = TileCfg<L, S, GX, TY, FW, CL, XN, MINB>;
  constexpr int D = L::D, Q = L::Q, C = L::C;
  constexpr int NCW = Sh::NCW, TXS = Sh::TXS, EX = Sh::EX, NE = Sh::NE;
  constexpr int NFW = Sh::NFW, SPF = Sh::SPF;
  constexpr int NFM = Cfg::NFM, NPP = Cfg::NPP, NST = Cfg::NST, NBUF = Cfg::NBUF;
  constexpr bool PF = Cfg::PF;
  constexpr bool PAIR = sizeof(S) == 2;
  static_assert(D == 3 || TY == 1, "2D tiles are one row high");
  static_assert(FW || NE <= NCW * 32, "in-collision fill: one ring slot per thread");
  static_assert(XN == 1 || (FW && PF), "several nodes per thread: fill warps, staged storage");
  static_assert(!CL || std::is_same<R, float>::value, "the learned closure runs in FP32");
  using Sm = typename Cfg::Smem;
  Sm* smp;
  if constexpr (Cfg::kDynamic) {
    extern __shared__ __align__(128) unsigned char fvlb_tile_smem[];
    smp = reinterpret_cast<Sm*>(fvlb_tile_smem);
  } else {
    __shared__ Sm tile_smem;
    smp = &tile_smem;
  }
  auto& ring = smp->ring;
  auto& sAd = smp->sAd;
  auto& sPf = smp->sPf;
  auto& cls = smp->cls;
  auto& stage = smp->stage;
  (void)cls;
  (void)stage;

  const int nx = g.nx, ny = g.ny;
  const int nm = (D == 3) ? g.nz : g.ny;
  const bool wall_x = WALLS && (g.walls & 1);
  const bool wall_y = WALLS && (D == 3) && ((g.walls >> 1) & 1);
  const bool wall_m = WALLS && ((g.walls >> (D - 1)) & 1);
  const int x0 = bx * TXS;
  const int y0 = (D == 3) ? by * TY : 0;
  const int m0 = bz * mchunk;
  const int m1 = min(m0 + mchunk, nm);
  const long long P = g.pitch;
  const uint32_t P32 = (uint32_t)P;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const bool filler = warp >= NCW;      // fill warps: ring only
  if constexpr (CL) mlp_load(cls.P, static_cast<const MlpPacked*>(ph.mlp));
  auto slot = [&](int q) { return (q - m0 + 1) & 3; };
  auto plane_of = [&](int q) -> int {  // -1: beyond a wall
    if (q < 0 || q >= nm) return wall_m ? -1 : (q + nm) % nm;
    return q;
  };

  // ring slot e of a plane: its node, or none beyond a wall
  auto slot_node = [&](int e, int& gx, int& gy) -> bool {
    if (e >= NE) return false;
    const int ex = e % EX, ey = e / EX;
    gx = x0 + ex - 1;
    gy = (D == 3) ? y0 + ey - 1 : 0;
    if (gx < 0 || gx >= nx) {
      if (wall_x) return false;
      gx = ((gx % nx) + nx) % nx;
    }
    if (D == 3 && (gy < 0 || gy >= ny)) {
      if (wall_y) return false;
      gy = ((gy % ny) + ny) % ny;
    }
    return true;
  };
  // velocity of ring slot e of plane q from its populations fv (loaded by
  // the caller when `ok`), into the plane's ring slot.  16-bit forms: fv
  // holds the Q stored values and then the node's stored velocity U, and
  // u = U + sum_i c_i s_i / KF + F/2 (the velocity part e_i(U) of the
  // stored deviations carries momentum U and no other first moment).
  constexpr bool V2 = Cfg::V2;
  // FP32 storage: the rest stress population from the post-collision zeroth
  // moment (see the collision)
  constexpr bool RS = std::is_same<S, float>::value;
  constexpr int FQ = V2 ? Q + D : Q;
  auto fill_store = [&](int e, bool ok, int mm, int gx, int gy, const R (&fv)[FQ], int q) {
    R u[D];
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = R(0);
    if (ok) {
      R F[3];
      body_force<L, R>(ph, gx, D == 3 ? gy : mm, F);
      if constexpr (ORIG) {  // the original scheme: + div tau_p of this node
        const uint32_t sf = (D == 3) ? ((uint32_t)mm * (uint32_t)ny + (uint32_t)gy) * (uint32_t)nx + (uint32_t)gx
                                     : (uint32_t)mm * (uint32_t)nx + (uint32_t)gx;
#pragma unroll
        for (int a = 0; a < D; ++a) F[a] += ph.fdiv[(uint32_t)a * P32 + sf];
      }
      if constexpr (V2) {
        R fq[Q], z3[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int i = 0; i < Q; ++i) fq[i] = fv[i];
        velocity<L, R>(fq, z3, u);
#pragma unroll
        for (int a = 0; a < D; ++a)
          u[a] = u[a] * R(1.0f / Store<S>::KF) + fv[Q + a] + R(0.5) * F[a];
      } else {
        velocity<L, R>(fv, F, u);
      }
    }
    Vel<R, D> t;
#pragma unroll
    for (int a = 0; a < (D == 3 ? 4 : 2); ++a) t.v[a] = a < D ? u[a] : R(0);
    if constexpr (D == 3) t.v[3] = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];  // |u|^2
    ring[slot(q)][e] = t;
  };
  // fill_store from the raw 16-bit populations sb and FP32 U (16-bit forms):
  // the momentum sums take each population with one mixed-precision add or
  // subtract, the accumulator's sign tracked at compile time (f - v = -(v - f)
  // exactly), so the sums equal those of the converted values
  auto fill_store_bits = [&](int e, bool ok, int mm, int gx, int gy,
                             const unsigned short (&sb)[Q], const R (&Ub)[D], int q) {
    R u[D];
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = R(0);
    if constexpr (V2 && sizeof(S) == 2) {
      if (ok) {
        R F[3];
        body_force<L, R>(ph, gx, D == 3 ? gy : mm, F);
        if constexpr (ORIG) {
          const uint32_t sf = (D == 3) ? ((uint32_t)mm * (uint32_t)ny + (uint32_t)gy) * (uint32_t)nx + (uint32_t)gx
                                       : (uint32_t)mm * (uint32_t)nx + (uint32_t)gx;
#pragma unroll
          for (int a = 0; a < D; ++a) F[a] += ph.fdiv[(uint32_t)a * P32 + sf];
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
          R v = R(0);
          bool neg = false;   // v = -(momentum sum) while set
#pragma unroll
          for (int i = 1; i < Q; ++i) {
            const int c = cc<L>(i, a);
            if (c == 0) continue;
            if ((c == 1) != neg) {
              v = Store<S>::accb(v, sb[i]);
            } else {
              v = Store<S>::subb(sb[i], v);
              neg = !neg;
            }
          }
          const R m = neg ? -v : v;
          u[a] = m * R(1.0f / Store<S>::KF) + Ub[a] + R(0.5) * F[a];
        }
      }
    }
    Vel<R, D> t;
#pragma unroll
    for (int a = 0; a < (D == 3 ? 4 : 2); ++a) t.v[a] = a < D ? u[a] : R(0);
    if constexpr (D == 3) t.v[3] = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];  // |u|^2
    ring[slot(q)][e] = t;
  };
  auto fill_load = [&](bool ok, int mm, int gx, int gy, R (&fv)[FQ]) {
    if (ok) {
      // 32-bit offsets (Q * pitch < 2^32)
      const uint32_t s = (D == 3) ? ((uint32_t)mm * (uint32_t)ny + (uint32_t)gy) * (uint32_t)nx + (uint32_t)gx
                                  : (uint32_t)mm * (uint32_t)nx + (uint32_t)gx;
#pragma unroll
      for (int i = 0; i < Q; ++i) fv[i] = Store<S>::ld(b.f_in + ((uint32_t)i * P32 + s));
      if constexpr (V2) {
        const float* U = f_ext<L>(b.f_in, P);
#pragma unroll
        for (int a = 0; a < D; ++a) fv[Q + a] = __ldg(U + ((uint32_t)a * P32 + s));
      }
    }
  };
  // ring slot e of plane q, whose node (gx, gy) the caller found (`has`)
  auto fill = [&](int e, bool has, int gx, int gy, int q) {
    if (e >= NE) return;
    const int mm = plane_of(q);
    const bool ok = has && mm >= 0;
    R fv[FQ];
    fill_load(ok, mm, gx, gy, fv);
    fill_store(e, ok, mm, gx, gy, fv, q);
  };

  // Ring slot of plane q: (q - m0 + 1) mod 4.  The collision of plane m
  // (between barriers A(m) and A(m + 1)) reads the slots of m - 1, m and
  // m + 1.  In the same interval the fill warps write plane m + 2, and the
  // in-collision fill (memory phase of m + 1) writes plane m + 2 as well:
  // its slot (that of plane m - 2) was last read by the collision of plane
  // m - 1, which every warp finished before A(m).
  // With an even nx and no walls across x (and fill_pairs), each fill thread
  // takes a pair of x-neighbouring nodes (x even, x + 1) of one ring row and
  // loads each of their populations with one load of two elements (and U as
  // one 8-byte pair), half the loads and held registers of one slot per
  // load.  Pair px of row ey holds ring slots 2 px - 1 and 2 px (those in
  // the row).
  constexpr bool PAIRFILL = fill_pairs<S, XN>() && sizeof(S) <= 4;
  constexpr int PX = (EX + 2) / 2;
  constexpr int NPR = Sh::EY * PX;
  if constexpr (FW && PAIRFILL) {
    static_assert((EX & 1) == 0, "ring rows hold whole pairs");
    using PT = typename std::conditional<sizeof(S) == 2, uint32_t, float2>::type;
    if (filler && (nx & 1) == 0 && !wall_x && NPR <= NFW * 32) {
      const int pp = tid - NCW * 32;
      const int ey = pp / PX, px = pp - ey * PX;
      const bool pact = pp < NPR;
      int gx0 = x0 + 2 * px - 2;                  // even
      gx0 = ((gx0 % nx) + nx) % nx;               // periodic in x (nx even: stays even)
      int gy = (D == 3) ? y0 + ey - 1 : 0;
      bool has = pact;
      if (D == 3 && (gy < 0 || gy >= ny)) {
        if (wall_y) has = false;
        gy = ((gy % ny) + ny) % ny;
      }
      const int ea = ey * EX + 2 * px - 1;        // slot of node gx0 (px > 0)
      const bool sa = pact && px > 0, sb = pact && 2 * px < EX;
      PT pv[Q];
      float2 pu[V2 ? D : 1];
      auto pload = [&](int mm) {
        if (has && mm >= 0) {
          const uint32_t s0 = (D == 3) ? ((uint32_t)mm * (uint32_t)ny + (uint32_t)gy) * (uint32_t)nx + (uint32_t)gx0
                                       : (uint32_t)mm * (uint32_t)nx + (uint32_t)gx0;
          const PT* fw = reinterpret_cast<const PT*>(b.f_in);
#pragma unroll
          for (int i = 0; i < Q; ++i) pv[i] = __ldg(fw + (((uint32_t)i * P32 + s0) >> 1));
          if constexpr (V2) {
            const float* U = f_ext<L>(b.f_in, P);
#pragma unroll
            for (int a = 0; a < D; ++a)
              pu[a] = __ldg(reinterpret_cast<const float2*>(U + ((uint32_t)a * P32 + s0)));
          }
        }
      };
      auto pstore = [&](int mm, int q) {
        const bool ok = has && mm >= 0;
#pragma unroll
        for (int n = 0; n < 2; ++n) {
          if (n == 0 ? !sa : !sb) continue;
          if constexpr (sizeof(S) == 2 && V2) {
            unsigned short hb[Q];
            R Ub[D];
#pragma unroll
            for (int i = 0; i < Q; ++i) hb[i] = (unsigned short)(n ? pv[i] >> 16 : pv[i] & 0xffffu);
#pragma unroll
            for (int a = 0; a < D; ++a) Ub[a] = n ? pu[a].y : pu[a].x;
            fill_store_bits(ea + n, ok, mm, gx0 + n, gy, hb, Ub, q);
            continue;
          }
          R fv[FQ];
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            if constexpr (sizeof(S) == 2)
              fv[i] = ok ? Store<S>::cvtb((unsigned short)(n ? pv[i] >> 16 : pv[i] & 0xffffu)) : R(0);
            else
              fv[i] = ok ? (n ? pv[i].y : pv[i].x) : R(0);
          }
          if constexpr (V2) {
#pragma unroll
            for (int a = 0; a < D; ++a) fv[Q + a] = ok ? (n ? pu[a].y : pu[a].x) : R(0);
          }
          fill_store(ea + n, ok, mm, gx0 + n, gy, fv, q);
        }
      };
      for (int q = m0 - 1; q <= m0 + 1; ++q) {
        const int mm = plane_of(q);
        pload(mm);
        pstore(mm, q);
      }
      int mq = plane_of(m0 + 2);
      if (m0 + 2 <= m1) pload(mq);
      __syncthreads();
      for (int m = m0; m < m1; ++m) {
        __syncthreads();               // A: collision loads of plane m done
        if constexpr (CL) __syncthreads();  // C: learned closure done
        if (m + 2 <= m1) {             // overlaps the collision of plane m
          pstore(mq, m + 2);
          mq = plane_of(m + 3);
          if (m + 3 <= m1) pload(mq);
        }
        if constexpr (NBUF == 1) __syncthreads();  // B
      }
      if constexpr (NBUF == 2) __syncthreads();  // tile done (shared memory reuse)
      return;
    }
  }
  if (FW && filler) {
    // ---------------- fill warps ---------------------------------------------
    // Each thread fills the ring slots e0 + t * 32 NFW, t < SPF; their node
    // coordinates are fixed for the whole tile.  The populations of the next
    // plane to fill are loaded one plane ahead (held in registers across the
    // barrier), so a plane's fill costs the velocity arithmetic only and the
    // DRAM latency hides behind the collision of the plane before.
    const int e0 = tid - NCW * 32;
    int sgx[SPF ? SPF : 1], sgy[SPF ? SPF : 1];
    bool shas[SPF ? SPF : 1];
#pragma unroll
    for (int t = 0; t < SPF; ++t) {
      sgx[t] = sgy[t] = 0;
      shas[t] = slot_node(e0 + t * NFW * 32, sgx[t], sgy[t]);
    }
#pragma unroll
    for (int t = 0; t < SPF; ++t) {
      const int e = e0 + t * NFW * 32;
      fill(e, shas[t], sgx[t], sgy[t], m0 - 1);
      fill(e, shas[t], sgx[t], sgy[t], m0);
      fill(e, shas[t], sgx[t], sgy[t], m0 + 1);
    }
    R fv[SPF ? SPF : 1][FQ];
    int mq = plane_of(m0 + 2);
    if (m0 + 2 <= m1) {
#pragma unroll
      for (int t = 0; t < SPF; ++t) fill_load(shas[t] && mq >= 0, mq, sgx[t], sgy[t], fv[t]);
    }
    __syncthreads();
    for (int m = m0; m < m1; ++m) {
      __syncthreads();               // A: collision loads of plane m done
      if constexpr (CL) __syncthreads();  // C: learned closure done
      if (m + 2 <= m1) {             // overlaps the collision of plane m
#pragma unroll
        for (int t = 0; t < SPF; ++t) {
          const int e = e0 + t * NFW * 32;
          if (e < NE) fill_store(e, shas[t] && mq >= 0, mq, sgx[t], sgy[t], fv[t], m + 2);
        }
        mq = plane_of(m + 3);
        if (m + 3 <= m1) {
#pragma unroll
          for (int t = 0; t < SPF; ++t) fill_load(shas[t] && mq >= 0, mq, sgx[t], sgy[t], fv[t]);
        }
      }
      if constexpr (NBUF == 1) __syncthreads();  // B
    }
    if constexpr (NBUF == 2) __syncthreads();  // tile done (shared memory reuse)
    return;
  }
  if (!FW) {
    int gx = 0, gy = 0;
    const bool has = slot_node(tid, gx, gy);
    fill(tid, has, gx, gy, m0 - 1);
    fill(tid, has, gx, gy, m0);
  }

  // ---------------- collision warps ------------------------------------------
  // Node n < XN of this thread: x + 32 n, sAd / sPf row node + 32 n, ring
  // slot e_own + 32 n, column 32 n + lane of the warp's stage buffer.
  const int lane = tid & 31;
  const int grp = warp / C;
  const int k = warp - grp * C;         // stress component of this thread
  const int gxi = grp % GX, gyi = grp / GX;
  const int tx = gxi * 32 * XN + lane;  // node of the tile
  const int ty = gyi;
  const int node = grp * 32 * XN + lane;
  const int x = x0 + tx;
  const int y = (D == 3) ? y0 + ty : 0;
  const bool yin = D == 2 || y < ny;
  const bool active = (x < nx) && yin;  // node 0 (nodes n > 0 only if node 0)
  auto active_n = [&](int n) { return x + 32 * n < nx && yin; };
  const int e_own = (D == 3) ? (ty + 1) * EX + tx + 1 : tx + 1;
  // this thread's component arrays; offsets within them are 32-bit
  // (Q * pitch < 2^32 is checked at creation)
  const S* __restrict__ hin_k = b.h_in + (long long)k * Q * P;
  S* __restrict__ hout_k = b.h_out + (long long)k * Q * P;
  // periodic neighbour offsets along y (constant over the march)
  const int oy_p = (D == 3) ? ((y == ny - 1) ? -(ny - 1) * nx : nx) : 0;
  const int oy_m = (D == 3) ? ((y == 0) ? (ny - 1) * nx : -nx) : 0;
  const bool pf = PF && (!PAIR || (nx & 1) == 0);
  const unsigned amask = __ballot_sync(0xffffffffu, active);  // all 32 lanes are here
  // Whole rows: when all 32 nodes of a warp's row are in the grid and the row
  // starts on a 16-byte boundary (nx a multiple of 16 bytes' worth of
  // elements; pitch and array bases are), the warp copies it in 16-byte
  // chunks, spread over the lanes, instead of one element per lane.
  constexpr int EPC = 16 / (int)sizeof(S);     // elements per chunk
  constexpr bool WIDE = D == 3 || sizeof(S) == 2;
  auto wide_n = [&](int n) {
    return PF && WIDE && yin && x0 + gxi * 32 * XN + 32 * n + 31 < nx && (nx % EPC) == 0;
  };
  // Bulk tensor copies: lane 0 copies the warp's whole row of BX nodes of
  // every staged array with one tensor copy per array group (the copy
  // engine reads past nx into the next row, and fills with zeros past the
  // end of the arrays); the row's first node must lie on a 16-byte
  // boundary, which nx % EPC == 0 and the 32-node warp rows give.
  constexpr int BX = 32 * XN;
  constexpr int NJ = (Q - C) / C + 1;   // flow rows k + j C in range for every k
  static_assert(Split<L>::nf(0) <= NJ + 1, "flow rows: NJ, or NJ + 1 for component 0");
  const bool tma = PF && tm != nullptr && tm->on && pf && (nx % EPC) == 0 &&
                   ((x0 + gxi * 32 * XN) % EPC) == 0;
  if constexpr (PF) {
    if (tma) {
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NST; ++q) mbar_init(&smp->bar[q][warp], 1);
        mbar_init_fence();
      }
      __syncwarp();
    }
  }
  // Issue the copies of plane q's populations of every node of this thread
  // into stage buffer st.  Every call by a thread that stages commits exactly
  // one group (empty past the end of the chunk), so a wait for all but the
  // newest NST - 2 groups completes plane m's copies.
  auto prefetch = [&](int q, int st) {
    if constexpr (PF) {
      if (!pf || !active) return;
      auto& W = stage[st][warp];
      if (tma) {
        if (lane == 0 && q < m1) {
          const int s0 = (D == 3) ? (q * ny + y) * nx + x0 + gxi * 32 * XN
                                  : q * nx + x0 + gxi * 32 * XN;
          constexpr int ES = (int)sizeof(S);
          const int nfr = Split<L>::nf(k) > NJ ? NJ + 1 : NJ;
          const unsigned bytes = (unsigned)((Q + nfr) * BX * ES + BX * 4 + (V2 ? (1 + D) * BX * 4 : 0));
          uint64_t* bar = &smp->bar[st][warp];
          fence_proxy_async();   // the warp's reads of this buffer (ordered by __syncwarp) first
          mbar_arrive_expect_tx(bar, bytes);
          tma_load_2d(&W.h[0][0], &tm->h, s0, k * Q, bar);
          if (nfr > NJ) tma_load_2d(&W.f[0][0], &tm->f4, s0, 0, bar);
          else tma_load_3d(&W.f[0][0], &tm->f3, s0, k, 0, bar);
          tma_load_2d(&W.chi[0], &tm->x, s0, k, bar);
          if constexpr (V2) {
            tma_load_2d(&W.ext[0][0], &tm->e0, s0, k, bar);
            tma_load_2d(&W.ext[1][0], &tm->u, s0, 0, bar);
          }
        }
        return;
      }
      if (q < m1) {
#pragma unroll
        for (int n = 0; n < XN; ++n) {
          if (!active_n(n)) continue;
          const long long sq = (D == 3) ? ((long long)q * ny + y) * nx + x + 32 * n
                                        : (long long)q * nx + x + 32 * n;
          const uint32_t sq32 = (uint32_t)sq;
          const int c = 32 * n + lane;          // this lane's column
          if (wide_n(n)) {
            constexpr int CPR = 32 / EPC;          // chunks per row of 32 nodes
            constexpr int NCP = NPP * CPR;         // population chunks
            constexpr int NCX = NCP + 32 * 4 / 16; // and chi (4-byte) chunks
            constexpr int NCH = NCX + (V2 ? 8 * (1 + D) : 0);  // and h0, U (16-bit forms)
            const uint32_t s0 = sq32 - (uint32_t)lane;  // node of lane 0
            const int wb = 32 * n;                 // the row's stage columns
#pragma unroll
            for (int jj = 0; jj < (NCH + 31) / 32; ++jj) {
              const int cc = lane + 32 * jj;
              if (cc < NCP) {
                const int v = cc / CPR, sub = cc % CPR;
                const int i = v < Q ? v : k + (v - Q) * C;
                const S* src = (v < Q ? hin_k : b.f_in) + ((uint32_t)i * P32 + s0 + (uint32_t)(sub * EPC));
                S* dst = (v < Q ? W.h[v < Q ? v : 0] : W.f[v < Q ? 0 : v - Q]) + wb + sub * EPC;
                // (16-bit forms: the rest stress population is in FP32)
                if (i < Q && !(V2 && v == 0)) cp_async<16>(dst, src);
              } else if (cc < NCX) {
                const int sub = cc - NCP;
                cp_async<16>(&W.chi[wb + sub * 4], b.chi + ((uint32_t)k * P32 + s0 + (uint32_t)(sub * 4)));
              } else if (V2 && cc < NCH) {
                const int arr = (cc - NCX) >> 3, sub = (cc - NCX) & 7;
                const float* src = arr == 0 ? h_ext<L>(b.h_in, P) + (uint32_t)k * P32
                                            : f_ext<L>(b.f_in, P) + (uint32_t)(arr - 1) * P32;
                if constexpr (V2)
                  cp_async<16>(&W.ext[arr][wb + sub * 4], src + s0 + (uint32_t)(sub * 4));
              }
            }
            continue;
          }
          if constexpr (PAIR) {
            // lanes 2j, 2j + 1 hold nodes sq, sq + 1 (x even, nx even)
            const int par = lane & 1;
            const int tb = c - par;
            const uint32_t sp = sq32 - (uint32_t)par;
#pragma unroll
            for (int jj = 0; jj < (NPP + 1) / 2; ++jj) {
              const int v = 2 * jj + par;
              const int i = v < Q ? v : k + (v - Q) * C;
              const S* src = (v < Q ? hin_k : b.f_in) + ((uint32_t)i * P32 + sp);
              if (v < NPP && i < Q && !(V2 && v == 0))
                cp_async<4>((v < Q ? W.h[v < Q ? v : 0] : W.f[v < Q ? 0 : v - Q]) + tb, src);
            }
            if constexpr (V2) {   // the FP32 values of this lane's own node
              cp_async<4>(&W.ext[0][c], h_ext<L>(b.h_in, P) + ((uint32_t)k * P32 + sq32));
#pragma unroll
              for (int a = 0; a < D; ++a)
                cp_async<4>(&W.ext[1 + a][c], f_ext<L>(b.f_in, P) + ((uint32_t)a * P32 + sq32));
            }
          } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) cp_async<4>(&W.h[i][c], hin_k + ((uint32_t)i * P32 + sq32));
#pragma unroll
            for (int j = 0; j < NFM; ++j) {
              const int i = k + j * C;
              if (i < Q) cp_async<4>(&W.f[j][c], b.f_in + ((uint32_t)i * P32 + sq32));
            }
          }
          static_assert(sizeof(X) == 4, "chi is staged in 4-byte copies");
          cp_async<4>(&W.chi[c], b.chi + ((uint32_t)k * P32 + sq32));
        }
      }
      cp_commit();
    }
  };
  // stage buffers of plane m and of the plane NST - 1 ahead
  int st = 0, st_ahead = NST - 1;
  prefetch(m0, 0);
  if constexpr (NST == 3) prefetch(m0 + 1, 1);
  __syncthreads();                      // ring prologue

  for (int m = m0; m < m1; ++m) {
    const int rm = slot(m - 1), rc = slot(m), rp = slot(m + 1);
    const long long s = (D == 3) ? ((long long)m * ny + y) * nx + x : (long long)m * nx + x;
    const uint32_t s32 = (uint32_t)s;   // node 0; node n is s32 + 32 n

    // ---- memory phase: this thread's populations of component k ---------------
    // (without fill warps, the first NE threads also load the populations of
    // their ring slot of plane m + 1)
    int fgx = 0, fgy = 0;
    const int mn = plane_of(m + 1);
    const bool fslot = !FW && tid < NE;
    const bool fok = fslot && slot_node(tid, fgx, fgy) && mn >= 0;
    R fn[FW ? 1 : FQ];
    if (!FW && fok) {
      const long long sn = (D == 3) ? ((long long)mn * ny + fgy) * nx + fgx
                                    : (long long)mn * nx + fgx;
#pragma unroll
      for (int i = 0; i < (FW ? 1 : Q); ++i) fn[i] = Store<S>::ld(b.f_in + i * P + sn);
      if constexpr (V2 && !FW) {
        const float* U = f_ext<L>(b.f_in, P);
#pragma unroll
        for (int a = 0; a < D; ++a) fn[Q + a] = __ldg(U + a * P + sn);
      }
    }
    // Staged storage types keep this plane's values in stage buffer st
    // until the collision has used them (read there again rather than held
    // in registers across the barrier); FP64 holds them in registers.
    R hv[PF ? 1 : Q], fo[PF ? 1 : NFM];
    R old = R(0);
    if (active) {
      if constexpr (PF) {
        if (pf) {
          // this plane's copies (issued NST - 1 planes ago); then start the
          // next.  Whole-row chunks and a pair's copies were issued by other
          // lanes too: the active lanes synchronise after the wait so that
          // each sees the others' (both lanes of a pair are active or
          // neither is; whole rows imply all 32 lanes).  The same
          // synchronisation tells them that every lane has finished the
          // collision of plane m - 1, whose buffer (NST = 2) the next
          // copies overwrite.
          if (tma) {
            mbar_wait(&smp->bar[st][warp], (unsigned)(((m - m0) / NST) & 1), ph.err);
            __syncwarp(amask);
          } else {
            if constexpr (NST == 3) cp_wait_group<1>();
            else cp_wait_all();
            if (PAIR || WIDE) __syncwarp(amask);
          }
          prefetch(m + NST - 1, st_ahead);
        } else {
          // no copies for this kernel: the nodes' own values into their own
          // stage columns
          auto& W = stage[st][warp];
#pragma unroll
          for (int n = 0; n < XN; ++n) {
            if (!active_n(n)) continue;
            const int c = 32 * n + lane;
            const uint32_t sn32 = s32 + 32u * n;
#pragma unroll
            for (int i = V2 ? 1 : 0; i < Q; ++i) W.h[i][c] = hin_k[(uint32_t)i * P32 + sn32];
#pragma unroll
            for (int j = 0; j < NFM; ++j) {
              const int i = k + j * C;
              if (i < Q) W.f[j][c] = b.f_in[(uint32_t)i * P32 + sn32];
            }
            W.chi[c] = b.chi[(uint32_t)k * P32 + sn32];
            if constexpr (V2) {
              W.ext[0][c] = h_ext<L>(b.h_in, P)[(uint32_t)k * P32 + sn32];
#pragma unroll
              for (int a = 0; a < D; ++a)
                W.ext[1 + a][c] = f_ext<L>(b.f_in, P)[(uint32_t)a * P32 + sn32];
            }
          }
        }
        auto& W = stage[st][warp];
#pragma unroll
        for (int n = 0; n < XN; ++n) {
          if (!active_n(n)) continue;
          const int c = 32 * n + lane;
          R a = R(0), psum = R(0);
          if constexpr (V2) a = W.ext[0][c];
          else a = Store<S>::cvt(W.h[0][c]);
#pragma unroll
          for (int i = 1; i < Q; ++i) a = Store<S>::acc(a, W.h[i][c]);
#pragma unroll
          for (int j = 0; j < NFM; ++j) {
            const int i = k + j * C;
            if (i != 0 && i < Q) psum = Store<S>::acc(psum, W.f[j][c]);
          }
          // (16-bit forms: the sum of the scaled deviations s_i, i != 0;
          // the collision adds the sum of e_i(U), i != 0, = 1.5 w_0 |U|^2)
          if constexpr (V2) psum *= R(1.0f / Store<S>::KF);
          sAd[m & (NBUF - 1)][node + 32 * n][k] = a;
          sPf[m & (NBUF - 1)][node + 32 * n][k] = psum;
        }
      } else {
        R a = R(0), psum = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) hv[i] = Store<S>::ld(hin_k + ((uint32_t)i * P32 + s32));
#pragma unroll
        for (int j = 0; j < NFM; ++j) {
          const int i = k + j * C;
          fo[j] = i < Q ? Store<S>::ld(b.f_in + ((uint32_t)i * P32 + s32)) : R(0);
        }
        old = R(b.chi[(uint32_t)k * P32 + s32]);
#pragma unroll
        for (int i = 0; i < Q; ++i) a += hv[i];
#pragma unroll
        for (int j = 0; j < NFM; ++j) {
          const int i = k + j * C;
          if (i != 0 && i < Q) psum += fo[j];
        }
        sAd[m & (NBUF - 1)][node][k] = a;
        sPf[m & (NBUF - 1)][node][k] = psum;
      }
    }
    if constexpr (!FW) {
      if (fslot) fill_store(tid, fok, mn, fgx, fgy, fn, m + 1);
    }
    __syncthreads();                    // A

    // ---- learned closure: two warps per group evaluate the network, each for
    // the 16 nodes of one m16 tile (lanes 16 k .. 16 k + 15 of warp k) -------
    if constexpr (CL) {
      if (k < 2) {
        constexpr int IN = MlpDims<D>::IN;
        const bool mine = (lane >> 4) == k;   // this lane's node is in warp k's tile
        float xin[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) xin[q] = 0.f;
        R gr[D][D], Ad[C], A[C];
        if (active && mine) {
#pragma unroll
          for (int bq = 0; bq < D; ++bq) {
            const R uo = ring[rc][e_own].v[bq];
            {
              const R up = ring[rc][e_own + 1].v[bq], um = ring[rc][e_own - 1].v[bq];
              R d = R(0.5) * (up - um);
              if (wall_x && x == 0) d = uo + up * R(1.0 / 3.0);
              if (wall_x && x == nx - 1) d = -(uo + um * R(1.0 / 3.0));
              gr[0][bq] = d;
            }
            if (D == 3) {
              const R up = ring[rc][e_own + EX].v[bq], um = ring[rc][e_own - EX].v[bq];
              R d = R(0.5) * (up - um);
              if (wall_y && y == 0) d = uo + up * R(1.0 / 3.0);
              if (wall_y && y == ny - 1) d = -(uo + um * R(1.0 / 3.0));
              gr[1][bq] = d;
            }
            {
              const R up = ring[slot(m + 1)][e_own].v[bq], um = ring[slot(m - 1)][e_own].v[bq];
              R d = R(0.5) * (up - um);
              if (wall_m && m == 0) d = uo + up * R(1.0 / 3.0);
              if (wall_m && m == nm - 1) d = -(uo + um * R(1.0 / 3.0));
              gr[D - 1][bq] = d;
            }
          }
#pragma unroll
          for (int q = 0; q < C; ++q) {
            Ad[q] = sAd[m & (NBUF - 1)][node][q];
            A[q] = Ad[q] + (diag<L>(q) ? R(1) : R(0));
          }
          int q = 0;
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int bq = 0; bq < D; ++bq) xin[q++] = float(ph.lam * gr[a][bq]);
#pragma unroll
          for (int c = 0; c < C; ++c) xin[q++] = float(Ad[c]);
          if (D == 2) xin[q++] = float(ph.inv_lam);
          (void)IN;
        }
        if (mine) {
#pragma unroll
          for (int q = 0; q < 16; q += 2)
            *reinterpret_cast<uint32_t*>(&cls.X[grp][lane][q]) = pack_f16x2(xin[q], xin[q + 1]);
        }
        __syncwarp();
        mlp_tile(cls.P, cls.X[grp], cls.Y[grp], k);
        __syncwarp();
        bool used = false;
        if (active && mine) {
          R chi_an[C];
          chi_tensor<L, R>(A, Ad, gr, ph, chi_an);
          float num = 0.f, den = 0.f;
          float chi_nn[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            chi_nn[c] = cls.Y[grp][lane][c] * float(ph.inv_lam);
            const float dd = chi_nn[c] - float(chi_an[c]);
            num += dd * dd;
            den += float(chi_an[c]) * float(chi_an[c]);
          }
          // per-node residual check: fall back to the analytic source
          used = num <= ph.cl_tol2 * den;
#pragma unroll
          for (int c = 0; c < C; ++c) cls.chi[c][node] = used ? chi_nn[c] : float(chi_an[c]);
        }
        const unsigned act = __ballot_sync(0xffffffffu, active && mine);
        const unsigned use = __ballot_sync(0xffffffffu, used);
        if (lane == 0 && ph.cl_count && act) {
          atomicAdd(ph.cl_count, (unsigned long long)__popc(use));
          atomicAdd(ph.cl_count + 1, (unsigned long long)__popc(act & ~use));
        }
      }
      __syncthreads();                  // C
    }

    // ---- collision phase ------------------------------------------------------
#pragma unroll 1
    for (int n = 0; n < XN; ++n) {
      if (!active_n(n)) break;
      const int xn = x + 32 * n;
      const int nd = node + 32 * n;
      const int eo = e_own + 32 * n;
      const int col = 32 * n + lane;      // column of the warp's stage buffer
      const uint32_t sn32 = s32 + 32u * n;
      R u[D];
      {
        const Vel<R, D> t = ring[rc][eo];
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = t.v[a];
      }
      R Ad[C];
      lds_row<R, C>(&sAd[m & (NBUF - 1)][nd][0], Ad);
      R sumf = R(0);
      {
        R pf[C];
        lds_row<R, C>(&sPf[m & (NBUF - 1)][nd][0], pf);
#pragma unroll
        for (int q = 0; q < C; ++q) sumf += pf[q];
      }
      // 16-bit forms: the node's stored velocity U (the reference of its
      // flow populations), and the sum of e_i(U) over i != 0
      R Us[V2 ? D : 1];
      R UU = R(0);
      if constexpr (V2) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          Us[a] = stage[st][warp].ext[1 + a][col];
          UU += Us[a] * Us[a];
        }
        sumf += R(1.5 * L::w(0)) * UU;
      }
      R F[3];
      body_force<L, R>(ph, xn, D == 3 ? y : m, F);
      if constexpr (ORIG) {  // the original scheme: + div tau_p of this node, no f^B
#pragma unroll
        for (int a = 0; a < D; ++a) F[a] += ph.fdiv[(uint32_t)a * P32 + sn32];
      }
      R uu = R(0), Fu = R(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        uu += u[a] * u[a];
        Fu += F[a] * u[a];
      }
      const R kB = ORIG ? R(0) : ph.eta_over_lam * ph.inv_tau_f;
      // pressure (Sec. 2.2, Appendix B)
      constexpr double w0 = L::w(0);
      const R fB0 = fB_dir<L, R>(0, Ad, kB);
      const R p = p_part<L, R>(sumf + R(-1.5 * w0) * uu +
                               ph.tau_f * (R(-3.0 * w0) * ph.kf * Fu) + ph.tau_f * fB0);

      // Work that depends on the stress component k is dispatched once on
      // k (warp-uniform), so that every population index and coefficient
      // in it is a compile-time constant.
      // stress source of this component (Sec. 2.3):
      // chi_ab = -P_ab / lambda + sum_r (A_ar d_r u_b + d_r u_a A_rb), with
      // P = A - I for Oldroyd-B (relax_part for the other models)
      R chi_k = R(0), Ad_k = R(0), A_k = R(0);
      on_component(k, [&](auto KC) {
        constexpr int q = decltype(KC)::value;
        if constexpr (q < C) {
          Ad_k = Ad[q];
          A_k = Ad[q] + (diag<L>(q) ? R(1) : R(0));
          if constexpr (CL) {
            chi_k = cls.chi[q][nd];
          } else {
            constexpr int a = L::ca(q), bb = L::cb(q);
            R v = -(ph.model ? relax_part<L, R>(q, Ad, ph.model, ph.mpar) : Ad[q]) * ph.inv_lam;
#pragma unroll
            for (int r = 0; r < D; ++r) {
              // d_r u_a and d_r u_b from the ring (central, or one-sided at walls)
              R dua, dub;
              {
                int e_p, e_m, r_p, r_m;
                bool lo, hi;
                if (r == 0) {
                  e_p = eo + 1; e_m = eo - 1; r_p = rc; r_m = rc;
                  lo = wall_x && xn == 0; hi = wall_x && xn == nx - 1;
                } else if (r == 1 && D == 3) {
                  e_p = eo + EX; e_m = eo - EX; r_p = rc; r_m = rc;
                  lo = wall_y && y == 0; hi = wall_y && y == ny - 1;
                } else {
                  e_p = eo; e_m = eo; r_p = rp; r_m = rm;
                  lo = wall_m && m == 0; hi = wall_m && m == nm - 1;
                }
                const Vel<R, D> vp = ring[r_p][e_p], vm = ring[r_m][e_m];
                const R pa = vp.v[a], ma = vm.v[a];
                const R pb = vp.v[bb], mb = vm.v[bb];
                dua = R(0.5) * (pa - ma);
                dub = R(0.5) * (pb - mb);
                if (lo) { dua = u[a] + pa * R(1.0 / 3.0); dub = u[bb] + pb * R(1.0 / 3.0); }
                if (hi) { dua = -(u[a] + ma * R(1.0 / 3.0)); dub = -(u[bb] + mb * R(1.0 / 3.0)); }
              }
              const R Aar = Ad[sym<L>(a, r)] + (a == r ? R(1) : R(0));
              const R Arb = Ad[sym<L>(r, bb)] + (r == bb ? R(1) : R(0));
              v += Aar * dub + dua * Arb;
            }
            chi_k = v;
          }
        }
      });
      R oldn = old;
      if constexpr (PF) oldn = R(stage[st][warp].chi[col]);
      if (ph.first) oldn = chi_k;
      b.chi[(uint32_t)k * P32 + sn32] = X(chi_k);
      const R src = R(1.5) * chi_k - R(0.5) * oldn;
      uint32_t rng = Store<S>::sr
                         ? hash32((sn32 * 8u + (uint32_t)k) * 0x9e3779b9u ^ hash32(ph.step))
                         : 0u;

      // neighbour offsets along x (this node) and the march axis (periodic wrap)
      const int ox_p = (xn == nx - 1) ? -(nx - 1) : 1;
      const int ox_m = (xn == 0) ? (nx - 1) : -1;
      const uint32_t wxp = (xn == nx - 1) ? (uint32_t)(-nx) : 0u;  // wrap corrections
      const uint32_t wxm = (xn == 0) ? (uint32_t)nx : 0u;
      const int strm = (D == 3) ? nx * ny : nx;
      const int om_p = (m == nm - 1) ? -(nm - 1) * strm : strm;
      const int om_m = (m == 0) ? (nm - 1) * strm : -strm;
      const int opos[3] = {ox_p, D == 3 ? oy_p : om_p, om_p};
      const int oneg[3] = {ox_m, D == 3 ? oy_m : om_m, om_m};
      const int posv[3] = {xn, D == 3 ? y : m, m};
      const int extv[3] = {nx, D == 3 ? ny : nm, nm};
      // destination of direction i (32-bit offset within a population
      // array): the neighbour, or the own node through a halfway-bounce-back
      // wall (direction reversed)
      auto dest = [&](int i, int& j) -> uint32_t {
        int d = (int)sn32;
        bool bb = false;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const int c = cc<L>(i, a);
          if (c == 1) {
            d += opos[a];
            if (WALLS) bb |= ((g.walls >> a) & 1) && posv[a] == extv[a] - 1;
          } else if (c == -1) {
            d += oneg[a];
            if (WALLS) bb |= ((g.walls >> a) & 1) && posv[a] == 0;
          }
        }
        if (WALLS && bb) {
          j = L::opp(i);
          return sn32;
        }
        j = i;
        return (uint32_t)d;
      };
      // A warp whose row and plane are neither the first nor the last (so
      // that no population crosses a periodic wrap or a wall in y or along
      // the march axis) finds the destination of direction i at the fixed
      // distance i * pitch + c_x + c_y nx (+ c_z nx ny) from its node, plus
      // nx or -nx for the lanes at the two ends of a periodic row; with walls
      // on x the row ends bounce back, so those grids take the general rule.
      const bool fast = (!WALLS || !(g.walls & 1)) && (D == 2 || (y > 0 && y < ny - 1)) &&
                        m > 0 && m < nm - 1;

      // h_k: h* = (1 - 1/tau_h) h + w_i [alpha + c_i.u beta] with
      // alpha = (A-I)_k / tau_h + src and beta = 3 (A_k / tau_h + kh src)
      const R om = ph.inv_tau_h;
      const R alpha = om * Ad_k + src;
      const R beta = R(3) * (om * A_k + ph.kh * src);
      const R keep = R(1) - om;
      if constexpr (V2) {
        // this node's velocity: the reference of the flow populations it
        // receives for the next step (component threads k < D write one each)
        if (k < D) {
          const R uk = k == 0 ? u[0] : (k == 1 ? u[1] : u[D - 1]);
          f_ext<L>(b.f_out, P)[(uint32_t)k * P32 + sn32] = float(uk);
        }
      }
      // velocity of the node that receives population i: the ring holds the
      // tile's neighbours (periodic images included); through a wall the
      // population comes back to this node
      // (and its |u|^2: the 3D ring record carries it in its fourth slot)
      auto dest_u = [&](int i, bool bounced, R (&ud)[D]) -> R {
        const int cm = D == 3 ? L::cz(i) : L::cy(i);
        const int rs = bounced ? rc : (cm == 1 ? rp : (cm == -1 ? rm : rc));
        const int es = bounced ? eo : eo + L::cx(i) + (D == 3 ? L::cy(i) * EX : 0);
        const Vel<R, D> t = ring[rs][es];
#pragma unroll
        for (int a = 0; a < D; ++a) ud[a] = t.v[a];
        if constexpr (D == 3) return t.v[3];
        else return ud[0] * ud[0] + ud[1] * ud[1];
      };
      auto emit = [&](auto FASTC) {
        constexpr bool FAST = decltype(FASTC)::value;
        // offset of the slot that receives population i; `bounced`: through
        // a wall, back to this node (the slot's direction is then opp(i))
        auto index = [&](int i, bool& bounced) -> uint32_t {
          if constexpr (FAST) {
            bounced = false;
            const int cx = L::cx(i);
            const uint32_t xw = cx == 1 ? wxp : (cx == -1 ? wxm : 0u);
            return sn32 + (uint32_t)i * P32 + (uint32_t)(cx + L::cy(i) * nx + L::cz(i) * strm) + xw;
          } else {
            int j;
            const uint32_t d = dest(i, j);
            bounced = j != i;
            return (uint32_t)j * P32 + d;
          }
        };
        // The rest population (i = 0, which stays at this node) keeps the
        // node's stored populations summing to the post-collision zeroth
        // moment (A - I)_k + src (sum_i w_i = 1, sum_i w_i c_i = 0):
        //  - FP32: it is that moment minus the other populations' sum, so
        //    neither the rounded weights (whose sum exceeds one by 7e-9 in
        //    2D, 1.5e-8 in 3D) nor the rounding of the collision moves A;
        //  - 16-bit forms: it takes the rounding residuals of the 16-bit
        //    stores, less the weights' excess times alpha.
        constexpr double kWx = weight_sum_excess<L, R>();
        R h0post = R(0), hres = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          R cu = R(0);
#pragma unroll
          for (int a = 0; a < D; ++a) {
            const int c = cc<L>(i, a);
            if (c == 1) cu += u[a];
            if (c == -1) cu -= u[a];
          }
          R hvi;
          if constexpr (PF) {
            if constexpr (V2) hvi = i == 0 ? R(stage[st][warp].ext[0][col]) : Store<S>::cvt(stage[st][warp].h[i][col]);
            else hvi = Store<S>::cvt(stage[st][warp].h[i][col]);
          } else {
            hvi = hv[i];
          }
          const R wa = R(L::w(i)) * alpha, wb = R(L::w(i)) * beta;
          R post = keep * hvi + (wa + cu * wb);
          if constexpr (V2) {
            if (i == 0) {
              h0post = post - R(kWx) * alpha;
            } else {
              bool bnc;
              const uint32_t o = index(i, bnc);
              hres -= Store<S>::st_d(hout_k + o, post, Store<S>::sr ? lcg_next(rng) : 0u);
            }
          } else if constexpr (RS) {
            if (i != 0) {
              hres += post;
              bool bnc;
              Store<S>::st(hout_k + index(i, bnc), post, 0u);
            }
          } else {
            bool bnc;
            Store<S>::st(hout_k + index(i, bnc), post, Store<S>::sr ? lcg_next(rng) : 0u);
          }
        }
        if constexpr (V2) h_ext<L>(b.h_out, P)[(uint32_t)k * P32 + sn32] = float(h0post + hres);
        if constexpr (RS) Store<S>::st(hout_k + sn32, (Ad_k + src) - hres, 0u);

        // f_i, i = k (mod C): f* = f - (f - f^eq)/tau_f + f^B + F_i (Sec. 2.2)
        on_component(k, [&](auto KC) {
          constexpr int kk = decltype(KC)::value;
          if constexpr (kk < C) {
#pragma unroll
            for (int jj = 0; jj < NFM; ++jj) {
              const int i = kk + jj * C;
              if (i >= Q) continue;
              R cu = R(0), cF = R(0);
#pragma unroll
              for (int a = 0; a < D; ++a) {
                const int c = cc<L>(i, a);
                if (c == 1) { cu += u[a]; cF += F[a]; }
                if (c == -1) { cu -= u[a]; cF -= F[a]; }
              }
              const R wi = R(L::w(i));
              const R lam_i = R(p_coef<L, R>(i));
              const R w3i = R(w3<L, R>(i));
              const R feq = lam_i * p + (w3i * cu + wi * (R(4.5) * cu * cu - R(1.5) * uu));
              const R Fi = ph.kf * (w3i * cF + wi * (R(9) * cF * cu - R(3) * Fu));
              const R fBi = fB_dir<L, R>(i, Ad, kB);
              R foi;
              if constexpr (PF && V2) {
                foi = Store<S>::dev_add(stage[st][warp].f[jj][col], feq_u<L, R>(i, Us, UU));
              } else {
                if constexpr (PF) foi = Store<S>::cvt(stage[st][warp].f[jj][col]);
                else foi = fo[jj];
                if constexpr (V2) foi = foi * R(1.0f / Store<S>::KF) + feq_u<L, R>(i, Us, UU);
              }
              const R post = foi - (foi - feq) * ph.inv_tau_f + fBi + Fi;
              bool bnc;
              const uint32_t o = index(i, bnc);
              if constexpr (V2) {
                // scaled deviation from e_j(u) of the receiving node
                R ud[D];
                const R uud = dest_u(i, bnc, ud);
                const R ej = feq_u<L, R>(bnc ? L::opp(i) : i, ud, uud);
                Store<S>::st(b.f_out + o, R(Store<S>::KF) * (post - ej),
                             Store<S>::sr ? lcg_next(rng) : 0u);
              } else {
                Store<S>::st(b.f_out + o, post, Store<S>::sr ? lcg_next(rng) : 0u);
              }
            }
          }
        });
      };
      if (fast) emit(std::true_type{});
      else emit(std::false_type{});
    }
    if constexpr (NBUF == 1) __syncthreads();  // B
    st = st + 1 == NST ? 0 : st + 1;
    st_ahead = st_ahead + 1 == NST ? 0 : st_ahead + 1;
  }
  if constexpr (NBUF == 2) __syncthreads();  // tile done (shared memory reuse)
}

template <class L, class S, int GX, int TY, int MINB, bool WALLS, bool FW, bool CL = false,
          int XN = 1, bool ORIG = false>
__global__ void __launch_bounds__(FusedShape<L, GX, TY, FW, XN, fill_warps_max<S, XN>()>::NT, MINB)
    k_step_fused(Grid g, Phys<RT<S>> ph, Bufs<S> b, int mchunk,
                 const __grid_constant__ StageMaps tm) {
  fused_tile<L, S, GX, TY, WALLS, FW, CL, XN, ORIG, MINB>(g, ph, b, mchunk, blockIdx.x, blockIdx.y,
                                                    blockIdx.z, &tm);
}

// ---------------------------------------------------------------------------
// Batched persistent step: many independent grids (instances) of one lattice
// in one launch.  The host lists the tiles of every instance (instance, x
// tile, march chunk); each resident block walks the list with a stride of
// the grid size, so no block waits on another and the assignment is fixed
// (deterministic).  Per-instance geometry, physics and array offsets come
// from `inst`; the double buffers of all instances live in two arenas and
// `parity` says which one holds the current state.  The step count is read
// from device memory so that a captured CUDA graph can replay steps.
// ---------------------------------------------------------------------------
template <class S>
struct BatchInst {
  Grid g;
  Phys<RT<S>> ph;          // first / step / Fv filled in per launch
  long long f_off, h_off, chi_off;  // element offsets into the arenas
  int cosine;              // F = F0 cos(omega t)
  double F0[3];
  double omega;
};

struct BatchTile {
  int inst;
  int bx;
  int bz;
};

template <class L, class S, int GX, int MINB>
__global__ void __launch_bounds__(FusedShape<L, GX, 1, false>::NT, MINB)
    k_step_batched(const BatchInst<S>* __restrict__ inst, const BatchTile* __restrict__ tiles,
                   int ntiles, S* fA, S* fB, S* hA, S* hB, typename Store<S>::X* chi,
                   int parity, int first, const long long* __restrict__ tstep, int mchunk) {
  using R = RT<S>;
  const long long t = *tstep;
  for (int q = blockIdx.x; q < ntiles; q += gridDim.x) {
    const BatchTile tl = tiles[q];
    const BatchInst<S>& I = inst[tl.inst];
    Phys<R> ph = I.ph;
    ph.first = first;
    ph.step = (uint32_t)t;
    if (I.cosine) {
      const double c = cos(I.omega * (double)t);
      ph.Fv[0] = R(I.F0[0] * c);
      ph.Fv[1] = R(I.F0[1] * c);
      ph.Fv[2] = R(I.F0[2] * c);
    }
    Bufs<S> b;
    b.f_in = (parity ? fB : fA) + I.f_off;
    b.f_out = (parity ? fA : fB) + I.f_off;
    b.h_in = (parity ? hB : hA) + I.h_off;
    b.h_out = (parity ? hA : hB) + I.h_off;
    b.chi = chi + I.chi_off;
    fused_tile<L, S, GX, 1, true, false>(I.g, ph, b, mchunk, tl.bx, 0, tl.bz);
  }
}

// t += 1 on the device (one thread), after a batched step
static __global__ void k_advance_step(long long* t) { *t += 1; }

// ---------------------------------------------------------------------------
// Original scheme (Sec. 1, Tables 1-2): the polymer stress of every node in
// a working array tau_p[C][pitch], then its divergence by finite
// differences: central (periodic wrap), and next to a wall the one-sided
// second-order difference (-3 t0 + 4 t1 - t2) / 2 through the two nodes
// inside (sign mirrored at the upper wall), since no stress is known at the
// wall.  Needs 3 nodes across a walled axis.
// ---------------------------------------------------------------------------
template <class L, class S>
__global__ void k_taup(Grid g, Phys<RT<S>> ph, const S* __restrict__ h,
                       RT<S>* __restrict__ taup, long long N) {
  using R = RT<S>;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
       s += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < L::C; ++k) {
      R a = R(0);  // (A - I)_k from the deviations h'
#pragma unroll
      for (int i = 0; i < L::Q; ++i) a += load_h<L, S>(h, g.pitch, s, k, i);
      taup[k * g.pitch + s] = ph.eta_over_lam * a;
    }
  }
}

// dv_b = sum_a d_a tau_ab at node (x, y, z) = s
template <class L, class R>
__device__ __forceinline__ void div_taup(const Grid& g, const R* __restrict__ tp, int x, int y,
                                         int z, long long s, R (&dv)[3]) {
  const int p[3] = {x, y, z};
  const int n[3] = {g.nx, g.ny, g.nz};
  const long long st[3] = {1, g.nx, (long long)g.nx * g.ny};
  dv[0] = dv[1] = dv[2] = R(0);
#pragma unroll
  for (int a = 0; a < L::D; ++a) {
    if (n[a] == 1) continue;
    const bool wall = (g.walls >> a) & 1;
    const bool edge = wall && (p[a] == 0 || p[a] == n[a] - 1);
    const long long e = p[a] == 0 ? st[a] : -st[a];
    const long long sp = p[a] + 1 < n[a] ? s + st[a] : s - (long long)(n[a] - 1) * st[a];
    const long long sm = p[a] > 0 ? s - st[a] : s + (long long)(n[a] - 1) * st[a];
#pragma unroll
    for (int b = 0; b < L::D; ++b) {
      const R* t = tp + (long long)sym<L>(a, b) * g.pitch;
      R d;
      if (edge) {
        d = R(0.5) * (R(-3) * t[s] + R(4) * t[s + e] - t[s + 2 * e]);
        if (p[a] != 0) d = -d;
      } else {
        d = R(0.5) * (t[sp] - t[sm]);
      }
      dv[b] += d;
    }
  }
}

// The original scheme ahead of the fused step: div tau_p of every node into
// fdiv[a * pitch + s] (read by the fused step as part of the body force).
template <class L, class S>
__global__ void k_fdiv(Grid g, const RT<S>* __restrict__ taup, RT<S>* __restrict__ fdiv,
                       long long N) {
  using R = RT<S>;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
       s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % g.nx);
    const int y = (int)((s / g.nx) % g.ny);
    const int z = (int)(s / ((long long)g.nx * g.ny));
    R dv[3];
    div_taup<L, R>(g, taup, x, y, z, s, dv);
#pragma unroll
    for (int a = 0; a < L::D; ++a) fdiv[a * g.pitch + s] = dv[a];
  }
}

// ---------------------------------------------------------------------------
// Split step: velocity field to a device buffer, then collide-and-push with
// the gradient read from that buffer.  One thread per site.  ORIG: the
// original scheme, the stress divergence added to the body force.
// ---------------------------------------------------------------------------
template <class L, class S, bool ORIG = false>
__global__ void k_velocity(Grid g, Phys<RT<S>> ph, const S* __restrict__ f,
                           RT<S>* __restrict__ ubuf, const RT<S>* __restrict__ taup,
                           long long N) {
  using R = RT<S>;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
       s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % g.nx);
    const int y = (int)((s / g.nx) % g.ny);
    R fv[L::Q];
    load_f<L, S>(f, g.pitch, s, fv);
    R F[3];
    body_force<L, R>(ph, x, y, F);
    if constexpr (ORIG) {
      R dv[3];
      div_taup<L, R>(g, taup, x, y, (int)(s / ((long long)g.nx * g.ny)), s, dv);
      F[0] += dv[0];
      F[1] += dv[1];
      F[2] += dv[2];
    }
    R u[L::D];
    velocity<L, R>(fv, F, u);
#pragma unroll
    for (int a = 0; a < L::D; ++a) ubuf[a * g.pitch + s] = u[a];
  }
}

template <class L, class S, bool HOLD_H, bool ORIG = false>
__global__ void k_collide_split(Grid g, Phys<RT<S>> ph, Bufs<S> b,
                                const RT<S>* __restrict__ ubuf, const RT<S>* __restrict__ taup,
                                long long N) {
  using R = RT<S>;
  constexpr int D = L::D;
  const long long P = g.pitch;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
       s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % g.nx);
    const int y = (int)((s / g.nx) % g.ny);
    const int z = (int)(s / ((long long)g.nx * g.ny));
    const int p[3] = {x, y, z};
    const int n[3] = {g.nx, g.ny, g.nz};
    const long long stride[3] = {1, g.nx, (long long)g.nx * g.ny};
    R u[D], gr[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = ubuf[a * P + s];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const bool wall = (g.walls >> a) & 1;
      const long long sp = p[a] + 1 < n[a] ? s + stride[a] : s - (long long)(n[a] - 1) * stride[a];
      const long long sm = p[a] > 0 ? s - stride[a] : s + (long long)(n[a] - 1) * stride[a];
#pragma unroll
      for (int bq = 0; bq < D; ++bq) {
        const R up = ubuf[bq * P + sp], um = ubuf[bq * P + sm];
        R d = R(0.5) * (up - um);
        if (wall && p[a] == 0) d = u[bq] + up * R(1.0 / 3.0);
        if (wall && p[a] == n[a] - 1) d = -(u[bq] + um * R(1.0 / 3.0));
        gr[a][bq] = d;
      }
    }
    R fv[L::Q];
    load_f<L, S>(b.f_in, P, s, fv);
    R F[3];
    body_force<L, R>(ph, x, y, F);
    if constexpr (ORIG) {
      R dv[3];
      div_taup<L, R>(g, taup, x, y, z, s, dv);
      F[0] += dv[0];
      F[1] += dv[1];
      F[2] += dv[2];
    }
    collide_site<L, S, HOLD_H, ORIG>(g, ph, b, s, x, y, z, u, gr, fv, F, ubuf);
  }
}

// ---------------------------------------------------------------------------
// Initial state: f = f^eq(p0, u0), h = w_i A0 (1 + c_i.u0 / c_s^2), chi = 0.
// u0 [N][D], p0 [N], A0 [N][C] in FP64 (each may be null: 0, 0, I).
// ---------------------------------------------------------------------------
template <class L, class S>
__global__ void k_init(Grid g, S* __restrict__ f, S* __restrict__ h,
                       typename Store<S>::X* __restrict__ chi,
                       const double* __restrict__ u0, const double* __restrict__ p0,
                       const double* __restrict__ A0, long long N) {
  using R = RT<S>;
  constexpr int D = L::D, Q = L::Q, C = L::C;
  const long long P = g.pitch;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
       s += (long long)gridDim.x * blockDim.x) {
    R u[D], A[C];
    R uu = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      u[a] = u0 ? R(u0[s * D + a]) : R(0);
      uu += u[a] * u[a];
    }
#pragma unroll
    for (int k = 0; k < C; ++k)
      A[k] = A0 ? R(A0[s * C + k]) : (L::ca(k) == L::cb(k) ? R(1) : R(0));
    const R p = p_part_of_p<L, R>(p0 ? R(p0[s]) : R(0));
    R hres[C];
#pragma unroll
    for (int k = 0; k < C; ++k) hres[k] = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      R cu = R(0);
#pragma unroll
      for (int a = 0; a < D; ++a) cu += R(cc<L>(i, a)) * u[a];
      const R wi = R(L::w(i));
      const R lam_i = R(p_coef<L, R>(i));
      if constexpr (Store<S>::V2) {
        // f^eq(p, u) - e_i(u) = lam_i p, scaled; U = u
        Store<S>::st(f + i * P + s, R(Store<S>::KF) * (lam_i * p), 0x80000000u);
      } else {
        Store<S>::st(f + i * P + s,
                     lam_i * p + (R(w3<L, R>(i)) * cu + wi * (R(4.5) * cu * cu - R(1.5) * uu)),
                     0x80000000u);
      }
#pragma unroll
      for (int k = 0; k < C; ++k) {
        const R v = wi * ((A[k] - (diag<L>(k) ? R(1) : R(0))) + A[k] * (R(3) * cu));
        if constexpr (Store<S>::V2) {
          if (i > 0) hres[k] += v - Store<S>::st_r(h + (long long)(k * Q + i) * P + s, v, 0x80000000u);
        } else {
          store_h<L, S>(h, P, s, k, i, v, 0x80000000u);
        }
      }
    }
    if constexpr (Store<S>::V2) {
      float* U = f_ext<L>(f, P);
      float* h0 = h_ext<L>(h, P);
#pragma unroll
      for (int a = 0; a < D; ++a) U[a * P + s] = float(u[a]);
#pragma unroll
      for (int k = 0; k < C; ++k) {
        R cu0 = R(0);
        const R v0 = R(L::w(0)) * ((A[k] - (diag<L>(k) ? R(1) : R(0))) + A[k] * (R(3) * cu0));
        h0[k * P + s] = float(v0 + hres[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < C; ++k) chi[k * P + s] = 0;
  }
}

// ---------------------------------------------------------------------------
// Macroscopic fields of the current state into a device FP64 buffer.
// which: 0 u [N][D], 1 p [N], 2 A [N][C], 3 tau_p [N][C].
// ---------------------------------------------------------------------------
template <class L, class S, bool ORIG = false>
__global__ void k_fields(Grid g, Phys<RT<S>> ph, const S* __restrict__ f,
                         const S* __restrict__ h, int which, double* __restrict__ out,
                         const RT<S>* __restrict__ taup, long long N) {
  using R = RT<S>;
  constexpr int D = L::D, Q = L::Q, C = L::C;
  const long long P = g.pitch;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
       s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % g.nx);
    const int y = (int)((s / g.nx) % g.ny);
    R fv[Q];
    load_f<L, S>(f, P, s, fv);
    R F[3];
    body_force<L, R>(ph, x, y, F);
    if constexpr (ORIG) {  // the original scheme: stress divergence in the force
      R dv[3];
      div_taup<L, R>(g, taup, x, y, (int)(s / ((long long)g.nx * g.ny)), s, dv);
      F[0] += dv[0];
      F[1] += dv[1];
      F[2] += dv[2];
    }
    R u[D];
    velocity<L, R>(fv, F, u);
    if (which == 0) {
#pragma unroll
      for (int a = 0; a < D; ++a) out[s * D + a] = double(u[a]);
      continue;
    }
    R A[C], tp[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
      R a = R(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) a += load_h<L, S>(h, P, s, k, i);
      A[k] = a + (diag<L>(k) ? R(1) : R(0));
      tp[k] = ph.eta_over_lam * a;
    }
    if (which == 1) {
      const R fB0 = ORIG ? R(0) : fB_dir<L, R>(0, tp, ph.inv_tau_f);
      out[s] = p_of_part<L, R>(pressure<L, R>(ph, fv, u, F, fB0));
    } else if (which == 2) {
#pragma unroll
      for (int k = 0; k < C; ++k) out[s * C + k] = double(A[k]);
    } else {
#pragma unroll
      for (int k = 0; k < C; ++k) out[s * C + k] = double(tp[k]);
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 diagnostics: per-block partial sums (fixed thread-to-site mapping and
// a fixed shuffle tree), then one block reduces the partials in index order.
// Deterministic for a given launch shape.
// part: [gridDim.x][8] = {mass, Px, Py, Pz, sum |u|^2/2, sum tr(tau_p)/2,
// non-finite count, max |u|}.
// ---------------------------------------------------------------------------
constexpr int kReduceThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

template <class L, class S, bool ORIG = false>
__global__ void __launch_bounds__(kReduceThreads)
    k_reduce_partial(Grid g, Phys<RT<S>> ph, const S* __restrict__ f,
                     const S* __restrict__ h, double* __restrict__ part, long long N,
                     const RT<S>* __restrict__ taup = nullptr) {
  using R = RT<S>;
  constexpr int D = L::D, Q = L::Q, C = L::C;
  const long long P = g.pitch;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
       s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % g.nx);
    const int y = (int)((s / g.nx) % g.ny);
    R fv[Q];
    load_f<L, S>(f, P, s, fv);
    bool bad = false;
    double m = 0.0, mom[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double v = double(fv[i]);
      bad |= !isfinite(v);
      m += v;
#pragma unroll
      for (int a = 0; a < D; ++a) mom[a] += double(cc<L>(i, a)) * v;
    }
    R F[3];
    body_force<L, R>(ph, x, y, F);
    if constexpr (ORIG) {  // the original scheme: stress divergence in the force
      R dv[3];
      div_taup<L, R>(g, taup, x, y, (int)(s / ((long long)g.nx * g.ny)), s, dv);
      F[0] += dv[0];
      F[1] += dv[1];
      F[2] += dv[2];
    }
    R u[D];
    velocity<L, R>(fv, F, u);
    double uu = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) uu += double(u[a]) * double(u[a]);
    double tr = 0.0;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      if (L::ca(k) != L::cb(k)) {
        // off-diagonal components only enter the finiteness check
#pragma unroll
        for (int i = 0; i < Q; ++i) bad |= !isfinite(double(load_h<L, S>(h, P, s, k, i)));
        continue;
      }
      double a = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) a += double(load_h<L, S>(h, P, s, k, i));
      bad |= !isfinite(a);
      tr += double(ph.eta_over_lam) * a;
    }
    bad |= !isfinite(uu);
    acc[0] += m;
    acc[1] += mom[0];
    acc[2] += mom[1];
    acc[3] += mom[2];
    acc[4] += 0.5 * uu;
    acc[5] += 0.5 * tr;
    acc[6] += bad ? 1.0 : 0.0;
    acc[7] = fmax(acc[7], isfinite(uu) ? sqrt(uu) : 0.0);
  }
  __shared__ double sm[kReduceThreads / 32][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double v = q == 7 ? warp_max(acc[q]) : warp_sum(acc[q]);
    if (lane == 0) sm[wid][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int q = threadIdx.x;
    double v = sm[0][q];
    for (int w = 1; w < kReduceThreads / 32; ++w) v = q == 7 ? fmax(v, sm[w][q]) : v + sm[w][q];
    part[blockIdx.x * 8 + q] = v;
  }
}

// One block of kReduceThreads threads reduces the partials in index order;
// out[8] as documented for fvlb_reduce in fvlb.h.  (static: each translation
// unit that launches it has its own copy.)
static __global__ void __launch_bounds__(kReduceThreads)
    k_reduce_final(const double* __restrict__ part, int nparts, long long nsites,
                   double* __restrict__ out) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double v = part[p * 8 + q];
      acc[q] = q == 7 ? fmax(acc[q], v) : acc[q] + v;
    }
  }
  __shared__ double sm[kReduceThreads / 32][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double v = q == 7 ? warp_max(acc[q]) : warp_sum(acc[q]);
    if (lane == 0) sm[wid][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int q = threadIdx.x;
    double v = sm[0][q];
    for (int w = 1; w < kReduceThreads / 32; ++w) v = q == 7 ? fmax(v, sm[w][q]) : v + sm[w][q];
    if (q == 4 || q == 5) v /= (double)nsites;
    out[q] = v;
  }
}

// ---------------------------------------------------------------------------
// Conformation check.  A = I + M must stay symmetric positive definite in
// every model; losing it is how a run at high Wi fails (the four-roll mill
// of Sec. 3.1 goes up to Wi = 5).  Per node the smallest eigenvalue of A:
// in 2D the closed form of a symmetric 2 x 2 matrix, in 3D the Jacobi
// eigenvalue method (plane rotations; accurate to rounding relative to |A|
// also for nearly repeated eigenvalues, where roots of the characteristic
// cubic lose half the digits).  Per block: number of
// nodes whose smallest eigenvalue is not > 0 (non-finite included), the
// smallest eigenvalue, the largest tr A.
// ---------------------------------------------------------------------------
template <class L>
__device__ __forceinline__ double min_eigenvalue(const double (&M)[L::C]) {
  constexpr int D = L::D;
  if constexpr (D == 2) {
    const double a = 1.0 + M[sym<L>(0, 0)], c = 1.0 + M[sym<L>(1, 1)], b = M[sym<L>(0, 1)];
    const double h = 0.5 * (a - c);
    return 0.5 * (a + c) - sqrt(h * h + b * b);
  } else {
    // cyclic Jacobi rotations: each zeroes one off-diagonal entry; six
    // sweeps of the three pairs take a 3 x 3 matrix to diagonal in double
    double a[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) a[r][c] = M[sym<L>(r, c)] + (r == c ? 1.0 : 0.0);
#pragma unroll 1
    for (int sweep = 0; sweep < 6; ++sweep) {
#pragma unroll
      for (int pr = 0; pr < 3; ++pr) {
        const int p = pr == 2 ? 1 : 0, q = pr == 0 ? 1 : 2, o = 3 - p - q;
        const double apq = a[p][q];
        if (apq == 0.0) continue;
        const double th = (a[q][q] - a[p][p]) / (2.0 * apq);
        const double t = copysign(1.0, th) / (fabs(th) + hypot(th, 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        a[p][p] -= t * apq;
        a[q][q] += t * apq;
        a[p][q] = a[q][p] = 0.0;
        const double aop = a[o][p], aoq = a[o][q];
        a[o][p] = a[p][o] = c * aop - sn * aoq;
        a[o][q] = a[q][o] = sn * aop + c * aoq;
      }
    }
    return fmin(a[0][0], fmin(a[1][1], a[2][2]));
  }
}

template <class L, class S>
__global__ void __launch_bounds__(kReduceThreads)
    k_conf_partial(Grid g, const S* __restrict__ h, double* __restrict__ part, long long N) {
  constexpr int Q = L::Q, C = L::C;
  const long long P = g.pitch;
  double cnt = 0.0, emin = INFINITY, trmax = -INFINITY;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
       s += (long long)gridDim.x * blockDim.x) {
    double M[C];
    double tr = 0.0;
    bool fin = true;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      double a = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) a += double(load_h<L, S>(h, P, s, k, i));
      M[k] = a;
      fin &= isfinite(a);
      if (L::ca(k) == L::cb(k)) tr += 1.0 + a;
    }
    if (!fin) {             // (fmin in the eigenvalue routine would drop a NaN)
      cnt += 1.0;
      continue;
    }
    const double e = min_eigenvalue<L>(M);
    cnt += (e > 0.0) ? 0.0 : 1.0;
    emin = fmin(emin, e);
    trmax = fmax(trmax, tr);
  }
  __shared__ double sm[kReduceThreads / 32][3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double v0 = warp_sum(cnt), v1 = -warp_max(-emin), v2 = warp_max(trmax);
  if (lane == 0) {
    sm[wid][0] = v0;
    sm[wid][1] = v1;
    sm[wid][2] = v2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double c = sm[0][0], mn = sm[0][1], mx = sm[0][2];
    for (int w = 1; w < kReduceThreads / 32; ++w) {
      c += sm[w][0];
      mn = fmin(mn, sm[w][1]);
      mx = fmax(mx, sm[w][2]);
    }
    part[blockIdx.x * 3 + 0] = c;
    part[blockIdx.x * 3 + 1] = mn;
    part[blockIdx.x * 3 + 2] = mx;
  }
}

// (static: each translation unit that launches it has its own copy.)
static __global__ void __launch_bounds__(kReduceThreads)
    k_conf_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  double c = 0.0, mn = INFINITY, mx = -INFINITY;
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
    c += part[p * 3 + 0];
    mn = fmin(mn, part[p * 3 + 1]);
    mx = fmax(mx, part[p * 3 + 2]);
  }
  __shared__ double sm[kReduceThreads / 32][3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double v0 = warp_sum(c), v1 = -warp_max(-mn), v2 = warp_max(mx);
  if (lane == 0) {
    sm[wid][0] = v0;
    sm[wid][1] = v1;
    sm[wid][2] = v2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kReduceThreads / 32; ++w) {
      sm[0][0] += sm[w][0];
      sm[0][1] = fmin(sm[0][1], sm[w][1]);
      sm[0][2] = fmax(sm[0][2], sm[w][2]);
    }
    out[0] = sm[0][0];
    out[1] = sm[0][1];
    out[2] = sm[0][2];
  }
}

// ---------------------------------------------------------------------------
// High-Wi repair of the conformation (fvlb_repair_conformation).  Per node,
// in FP64: A from the stress populations, its eigen-decomposition by cyclic
// Jacobi rotations with the rotations accumulated into the eigenvectors
// (ten sweeps), and where the smallest eigenvalue is below eps,
// A' = V max(Lambda, eps) V^T, applied as h'_{k,i} += w_i (A' - A)_k, which
// moves the zeroth moment of h only (sum_i w_i c_i = 0).  16-bit forms: the
// 16-bit populations are re-rounded and their rounding residual goes to the
// FP32 rest population, as in the step.  count[0] += nodes changed (a node
// with a non-finite A is counted and left as it is).
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void jacobi_eig(double (&a)[3][3], double (&v)[3][3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) v[r][c] = r == c ? 1.0 : 0.0;
#pragma unroll 1
  for (int sweep = 0; sweep < 10; ++sweep) {
#pragma unroll
    for (int pr = 0; pr < (D == 3 ? 3 : 1); ++pr) {
      const int p = pr == 2 ? 1 : 0, q = pr == 0 ? 1 : 2;
      const double apq = a[p][q];
      if (apq == 0.0) continue;
      const double th = (a[q][q] - a[p][p]) / (2.0 * apq);
      const double t = copysign(1.0, th) / (fabs(th) + hypot(th, 1.0));
      const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
      // a <- J^T a J and v <- v J for the rotation J in the (p, q) plane
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - sn * akq;
        a[k][q] = sn * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - sn * aqk;
        a[q][k] = sn * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - sn * vkq;
        v[k][q] = sn * vkp + c * vkq;
      }
    }
  }
}

template <class L, class S>
__global__ void __launch_bounds__(kReduceThreads)
    k_repair(Grid g, S* __restrict__ h, double eps, unsigned long long* __restrict__ count,
             long long N) {
  using R = RT<S>;
  constexpr int D = L::D, Q = L::Q, C = L::C;
  const long long P = g.pitch;
  unsigned long long mine = 0;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
       s += (long long)gridDim.x * blockDim.x) {
    double M[C];
    bool fin = true;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) acc += double(load_h<L, S>(h, P, s, k, i));
      M[k] = acc;
      fin &= isfinite(acc);
    }
    if (!fin) {
      ++mine;
      continue;
    }
    double a[3][3], v[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        a[r][c] = (r < D && c < D) ? M[sym<L>(r, c)] + (r == c ? 1.0 : 0.0) : 0.0;
    jacobi_eig<D>(a, v);
    double lmin = a[0][0];
#pragma unroll
    for (int k = 1; k < D; ++k) lmin = fmin(lmin, a[k][k]);
    if (!(lmin < eps)) continue;
    ++mine;
    double dA[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const int ra = L::ca(k), rb = L::cb(k);
      double An = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) An += v[ra][j] * fmax(a[j][j], eps) * v[rb][j];
      dA[k] = An - (M[k] + (ra == rb ? 1.0 : 0.0));
    }
#pragma unroll
    for (int k = 0; k < C; ++k) {
      R res = R(0);
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        S* q = h + (long long)(k * Q + i) * P + s;
        const R nv = R(double(Store<S>::cvt(*q)) + L::w(i) * dA[k]);
        if constexpr (Store<S>::V2) res += nv - Store<S>::st_r(q, nv, 0x80000000u);
        else Store<S>::st(q, nv, 0u);
      }
      if constexpr (Store<S>::V2) {
        float* h0 = h_ext<L>(h, P) + k * P + s;
        *h0 = float(double(*h0) + L::w(0) * dA[k] + double(res));
      } else {
        S* q = h + (long long)(k * Q) * P + s;
        Store<S>::st(q, R(double(Store<S>::cvt(*q)) + L::w(0) * dA[k]), 0u);
      }
    }
  }
  // block total, then one atomic per block (an integer sum: order-free)
  __shared__ unsigned long long sm[kReduceThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kReduceThreads / 32; ++w) t += sm[w];
    if (t) atomicAdd(count, t);
  }
}

}  // namespace fvlb
