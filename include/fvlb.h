/*
 * fvlb.h -- C ABI of the GB300 (sm_103a) library for the fluctuating lattice
 * Boltzmann method for Oldroyd-B fluids of Wang, Liu, Wang, Yu and Ji
 * (arXiv 2506.13072).
 *
 * One handle is one simulation on one GPU: a D2Q9 or D3Q19 grid of
 * nx * ny * nz sites carrying the flow populations f_i (Sec. 2.2, evolution
 * equation with the polymer-stress fluctuation term f^B and Guo forcing),
 * the conformation-tensor populations h_{ab,i} (Sec. 2.3) and the previous
 * step's stress source chi (for the 0.5 dt^2 d(chi_i)/dt term).  One call of
 * fvlb_step advances every site by one fused collide-and-stream update.
 *
 * Conventions shared by every entry point
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3, rho_0 = 1.
 *   - Sites are ordered x fastest: s = (z * ny + y) * nx + x (nz = 1 in 2D).
 *   - Host field arrays are FP64, site-major, components last:
 *       velocity u        [N][D]
 *       pressure p        [N]
 *       conformation A    [N][C]  symmetric components,
 *       polymer stress    [N][C]  C = 3 in 2D (xx, xy, yy),
 *                                 C = 6 in 3D (xx, yy, zz, xy, xz, yz).
 *   - Ownership: the caller owns every host buffer it passes; the library
 *     owns all device memory of a handle and never returns device pointers.
 *   - Errors: every entry point returns an int status (FVLB_OK = 0 or a
 *     negative FVLB_E* code); no C++ exception crosses the ABI.  A failed
 *     call leaves the simulation state unchanged unless stated otherwise.
 *     fvlb_last_error gives a one-line description.
 *   - Threading: a handle is not thread-safe; distinct handles are
 *     independent.  All GPU work of a handle runs on its stream, in order.
 */
#ifndef FVLB_H
#define FVLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fvlb_s *fvlb_t; /* opaque simulation handle */
typedef struct fvlb_mlp_s *fvlb_mlp_t; /* learned stress closure (see below) */

/* Lattices: D2Q9 (Sec. 2.2 c_i matrix and weights), D3Q19 (Appendix A c_i
 * matrix; weights 1/3, 1/18, 1/36). */
enum { FVLB_D2Q9 = 9, FVLB_D3Q19 = 19 };

/* Status codes. */
enum {
  FVLB_OK = 0,
  FVLB_EINVAL = -1,    /* invalid argument; nothing was changed */
  FVLB_ENOMEM = -2,    /* a device allocation failed */
  FVLB_ECUDA = -3,     /* a CUDA call failed */
  FVLB_EUNSTABLE = -4, /* the diagnostics found a non-finite value */
  FVLB_ETIMEOUT = -5,  /* a bounded device wait ran out: a step kernel's staged
                        * copies did not arrive within about 2 s; the state is
                        * invalid until fvlb_init_fields / fvlb_load_state.
                        * Reported by fvlb_fields, fvlb_reduce and
                        * fvlb_status(h, 1). */
  FVLB_ESTATE = -6     /* call not allowed in the handle's current state */
};

/* Body force F(x, t) entering u = sum c_i f_i + F/2 and the Guo term F_i
 * (Sec. 2.2).  Positions are node indices, t is the step count.
 *   NONE       F = 0
 *   CONST      F = F0                                       (Sec. 3.2)
 *   FOUR_ROLL  F = F0[0] (sin kx cos ky, -cos kx sin ky, 0) (Sec. 3.1)
 *   COSINE     F = F0 cos(omega t)                          (Sec. 3.3) */
enum {
  FVLB_FORCE_NONE = 0,
  FVLB_FORCE_CONST = 1,
  FVLB_FORCE_FOUR_ROLL = 2,
  FVLB_FORCE_COSINE = 3
};

typedef struct {
  int kind;     /* FVLB_FORCE_* */
  double F0[3]; /* amplitude vector, lattice units */
  double k;     /* FOUR_ROLL wavenumber (2 pi / n for n periodic nodes) */
  double omega; /* COSINE angular frequency per step */
} fvlb_force;

/* Storage precision of the populations (set before the first state-using
 * call).  Every form stores f (whose rest equilibrium is 0) and
 * h_ab,i - w_i delta_ab (the deviation from the rest equilibrium A = I).
 * FP64 and FP32 compute in that precision.  The 16-bit forms compute in
 * FP32 and keep chi in FP32; FP16_DEV and BF16_DEV round to nearest when
 * storing, FP16_DEV_SR and BF16_DEV_SR round stochastically (unbiased, with
 * random bits from a counter-based hash of site and step, so runs are
 * reproducible).  So that rounding to 16 bits every step does not bias
 * slowly evolving flows, the 16-bit forms store
 *   f as KF (f_i - e_i(U)), the deviation from the velocity part of the
 *     equilibrium, e_i(U) = w_i (3 c_i.U + 4.5 (c_i.U)^2 - 1.5 U.U), at the
 *     velocity U of the receiving node in the step that wrote it, scaled
 *     by KF = 4096 (FP16) or 1 (BF16); U itself in FP32, U[D][pitch]
 *     right after f[Q][pitch] in the same buffer;
 *   the rest stress population h'_ab,0 in FP32, h0[C][pitch] right after
 *     h'[C][Q][pitch] (whose i = 0 slots are unused), where each store
 *     also adds the rounding residuals of the component's 16-bit
 *     populations, so that their sum carries no rounding bias.
 * Bytes per node update: 196 (D2Q9) and 628 (D3Q19), against 312 and 1112
 * for FP32. */
enum {
  FVLB_FP64 = 0,
  FVLB_FP32 = 1,
  FVLB_FP16_DEV = 2,
  FVLB_BF16_DEV = 3,
  FVLB_FP16_DEV_SR = 4,
  FVLB_BF16_DEV_SR = 5
};

/* Kernel variant: FUSED is one launch per step (the velocity gradient comes
 * from a shared-memory ring of velocity planes); SPLIT is two launches per
 * step (velocity field to a device buffer, then collide-and-stream). */
enum { FVLB_KERNEL_FUSED = 0, FVLB_KERNEL_SPLIT = 1 };

/* Scheme: PRESENT is the paper's method (the polymer stress enters the flow
 * through the fluctuation term f^B, Sec. 2.2); ORIGINAL is the conventional
 * scheme the paper compares it with (Sec. 1, Tables 1 and 2): no f^B, the
 * stress divergence added to the body force. */
enum { FVLB_SCHEME_PRESENT = 0, FVLB_SCHEME_ORIGINAL = 1 };

/* Constitutive model of the polymer (fvlb_set_model).  The paper solves
 * Oldroyd-B (Sec. 2.1) and names Giesekus and Phan-Thien-Tanner as the other
 * common differential models (Sec. 1, future work in Sec. 4); they differ
 * only in the relaxation part of the stress source chi of Sec. 2.3. */
enum {
  FVLB_MODEL_OLDROYD_B = 0,
  FVLB_MODEL_GIESEKUS = 1,
  FVLB_MODEL_PTT_LINEAR = 2,
  FVLB_MODEL_PTT_EXP = 3
};

/* Fields for fvlb_fields. */
enum {
  FVLB_FIELD_U = 0,    /* u = sum_{i!=0} c_i f_i + F/2 (Sec. 2.2)            */
  FVLB_FIELD_P = 1,    /* p of Sec. 2.2 / Appendix B                         */
  FVLB_FIELD_A = 2,    /* A_ab = sum_i h_ab,i (Sec. 2.3)                     */
  FVLB_FIELD_TAU_P = 3 /* tau_p = (eta_p / lambda)(A - I) (Sec. 2.1)         */
};

/* Device-memory hooks.  alloc(bytes, ctx) must return device memory aligned
 * to at least 256 bytes on the device that is current, or NULL; free(ptr,
 * ctx) releases it.  The hooks are process-wide and are captured by each
 * handle when it first allocates, so changing them later does not affect
 * existing handles.  Passing NULL for both restores cudaMalloc / cudaFree.
 * Returns FVLB_EINVAL if exactly one of the two is NULL. */
typedef void *(*fvlb_alloc_fn)(size_t bytes, void *ctx);
typedef void (*fvlb_free_fn)(void *ptr, void *ctx);
int fvlb_set_allocator(fvlb_alloc_fn alloc_fn, fvlb_free_fn free_fn, void *ctx);

/* Create a simulation on the current CUDA device.
 *   lattice   FVLB_D2Q9 or FVLB_D3Q19
 *   nx,ny,nz  grid size, each >= 1 (nz is ignored and taken as 1 in 2D);
 *             Q * N must stay below 2^32 (N <= ~226 M sites for D3Q19)
 *   tau_s     flow relaxation time tau_f = nu_s / c_s^2 + 1/2 (Sec. 2.2);
 *             must be > 0.5
 *   eta_p     polymer viscosity mu_p = nu_p (rho_0 = 1), >= 0 (Sec. 2.1)
 *   lambda    polymer relaxation time, > 0 (Sec. 2.1)
 *   force     body force, or NULL for none (copied)
 * The stress relaxation time is tau_h = 0.501 (Sec. 3).  No device memory
 * is allocated here: the state is allocated, and set to rest (u = 0, p = 0,
 * A = I) unless fvlb_init_fields was called, by the first call that needs
 * it.  Defaults: no walls (fully periodic), FVLB_FP64, FVLB_KERNEL_FUSED,
 * the legacy default stream.  On error *out is set to NULL. */
int fvlb_create(fvlb_t *out, int lattice, int nx, int ny, int nz,
                double tau_s, double eta_p, double lambda,
                const fvlb_force *force);

/* Halfway bounce-back walls: bit a of axis_mask puts a wall on both ends of
 * axis a (0 = x, 1 = y, 2 = z), at distance 1/2 outside the first and last
 * nodes, for both f and h; other axes are periodic.  A walled axis needs
 * at least 2 nodes.  FVLB_ESTATE once the state is allocated. */
int fvlb_set_walls(fvlb_t h, unsigned axis_mask);

/* Storage precision (FVLB_FP64 ...); FVLB_ESTATE once the state is
 * allocated. */
int fvlb_set_precision(fvlb_t h, int storage);

/* Kernel variant (FVLB_KERNEL_FUSED or FVLB_KERNEL_SPLIT); may be changed
 * at any time, both give the same results up to rounding order. */
int fvlb_set_kernel(fvlb_t h, int variant);

/* Scheme (FVLB_SCHEME_PRESENT, the default, or FVLB_SCHEME_ORIGINAL); may be
 * changed between steps.  The original scheme (Sec. 1; the comparison of
 * Tables 1 and 2) keeps the stress LB of Sec. 2.3 and replaces f^B by the
 * body force div tau_p: the polymer stress of every node goes to a working
 * array of C x pitch values (allocated through the allocator hooks at the
 * first step, field or reduction that needs it), its divergence is taken by
 * central differences (periodic wrap) and, next to a wall, by the one-sided
 * second-order difference through the two nodes inside, and it enters the
 * velocity, the Guo forcing term and the pressure as the body force does.
 * It runs as three launches per step: with FVLB_KERNEL_FUSED the stress,
 * its divergence per node (a second working array of D x pitch values) and
 * the fused step with that divergence in the body force and f^B off; with
 * FVLB_KERNEL_SPLIT the stress, the velocity and the collide-and-stream
 * kernel.  fvlb_fields and fvlb_reduce use the same total force.  FVLB_EINVAL for an unknown scheme, for a walled axis of
 * fewer than 3 nodes, or while a learned closure is attached. */
int fvlb_set_scheme(fvlb_t h, int scheme);

/* Constitutive model and its parameter; may be changed between steps.  With
 * M = A - I the stress source is chi = -P(M)/lambda + A.grad u +
 * (grad u)^T.A (Sec. 2.3) and P is
 *   FVLB_MODEL_OLDROYD_B   M                      (param ignored; default)
 *   FVLB_MODEL_GIESEKUS    M + alpha M.M           (param = alpha in [0, 1])
 *   FVLB_MODEL_PTT_LINEAR  (1 + eps tr M) M        (param = eps >= 0)
 *   FVLB_MODEL_PTT_EXP     exp(eps tr M) M         (param = eps >= 0)
 * (PTT without the slip parameter); tau_p = (eta_p/lambda) M in every model,
 * so f^B, the original scheme's body force, the fields and the diagnostics
 * are unchanged.  Every kernel variant, storage and scheme takes it.
 * FVLB_EINVAL for an unknown model, a negative or non-finite parameter, a
 * Giesekus alpha above 1, or a non-Oldroyd-B model while a learned closure
 * is attached (the network stands for the Oldroyd-B source). */
int fvlb_set_model(fvlb_t h, int model, double param);

/* CUDA stream (a cudaStream_t, or NULL for the legacy default stream) on
 * which all later GPU work of the handle is enqueued. */
int fvlb_set_stream(fvlb_t h, void *stream);

/* Initial state (Sec. 2.2 / 2.3 equilibria): f = f^eq(p0, u0),
 * h_ab,i = w_i A0_ab (1 + c_i.u0 / c_s^2), chi of the previous step unset
 * (the first step's d(chi)/dt correction is 0), t = 0.  u0 [N][D], p0 [N],
 * A0 [N][C] are host FP64 arrays; NULL means u0 = 0, p0 = 0, A0 = I.
 * Allocates the state if needed.  Returns after the upload completed. */
int fvlb_init_fields(fvlb_t h, const double *u0, const double *p0,
                     const double *A0);

/* Enqueue n >= 0 time steps on the handle's stream and return without
 * waiting.  Each step evaluates the force at the current t, then t += 1. */
int fvlb_step(fvlb_t h, long n);

/* Periodic finiteness check (failure detection): every `every` steps
 * fvlb_step enqueues the FP64 diagnostics of fvlb_reduce on the handle's
 * stream and copies them to page-locked host memory behind an event; no
 * call waits for it.  The result is collected by the next fvlb_step or
 * fvlb_status: once a check has found a non-finite value, fvlb_step enqueues
 * nothing more and returns FVLB_EUNSTABLE (the message names the step of the
 * check) until fvlb_init_fields or fvlb_load_state installs a new state.  At
 * most one check is in flight; a check point reached while the previous one
 * is still running is skipped.  every = 0 (the default) turns it off.
 * FVLB_EINVAL for every < 0. */
int fvlb_set_check_interval(fvlb_t h, long every);

/* Result of the periodic check: FVLB_OK, or FVLB_EUNSTABLE once a check has
 * found a non-finite value.  wait != 0 first waits for a check in flight,
 * then synchronises the stream and returns FVLB_ETIMEOUT if a step kernel's
 * bounded wait ran out. */
int fvlb_status(fvlb_t h, int wait);

/* Copy one field of the current state into host_out (FP64, layouts above),
 * synchronising the handle's stream.  count is the number of doubles the
 * buffer holds; if it is smaller than N * components, FVLB_EINVAL is
 * returned and nothing is written.  FVLB_ETIMEOUT (after the copy) if a step
 * kernel's bounded wait ran out since the state was installed. */
int fvlb_fields(fvlb_t h, int which, double *host_out, size_t count);

/* FP64 diagnostics of the current state, reduced on the GPU in a fixed
 * order (deterministic), synchronising the handle's stream:
 *   out[0]   sum_x sum_i f_i                      (mass drift; 0 at rest)
 *   out[1..3] sum_x sum_i c_i f_i                 (population momentum)
 *   out[4]   KE = (1/M) sum_x |u|^2 / 2           (Sec. 3.4)
 *   out[5]   PE = (1/M) sum_x tr(tau_p) / 2       (Sec. 3.4)
 *   out[6]   number of sites with a non-finite f, h or u
 *   out[7]   max_x |u|
 * Returns FVLB_EUNSTABLE (with out filled) if out[6] > 0, FVLB_ETIMEOUT (with
 * out filled) if a step kernel's bounded wait ran out. */
int fvlb_reduce(fvlb_t h, double out[8]);

/* Conformation check of the current state, FP64, on the GPU, synchronising
 * the handle's stream.  A must stay symmetric positive definite (Sec. 2.1;
 * it is the covariance of the polymer end-to-end vector), and losing that
 * is how runs fail at high Wi (the four-roll mill of Sec. 3.1 reaches
 * Wi = 5).  Per node the smallest eigenvalue of A (2D: closed form; 3D:
 * Jacobi plane rotations, six sweeps; both accurate to rounding relative to
 * |A|):
 *   out[0]   number of nodes whose smallest eigenvalue is not > 0
 *            (nodes with a non-finite A included)
 *   out[1]   smallest eigenvalue over the grid (non-finite nodes skipped)
 *   out[2]   largest tr A over the grid (Sec. 3.1 plots tr A)
 * Deterministic.  Uses the handle's reduction scratch; allocates the state
 * (at rest) if needed. */
int fvlb_conformation(fvlb_t h, double out[3]);

/* High-Wi repair of the conformation.  The paper runs the four-roll mill up
 * to Wi = 5 (Sec. 3.1) and leaves robustness at high Wi to future work
 * (Sec. 4); what fails there first is the positive definiteness of A.  For
 * every node whose A has its smallest eigenvalue below eps (> 0), A is
 * replaced by V max(Lambda, eps) V^T (eigenvalues clipped, eigenvectors
 * kept: cyclic Jacobi rotations in FP64), applied as h'_{ab,i} +=
 * w_i (A' - A)_ab on the node's stress populations, which leaves every
 * other moment of h unchanged.  Nodes with a non-finite A are counted and
 * left as they are.  *repaired (may be NULL) receives the number of nodes
 * changed.  Acts on the current state between steps; call it every few
 * steps (with fvlb_conformation to see when it is needed).  16-bit forms:
 * the changed populations are rounded again, their residual kept in the
 * FP32 rest population.  Errors: FVLB_EINVAL for eps <= 0 or not finite. */
int fvlb_repair_conformation(fvlb_t h, double eps, long long *repaired);

/* The diagnostics of fvlb_reduce for a state the caller holds in its own
 * device memory, with no device allocation at all.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory, such as code running inside a framework whose allocator
 * has reserved the GPU's memory for itself, or an asynchronous pipeline
 * that must not call cudaMalloc / cudaFree because they can synchronise
 * the device.
 *   lattice, storage  FVLB_D2Q9 / FVLB_D3Q19 and an FVLB_FP64 ... storage
 *   nx, ny, nz        grid (nz ignored in 2D); N = nx ny nz
 *   f                 device array f[Q][pitch] of the storage type
 *                     (16-bit forms: followed by U[D][pitch] in FP32)
 *   h                 device array h'[C][Q][pitch], h' = h - w_i delta_ab
 *                     (16-bit forms: followed by h0[C][pitch] in FP32);
 *                     the layouts of fvlb_save_state's image after its
 *                     64-byte header
 *   pitch             elements between population arrays, >= N
 *   eta_p, lambda     polymer viscosity and relaxation time (PE = tr tau_p/2)
 *   F                 host array of the uniform body force entering
 *                     u = sum c_i f_i + F/2, or NULL for 0
 *   out               device array of 8 doubles, filled as fvlb_reduce
 *                     fills it for a state of the present scheme with a
 *                     uniform body force (no FVLB_EUNSTABLE check: read
 *                     out[6]); for a four-roll force or an original-scheme
 *                     state, whose force varies from node to node, u and
 *                     KE are those of the uniform force F given here
 *   stream            cudaStream_t, or NULL for the legacy default stream
 * The work is enqueued on `stream` and the call returns without waiting.
 * Scratch: the per-block partial sums live in a file-scope device array of
 * 1024 x 8 doubles (64 KiB) that every GPU using the library keeps until
 * the process exits; a grid beyond the library's limit (Q * pitch >= 2^32)
 * is rejected with FVLB_EINVAL (the number of partial sums is capped at
 * 1024 for any N).  The first call on a device, and the first after its
 * context was reset, looks up the array's device address
 * (cudaGetSymbolAddress), so make that call before any stream capture.  All
 * calls share the array: calls whose kernels overlap on the GPU race and
 * give wrong results.  Rejected calls leave `out` untouched. */
int fvlb_reduce_noalloc(int lattice, int storage, int nx, int ny, int nz,
                        const void *f, const void *h, long long pitch,
                        double eta_p, double lambda, const double F[3],
                        double *out, void *stream);

/* ---------------------------------------------------------------------------
 * Batches: many independent D2Q9 grids (uneven sizes and parameters) in one
 * object, advanced by ONE persistent kernel launch per step (each resident
 * block walks a fixed list of tiles of all grids), the steps replayed from a
 * captured CUDA graph.  The update of every node is the one of fvlb_step
 * (Sec. 2.2-2.3) with the paper's scheme and the Oldroyd-B model (no scheme,
 * model or closure setting per instance); the arithmetic does not depend on
 * the tile shape, which an autotuner picks by timing candidate shapes on the
 * batch itself.
 * ------------------------------------------------------------------------- */
typedef struct fvlb_batch_s *fvlb_batch_t;

typedef struct {
  int nx, ny;          /* grid of this instance, >= 1 each */
  double tau_s;        /* > 0.5 */
  double eta_p;        /* >= 0 */
  double lambda;       /* > 0 */
  fvlb_force force;    /* body force (as for fvlb_create) */
  unsigned walls;      /* bit 0: walls on x, bit 1: walls on y */
} fvlb_instance;

/* Create a batch of `count` D2Q9 instances (specs copied) with storage
 * FVLB_FP64, FVLB_FP32, FVLB_FP16_DEV or FVLB_BF16_DEV; allocates all state
 * (through the allocator hooks) and sets every instance to rest.  The batch
 * owns a non-blocking stream until fvlb_batch_set_stream. */
int fvlb_batch_create(fvlb_batch_t *out, int lattice, int count,
                      const fvlb_instance *specs, int storage);

/* Use a caller stream (non-NULL: graph capture needs a non-legacy stream). */
int fvlb_batch_set_stream(fvlb_batch_t b, void *stream);

/* Initial fields of instance `index` (layouts as fvlb_init_fields); only
 * before the first step. */
int fvlb_batch_init_fields(fvlb_batch_t b, int index, const double *u0,
                           const double *p0, const double *A0);

/* Advance every instance n steps.  The first step is launched directly; the
 * first call with at least 18 further steps times 9 tile shapes over two real
 * steps each (synchronising) and keeps the fastest; later pairs of steps
 * replay a captured two-step graph. */
int fvlb_batch_step(fvlb_batch_t b, long n);

/* One field of instance `index` (as fvlb_fields), synchronising. */
int fvlb_batch_fields(fvlb_batch_t b, int index, int which, double *host_out,
                      size_t count);

/* Total nodes, algorithmic bytes per node update, chosen tile shape (32 gx
 * nodes x rows) and the tuned time per step in ms (0 before tuning); any
 * pointer may be NULL. */
int fvlb_batch_info(fvlb_batch_t b, long long *sites, double *bytes_per_update,
                    int *gx, int *rows, double *tuned_ms_per_step);

int fvlb_batch_synchronize(fvlb_batch_t b);
int fvlb_batch_get_time(fvlb_batch_t b, long *t);
const char *fvlb_batch_last_error(fvlb_batch_t b);
int fvlb_batch_destroy(fvlb_batch_t b); /* NULL-safe */

/* ---------------------------------------------------------------------------
 * Learned stress closure (no counterpart in the paper; a learned stand-in
 * for the analytic stress source chi of Sec. 2.3).  A network maps a node's
 * lambda-scaled state x = (lambda d_a u_b [D x D], A - I [C], dt/lambda [2D
 * only]) to y = lambda chi [C]: D2Q9 8 -> 64 -> 64 -> 3, D3Q19
 * 15 -> 64 -> 64 -> 6, GELU (tanh form).  It is trained on the GPU (FP32
 * master weights, Adam) on pairs that the plain method's state provides, and
 * runs in the step with FP16 weights on the tensor cores (FP32 accumulate);
 * per node, if ||chi_net - chi|| > tol ||chi|| the analytic chi is used.
 * ------------------------------------------------------------------------- */

/* Create a network for the lattice with room for `capacity` training pairs;
 * He-initialised from `seed`. */
int fvlb_mlp_create(fvlb_mlp_t *out, int lattice, long capacity, unsigned seed);

/* Append the pairs (x, lambda chi) of every stride-th node of the handle's
 * current state (FP64 or FP32 storage), up to the capacity. */
int fvlb_mlp_collect(fvlb_mlp_t m, fvlb_t h, long stride);
int fvlb_mlp_count(fvlb_mlp_t m, long *count);
/* First n collected pairs to host: x [n][IN], y [n][OUT] (FP32). */
int fvlb_mlp_get_pairs(fvlb_mlp_t m, float *x, float *y, long n);

/* Loss of training and of fvlb_mlp_grad: delta = 0 (default) the mean
 * squared error; delta > 0 the error of each pair weighted by
 * 1 / (mean_o y_o^2 + delta^2), i.e. relative to the pair's target. */
int fvlb_mlp_set_loss(fvlb_mlp_t m, double delta);

/* `steps` Adam steps (beta 0.9 / 0.999) of the loss on minibatches
 * of `batch` pairs (multiple of 64) drawn with a counter-based hash; the
 * last minibatch loss is returned.  Repacks the inference weights. */
int fvlb_mlp_train(fvlb_mlp_t m, long steps, int batch, double lr, double *last_loss);

/* FP32 master parameters W1[64][IN] b1[64] W2[64][64] b2[64] W3[OUT][64]
 * b3[OUT], concatenated. */
int fvlb_mlp_num_params(fvlb_mlp_t m, size_t *n);
int fvlb_mlp_get_params(fvlb_mlp_t m, float *host, size_t count);
int fvlb_mlp_set_params(fvlb_mlp_t m, const float *host, size_t count);

/* Gradient of the loss over n host pairs, computed by the training kernels
 * (FP32), and the loss. */
int fvlb_mlp_grad(fvlb_mlp_t m, const float *x, const float *y, long n, float *grad,
                  double *loss);

/* Tensor-core inference (FP16 weights, FP32 accumulate) of n host inputs. */
int fvlb_mlp_infer(fvlb_mlp_t m, const float *x, long n, float *y);

const char *fvlb_mlp_last_error(fvlb_mlp_t m);
int fvlb_mlp_destroy(fvlb_mlp_t m); /* NULL-safe */

/* Use the network m (NULL: the analytic source) in the handle's steps, with
 * fallback tolerance tol; needs FP32 storage and the fused kernel.  The
 * network must outlive its use.  Resets the closure statistics. */
int fvlb_set_closure(fvlb_t h, fvlb_mlp_t m, double tol);

/* Node updates that used the network, and fallbacks to the analytic source,
 * since fvlb_set_closure. */
int fvlb_closure_stats(fvlb_t h, long long *network_nodes, long long *fallback_nodes);

/* Wait for all GPU work of the handle. */
int fvlb_synchronize(fvlb_t h);

/* Current step count. */
int fvlb_get_time(fvlb_t h, long *t);

/* Checkpoint / resume: the raw state (populations, previous chi, step
 * count and first-step flag) as an opaque byte image of fvlb_state_size
 * bytes, valid for a handle with the same lattice, grid and precision.
 * fvlb_load_state returns FVLB_EINVAL on a size or header mismatch. */
int fvlb_state_size(fvlb_t h, size_t *bytes);
int fvlb_save_state(fvlb_t h, void *host_buf, size_t bytes);
int fvlb_load_state(fvlb_t h, const void *host_buf, size_t bytes);

/* Bytes of HBM the step kernel moves per lattice update by construction
 * (each population and chi read once and written once), for roofline
 * accounting: 2 (Q + C Q) s + 2 C s_chi with s the storage size. */
int fvlb_bytes_per_update(fvlb_t h, double *bytes);

/* Last error message of the handle, or of the last failed fvlb_create /
 * fvlb_set_allocator if h is NULL.  Never NULL. */
const char *fvlb_last_error(fvlb_t h);

/* Release the handle and its device memory (after waiting for its stream).
 * NULL-safe. */
int fvlb_destroy(fvlb_t h);

#ifdef __cplusplus
}
#endif

#endif /* FVLB_H */
