/*
 * fvlb_oracle.c -- plain, slow FP64 CPU oracle for the fluctuating lattice
 * Boltzmann method for Oldroyd-B fluids (Wang, Liu, Wang, Yu, Ji,
 * arXiv 2506.13072, "A fluctuating lattice Boltzmann method for viscoelastic
 * fluid flows").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or helper
 * with the CUDA library; the lattice constants and the f^B matrices below are
 * typed in from the paper on their own.
 *
 * Everything is FP64, site-major (array-of-structures), one loop per step of
 * the algorithm, in the order the paper states them.  The full D x D
 * conformation tensor is stored (4 components in 2D, 9 in 3D, as in the
 * paper's Tables 1 and 2), so symmetry of A can be checked rather than
 * assumed.
 *
 * Lattice units: dx = dt = c = 1, c_s^2 = 1/3.
 *
 * Readings of points the paper leaves open:
 *   R1  D3Q19 weights are not printed: 1/3, 1/18 (axis), 1/36 (diagonal).
 *   R2  grad u is a second-order central difference of the same-step
 *       velocity; at a node next to a halfway-bounce-back wall the one-sided
 *       three-point derivative through the wall point (distance 1/2, u = 0)
 *       is used.  (grad u)_{ab} = d_a u_b.
 *   R3  The 0.5 dt^2 d(chi_i)/dt term of the stress LB (Sec. 2.3) is the
 *       backward difference 0.5 * phi_i(u^n) * (chi^n - chi^{n-1}) with
 *       phi_i = w_i [1 + (1 - 1/(2 tau_h)) c_i.u / c_s^2]; it is zero on the
 *       first step.
 *   R4  The stress distributions h use the same lattice as the flow.
 *   R5  Walls are halfway bounce-back for both f and h.
 *   R6  The body force is evaluated at the time level of the step, t_n = n.
 *   R7  Initial state: f = f^eq(p0, u0), h = h^eq(A0, u0) (with R10).
 *   R8  The "original" scheme the paper compares against (Sec. 1, Tables 1
 *       and 2) adds the polymer stress divergence to the momentum equation
 *       as a body force instead of the fluctuation term: f^B = 0 and
 *       F -> F + div tau_p, with tau_p from A of the same step and
 *       (div tau_p)_b = sum_a d_a tau_ab by second-order central
 *       differences (periodic wrap); at a node next to a wall the
 *       second-order one-sided difference through the two nodes inside,
 *       (-3 t0 + 4 t1 - t2) / 2 (sign mirrored at the upper wall), since no
 *       stress is known at the wall.  The total force enters u, the Guo
 *       term and the pressure as the body force does in the present scheme.
 *   R9  Other constitutive models (the paper names Giesekus and
 *       Phan-Thien-Tanner in Sec. 1 and leaves them to future work in
 *       Sec. 4) change only the relaxation part of chi (Sec. 2.3):
 *       chi = -P(A)/lambda + A.grad u + (grad u)^T.A, with M = A - I and
 *         Oldroyd-B          P = M
 *         Giesekus (alpha)   P = M + alpha M.M
 *         linear PTT (eps)   P = (1 + eps tr M) M
 *         exponential PTT    P = exp(eps tr M) M
 *       (PTT without the slip parameter), tau_p = (eta_p/lambda) M in all
 *       four.  The trace runs over the D x D tensor; in 2D A_zz = 1, so M has
 *       no z entries and the 2D restriction is exact.
 *   R11 High-Wi repair (the paper runs the four-roll mill up to Wi = 5,
 *       Sec. 3.1, and leaves robustness at high Wi to future work, Sec. 4):
 *       A must stay symmetric positive definite; a node whose A = sum_i h_i
 *       has its smallest eigenvalue below a floor eps is given
 *       A' = V max(Lambda, eps) V^T (eigenvalues clipped, eigenvectors
 *       kept) by adding w_i (A' - A) to its stress populations, which
 *       changes the zeroth moment of h only (sum_i w_i c_i = 0).  Applied
 *       between steps, on request.
 *   R10 The stress equilibrium has zeroth moment A (Sec. 2.3: A is the
 *       zeroth moment of h, and the collision conserves it apart from the
 *       source).  The weights typed in below sum to 1 - 5.6e-17 in FP64,
 *       and with h ~ w_i A every collision would then scale A by about
 *       1 - 1.1e-16 (1/tau_h ~ 2); over thousands of steps that drift is
 *       a relative error of 1e-12 in A - I where |A - I| << |A|.  So the
 *       rest direction's equilibrium is the zeroth-moment condition solved
 *       for it, h^eq_0 = A - sum_{i>=1} h^eq_i, which equals w_0 A exactly
 *       for exact weights.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_D2Q9 9
#define ORC_D3Q19 19

#define ORC_FORCE_NONE 0
#define ORC_FORCE_CONST 1
#define ORC_FORCE_FOUR_ROLL 2
#define ORC_FORCE_COSINE 3

#define ORC_FIELD_U 0
#define ORC_FIELD_P 1
#define ORC_FIELD_A 2
#define ORC_FIELD_TAU_P 3

#define CS2 (1.0 / 3.0)

/* ---------------------------------------------------------------------------
 * Lattices.
 * D2Q9 velocities and weights: Sec. 2.2 (the c_i matrix and the w_i cases).
 * D3Q19 velocities: Appendix A (c_i matrix).  Weights: reading R1.
 * ------------------------------------------------------------------------- */
static const int C9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const int C19[19][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W19[19] = {
    1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* ---------------------------------------------------------------------------
 * f^B matrices (pseudo-inverse solutions of the moment constraints).
 * D2Q9, Sec. 2.2 / Appendix A: f^B = -1/(72 tau_f) * FB9 * (t_yx, t_xx, t_xy,
 * t_yy)^T.
 * ------------------------------------------------------------------------- */
static const double FB9[9][4] = {
    {0, -24, 0, -24}, {0, 12, 0, -24},  {0, -24, 0, 12},
    {0, 12, 0, -24},  {0, -24, 0, 12},  {9, 12, 9, 12},
    {-9, 12, -9, 12}, {9, 12, 9, 12},   {-9, 12, -9, 12}};

/* D3Q19, Appendix A: f^B = FB19 * b with
 * b = (-t_xx, -t_yy, -t_zz, -t_xy, -t_xz, -t_yx, -t_yz, -t_zx, -t_zy,
 *      0, 0, 0, 0) / tau_f.
 * Only the first nine columns multiply non-zero entries of b; the last four
 * (momentum and mass rows of the constraint system) are kept for the
 * pseudo-inverse check in the tests. */
#define R(a, b) ((double)(a) / (double)(b))
static const double FB19[19][13] = {
    {R(-5, 21), R(-5, 21), R(-5, 21), 0, 0, 0, 0, 0, 0, 0, 0, 0, R(3, 7)},
    {R(1, 42), R(-1, 7), R(-1, 7), 0, 0, 0, 0, 0, 0, R(1, 10), 0, 0, R(4, 21)},
    {R(1, 42), R(-1, 7), R(-1, 7), 0, 0, 0, 0, 0, 0, R(-1, 10), 0, 0, R(4, 21)},
    {R(-1, 7), R(1, 42), R(-1, 7), 0, 0, 0, 0, 0, 0, 0, R(1, 10), 0, R(4, 21)},
    {R(-1, 7), R(1, 42), R(-1, 7), 0, 0, 0, 0, 0, 0, 0, R(-1, 10), 0, R(4, 21)},
    {R(-1, 7), R(-1, 7), R(1, 42), 0, 0, 0, 0, 0, 0, 0, 0, R(1, 10), R(4, 21)},
    {R(-1, 7), R(-1, 7), R(1, 42), 0, 0, 0, 0, 0, 0, 0, 0, R(-1, 10), R(4, 21)},
    {R(5, 42), R(5, 42), R(-1, 21), R(1, 8), 0, R(1, 8), 0, 0, 0, R(1, 10), R(1, 10), 0, R(-1, 21)},
    {R(5, 42), R(5, 42), R(-1, 21), R(1, 8), 0, R(1, 8), 0, 0, 0, R(-1, 10), R(-1, 10), 0, R(-1, 21)},
    {R(5, 42), R(5, 42), R(-1, 21), R(-1, 8), 0, R(-1, 8), 0, 0, 0, R(1, 10), R(-1, 10), 0, R(-1, 21)},
    {R(5, 42), R(5, 42), R(-1, 21), R(-1, 8), 0, R(-1, 8), 0, 0, 0, R(-1, 10), R(1, 10), 0, R(-1, 21)},
    {R(5, 42), R(-1, 21), R(5, 42), 0, R(1, 8), 0, 0, R(1, 8), 0, R(1, 10), 0, R(1, 10), R(-1, 21)},
    {R(5, 42), R(-1, 21), R(5, 42), 0, R(1, 8), 0, 0, R(1, 8), 0, R(-1, 10), 0, R(-1, 10), R(-1, 21)},
    {R(5, 42), R(-1, 21), R(5, 42), 0, R(-1, 8), 0, 0, R(-1, 8), 0, R(1, 10), 0, R(-1, 10), R(-1, 21)},
    {R(5, 42), R(-1, 21), R(5, 42), 0, R(-1, 8), 0, 0, R(-1, 8), 0, R(-1, 10), 0, R(1, 10), R(-1, 21)},
    {R(-1, 21), R(5, 42), R(5, 42), 0, 0, 0, R(1, 8), 0, R(1, 8), 0, R(1, 10), R(1, 10), R(-1, 21)},
    {R(-1, 21), R(5, 42), R(5, 42), 0, 0, 0, R(1, 8), 0, R(1, 8), 0, R(-1, 10), R(-1, 10), R(-1, 21)},
    {R(-1, 21), R(5, 42), R(5, 42), 0, 0, 0, R(-1, 8), 0, R(-1, 8), 0, R(1, 10), R(-1, 10), R(-1, 21)},
    {R(-1, 21), R(5, 42), R(5, 42), 0, 0, 0, R(-1, 8), 0, R(-1, 8), 0, R(-1, 10), R(1, 10), R(-1, 21)}};
#undef R

/* Full-tensor index helpers: component (a, b) of a D x D tensor. */
#define T(D, a, b) ((a) * (D) + (b))

typedef struct {
  int Q, D;
  const int (*c)[3];
  const double *w;
  int opp[19];
} lattice_t;

static int lattice_get(int lattice, lattice_t *L) {
  if (lattice == ORC_D2Q9) {
    L->Q = 9; L->D = 2; L->c = C9; L->w = W9;
  } else if (lattice == ORC_D3Q19) {
    L->Q = 19; L->D = 3; L->c = C19; L->w = W19;
  } else {
    return -1;
  }
  for (int i = 0; i < L->Q; ++i) {
    for (int j = 0; j < L->Q; ++j) {
      if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] &&
          L->c[j][2] == -L->c[i][2]) {
        L->opp[i] = j;
      }
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Per-site building blocks (each exported for the tests).
 * ------------------------------------------------------------------------- */

static double dot3(const int c[3], const double v[3]) {
  return c[0] * v[0] + c[1] * v[1] + c[2] * v[2];
}

/* s_i(u) = w_i [3 c_i.u + 4.5 (c_i.u)^2 - 1.5 |u|^2]   (Sec. 2.2, s_i(u)). */
static double s_i(const lattice_t *L, int i, const double u[3]) {
  const double cu = dot3(L->c[i], u);
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return L->w[i] * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* lambda_i = w_i / c_s^2 for i != 0, lambda_0 = (w_0 - 1)/c_s^2 (Sec. 2.2). */
static double lambda_i(const lattice_t *L, int i) {
  return i == 0 ? (L->w[0] - 1.0) / CS2 : L->w[i] / CS2;
}

/* f_i^eq = lambda_i p + w_i [c_i.u / c_s^2 + uu:(c_i c_i - c_s^2 I)/(2 c_s^4)]
 * (Sec. 2.2, equilibrium).  The bracket equals s_i(u) / w_i. */
static void feq_site(const lattice_t *L, double p, const double u[3],
                     double *out) {
  for (int i = 0; i < L->Q; ++i) out[i] = lambda_i(L, i) * p + s_i(L, i, u);
}

/* Guo forcing term (Sec. 2.2):
 * F_i = w_i (1 - 1/(2 tau_f)) [c_i.F / c_s^2 + (Fu + uF):(c_i c_i - c_s^2 I)
 *       / (2 c_s^4)], written out as
 *       w_i (1 - 1/(2 tau_f)) [3 c_i.F + 9 (c_i.F)(c_i.u) - 3 F.u]. */
static void forcing_site(const lattice_t *L, double tau_f, const double F[3],
                         const double u[3], double *out) {
  const double pref = 1.0 - 0.5 / tau_f;
  const double Fu = F[0] * u[0] + F[1] * u[1] + F[2] * u[2];
  for (int i = 0; i < L->Q; ++i) {
    const double cF = dot3(L->c[i], F);
    const double cu = dot3(L->c[i], u);
    out[i] = L->w[i] * pref * (3.0 * cF + 9.0 * cF * cu - 3.0 * Fu);
  }
}

/* Polymer stress fluctuation term f^B from the full D x D polymer stress
 * tau_p (row-major), Sec. 2.2 and Appendix A. */
static void fB_site(const lattice_t *L, double tau_f, const double *tau_p,
                    double *out) {
  if (L->D == 2) {
    const double v[4] = {tau_p[T(2, 1, 0)], tau_p[T(2, 0, 0)],
                         tau_p[T(2, 0, 1)], tau_p[T(2, 1, 1)]};
    for (int i = 0; i < 9; ++i) {
      double acc = 0.0;
      for (int k = 0; k < 4; ++k) acc += FB9[i][k] * v[k];
      out[i] = -acc / (72.0 * tau_f);
    }
  } else {
    double b[13];
    b[0] = -tau_p[T(3, 0, 0)] / tau_f;
    b[1] = -tau_p[T(3, 1, 1)] / tau_f;
    b[2] = -tau_p[T(3, 2, 2)] / tau_f;
    b[3] = -tau_p[T(3, 0, 1)] / tau_f;
    b[4] = -tau_p[T(3, 0, 2)] / tau_f;
    b[5] = -tau_p[T(3, 1, 0)] / tau_f;
    b[6] = -tau_p[T(3, 1, 2)] / tau_f;
    b[7] = -tau_p[T(3, 2, 0)] / tau_f;
    b[8] = -tau_p[T(3, 2, 1)] / tau_f;
    b[9] = b[10] = b[11] = b[12] = 0.0;
    for (int i = 0; i < 19; ++i) {
      double acc = 0.0;
      for (int k = 0; k < 13; ++k) acc += FB19[i][k] * b[k];
      out[i] = acc;
    }
  }
}

/* Pressure, Sec. 2.2 and Appendix B:
 * p = c_s^2/(1 - w_0) [sum_{i!=0} f_i + s_0(u) + tau_f F_0 + tau_f f_0^B]. */
static double pressure_site(const lattice_t *L, double tau_f, const double *f,
                            const double u[3], double F0, double fB0) {
  double sum = 0.0;
  for (int i = 1; i < L->Q; ++i) sum += f[i];
  return CS2 / (1.0 - L->w[0]) * (sum + s_i(L, 0, u) + tau_f * F0 + tau_f * fB0);
}

/* ---------------------------------------------------------------------------
 * The simulation object.
 * ------------------------------------------------------------------------- */
typedef struct orc {
  lattice_t L;
  int D, Q, DD;
  int n[3];          /* nx, ny, nz (nz = 1 in 2D) */
  long N;
  int walls[3];      /* halfway bounce-back walls bounding axis a */
  double tau_f, tau_h, eta_p, lambda;
  int force_kind;
  double F0[3], k, omega;
  double *f, *f_new; /* [N][Q] */
  double *h, *h_new; /* [N][DD][Q] */
  double *chi_old;   /* [N][DD] */
  double *u;         /* [N][3] velocity of the current step */
  double *A;         /* [N][DD] conformation of the current step */
  int scheme;        /* 0: present (f^B), 1: original (div tau_p as a force) */
  int model;         /* constitutive model (reading R9): 0 Oldroyd-B,
                        1 Giesekus, 2 linear PTT, 3 exponential PTT */
  double mpar;       /* its parameter: alpha (Giesekus) or eps (PTT) */
  double *divt;      /* [N][3] div tau_p of the current step (scheme 1) */
  int first;
  long t;
} orc;

static long site_index(const orc *o, int x, int y, int z) {
  return ((long)z * o->n[1] + y) * o->n[0] + x;
}

/* Body force at node (x, y, z) and time t (reading R6). */
static void force_at(const orc *o, int x, int y, int z, long t, double F[3]) {
  (void)z;
  F[0] = F[1] = F[2] = 0.0;
  switch (o->force_kind) {
    case ORC_FORCE_CONST:
      F[0] = o->F0[0]; F[1] = o->F0[1]; F[2] = o->F0[2];
      break;
    case ORC_FORCE_FOUR_ROLL:
      /* Sec. 3.1: g = A (sin x cos y, -cos x sin y) on a 2 pi periodic box;
       * on the lattice the phase of node i is k i. */
      F[0] = o->F0[0] * sin(o->k * x) * cos(o->k * y);
      F[1] = -o->F0[0] * cos(o->k * x) * sin(o->k * y);
      break;
    case ORC_FORCE_COSINE: {
      /* Sec. 3.3: g_x = A cos(omega t). */
      const double c = cos(o->omega * (double)t);
      F[0] = o->F0[0] * c; F[1] = o->F0[1] * c; F[2] = o->F0[2] * c;
      break;
    }
    default:
      break;
  }
}

orc *orc_create(int lattice, int nx, int ny, int nz, double tau_s,
                double eta_p, double lambda, int force_kind,
                const double *F0, double k, double omega) {
  orc *o = (orc *)calloc(1, sizeof(orc));
  if (!o) return NULL;
  if (lattice_get(lattice, &o->L) != 0) { free(o); return NULL; }
  o->D = o->L.D; o->Q = o->L.Q; o->DD = o->D * o->D;
  if (o->D == 2) nz = 1;
  if (nx < 1 || ny < 1 || nz < 1 || tau_s <= 0.5 || lambda <= 0.0 ||
      eta_p < 0.0) {
    free(o);
    return NULL;
  }
  o->n[0] = nx; o->n[1] = ny; o->n[2] = nz;
  o->N = (long)nx * ny * nz;
  o->tau_f = tau_s;
  o->tau_h = 0.501; /* Sec. 3: tau_h fixed at 0.501 */
  o->eta_p = eta_p;
  o->lambda = lambda;
  o->force_kind = force_kind;
  if (F0) { o->F0[0] = F0[0]; o->F0[1] = F0[1]; o->F0[2] = F0[2]; }
  o->k = k;
  o->omega = omega;
  const long N = o->N;
  o->f = (double *)calloc((size_t)N * o->Q, sizeof(double));
  o->f_new = (double *)calloc((size_t)N * o->Q, sizeof(double));
  o->h = (double *)calloc((size_t)N * o->DD * o->Q, sizeof(double));
  o->h_new = (double *)calloc((size_t)N * o->DD * o->Q, sizeof(double));
  o->chi_old = (double *)calloc((size_t)N * o->DD, sizeof(double));
  o->u = (double *)calloc((size_t)N * 3, sizeof(double));
  o->A = (double *)calloc((size_t)N * o->DD, sizeof(double));
  o->divt = (double *)calloc((size_t)N * 3, sizeof(double));
  if (!o->f || !o->f_new || !o->h || !o->h_new || !o->chi_old || !o->u ||
      !o->A || !o->divt) {
    free(o->f); free(o->f_new); free(o->h); free(o->h_new);
    free(o->chi_old); free(o->u); free(o->A); free(o->divt); free(o);
    return NULL;
  }
  o->first = 1;
  return o;
}

void orc_destroy(orc *o) {
  if (!o) return;
  free(o->f); free(o->f_new); free(o->h); free(o->h_new);
  free(o->chi_old); free(o->u); free(o->A); free(o->divt); free(o);
}

int orc_set_walls(orc *o, unsigned mask) {
  for (int a = 0; a < 3; ++a) {
    const int on = (mask >> a) & 1u;
    if (on && (a >= o->D || o->n[a] < (o->scheme ? 3 : 2))) return -1;
  }
  for (int a = 0; a < 3; ++a) o->walls[a] = (mask >> a) & 1u;
  return 0;
}

/* Scheme 0: the present method (Sec. 2.2, f^B); scheme 1: the original one
 * (reading R8), which needs 3 nodes across a walled axis. */
int orc_set_scheme(orc *o, int scheme) {
  if (scheme != 0 && scheme != 1) return -1;
  if (scheme == 1)
    for (int a = 0; a < 3; ++a)
      if (o->walls[a] && o->n[a] < 3) return -1;
  o->scheme = scheme;
  return 0;
}

/* Constitutive model (reading R9) and its parameter. */
int orc_set_model(orc *o, int model, double par) {
  if (model < 0 || model > 3 || !(par >= 0.0)) return -1;
  o->model = model;
  o->mpar = par;
  return 0;
}

void orc_set_tau_h(orc *o, double tau_h) { o->tau_h = tau_h; }

long orc_time(const orc *o) { return o->t; }

/* Initial state (reading R7): f = f^eq(p0, u0), h_ab = w_i A0_ab (1 + 3 c.u0).
 * u0: [N][D] or NULL (rest); p0: [N] or NULL (0); A0: [N][DD] or NULL (I). */
void orc_init(orc *o, const double *u0, const double *p0, const double *A0) {
  const lattice_t *L = &o->L;
  for (long s = 0; s < o->N; ++s) {
    double u[3] = {0.0, 0.0, 0.0};
    if (u0) for (int a = 0; a < o->D; ++a) u[a] = u0[s * o->D + a];
    const double p = p0 ? p0[s] : 0.0;
    feq_site(L, p, u, &o->f[s * o->Q]);
    for (int ab = 0; ab < o->DD; ++ab) {
      const int a = ab / o->D, b = ab % o->D;
      const double Aab = A0 ? A0[s * o->DD + ab] : (a == b ? 1.0 : 0.0);
      double *h = &o->h[(s * o->DD + ab) * o->Q];
      double moving = 0.0;   /* rest direction from the zeroth moment (R10) */
      for (int i = 1; i < o->Q; ++i) {
        h[i] = L->w[i] * Aab * (1.0 + dot3(L->c[i], u) / CS2);
        moving += h[i];
      }
      h[0] = Aab - moving;
    }
    for (int ab = 0; ab < o->DD; ++ab) o->chi_old[s * o->DD + ab] = 0.0;
  }
  o->first = 1;
  o->t = 0;
}

/* (eta_p / lambda)(A - I)_{ab} at site s (Sec. 2.1) */
static double tau_p_at(const orc *o, long s, int a, int b) {
  return o->eta_p / o->lambda * (o->A[s * o->DD + T(o->D, a, b)] - (a == b ? 1.0 : 0.0));
}

/* d_a tau_ab at node p (reading R8). */
static double dtau(const orc *o, const int p[3], int a, int b) {
  const int n = o->n[a];
  int q[3] = {p[0], p[1], p[2]};
  if (n == 1) return 0.0;
  if (o->walls[a] && (p[a] == 0 || p[a] == n - 1)) {
    const int dir = p[a] == 0 ? 1 : -1;
    const double t0 = tau_p_at(o, site_index(o, p[0], p[1], p[2]), a, b);
    q[a] = p[a] + dir;
    const double t1 = tau_p_at(o, site_index(o, q[0], q[1], q[2]), a, b);
    q[a] = p[a] + 2 * dir;
    const double t2 = tau_p_at(o, site_index(o, q[0], q[1], q[2]), a, b);
    return dir * 0.5 * (-3.0 * t0 + 4.0 * t1 - t2);
  }
  q[a] = (p[a] + 1) % n;
  const double tp = tau_p_at(o, site_index(o, q[0], q[1], q[2]), a, b);
  q[a] = (p[a] - 1 + n) % n;
  const double tm = tau_p_at(o, site_index(o, q[0], q[1], q[2]), a, b);
  return 0.5 * (tp - tm);
}

/* Body force of the step at a site: the external force, plus div tau_p in
 * the original scheme. */
static void total_force(const orc *o, int x, int y, int z, double F[3]) {
  force_at(o, x, y, z, o->t, F);
  if (o->scheme) {
    const long s = site_index(o, x, y, z);
    for (int b = 0; b < 3; ++b) F[b] += o->divt[s * 3 + b];
  }
}

/* Conformation (Sec. 2.3, A_ab = sum_i h_ab,i), in the original scheme the
 * stress divergence (reading R8), and velocity (Sec. 2.2,
 * u = sum_{i!=0} c_i f_i + F/2) of every site, at the current time. */
static void moments_sweep(orc *o) {
  for (long s = 0; s < o->N; ++s)
    for (int ab = 0; ab < o->DD; ++ab) {
      double m = 0.0;
      for (int i = 0; i < o->Q; ++i) m += o->h[(s * o->DD + ab) * o->Q + i];
      o->A[s * o->DD + ab] = m;
    }
  if (o->scheme)
    for (int z = 0; z < o->n[2]; ++z)
      for (int y = 0; y < o->n[1]; ++y)
        for (int x = 0; x < o->n[0]; ++x) {
          const int p[3] = {x, y, z};
          const long s = site_index(o, x, y, z);
          for (int b = 0; b < 3; ++b) {
            double d = 0.0;
            if (b < o->D)
              for (int a = 0; a < o->D; ++a) d += dtau(o, p, a, b);
            o->divt[s * 3 + b] = d;
          }
        }
  for (int z = 0; z < o->n[2]; ++z)
    for (int y = 0; y < o->n[1]; ++y)
      for (int x = 0; x < o->n[0]; ++x) {
        const long s = site_index(o, x, y, z);
        const double *f = &o->f[s * o->Q];
        double F[3];
        total_force(o, x, y, z, F);
        for (int a = 0; a < 3; ++a) {
          double m = 0.0;
          for (int i = 1; i < o->Q; ++i) m += o->L.c[i][a] * f[i];
          o->u[s * 3 + a] = m + 0.5 * F[a];
        }
      }
}

/* Relaxation part P(A) of chi (Sec. 2.3; other models: reading R9), full
 * D x D tensor. */
static void relax_term(const orc *o, const double *A, double *P) {
  const int D = o->D;
  double M[9];
  double tr = 0.0;
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) M[T(D, a, b)] = A[T(D, a, b)] - (a == b ? 1.0 : 0.0);
  for (int a = 0; a < D; ++a) tr += M[T(D, a, a)];
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      const double m = M[T(D, a, b)];
      double v;
      if (o->model == 1) {
        double mm = 0.0;
        for (int g = 0; g < D; ++g) mm += M[T(D, a, g)] * M[T(D, g, b)];
        v = m + o->mpar * mm;
      } else if (o->model == 2) {
        v = (1.0 + o->mpar * tr) * m;
      } else if (o->model == 3) {
        v = exp(o->mpar * tr) * m;
      } else {
        v = m;
      }
      P[T(D, a, b)] = v;
    }
}

/* d u_b / d x_a at node p (reading R2). */
static double grad_component(const orc *o, const int p[3], int a, int b) {
  const int n = o->n[a];
  int q[3] = {p[0], p[1], p[2]};
  if (!o->walls[a]) {
    if (n == 1) return 0.0;
    q[a] = (p[a] + 1) % n;
    const double up = o->u[site_index(o, q[0], q[1], q[2]) * 3 + b];
    q[a] = (p[a] - 1 + n) % n;
    const double um = o->u[site_index(o, q[0], q[1], q[2]) * 3 + b];
    return 0.5 * (up - um);
  }
  const double u0 = o->u[site_index(o, p[0], p[1], p[2]) * 3 + b];
  if (p[a] == 0) {
    /* quadratic through (-1/2, 0), (0, u0), (1, u1), differentiated at 0 */
    q[a] = 1;
    const double u1 = o->u[site_index(o, q[0], q[1], q[2]) * 3 + b];
    return u0 + u1 / 3.0;
  }
  if (p[a] == n - 1) {
    /* mirror image at the upper wall */
    q[a] = n - 2;
    const double u1 = o->u[site_index(o, q[0], q[1], q[2]) * 3 + b];
    return -(u0 + u1 / 3.0);
  }
  q[a] = p[a] + 1;
  const double up = o->u[site_index(o, q[0], q[1], q[2]) * 3 + b];
  q[a] = p[a] - 1;
  const double um = o->u[site_index(o, q[0], q[1], q[2]) * 3 + b];
  return 0.5 * (up - um);
}

/* Destination of population i leaving node p: periodic wrap, or halfway
 * bounce-back (same node, opposite direction) through a wall. */
static long stream_dest(const orc *o, const int p[3], int i, int *i_out) {
  int q[3];
  for (int a = 0; a < 3; ++a) {
    q[a] = p[a] + o->L.c[i][a];
    if (q[a] < 0 || q[a] >= o->n[a]) {
      if (o->walls[a]) {
        *i_out = o->L.opp[i];
        return site_index(o, p[0], p[1], p[2]);
      }
      q[a] = (q[a] + o->n[a]) % o->n[a];
    }
  }
  *i_out = i;
  return site_index(o, q[0], q[1], q[2]);
}

/* One time step: collide (Sec. 2.2 evolution equation for f, Sec. 2.3
 * evolution equation for h), then stream. */
static void step_once(orc *o) {
  const lattice_t *L = &o->L;
  const int Q = o->Q, D = o->D, DD = o->DD;
  double fB[19], Fi[19], feq[19], tau_p[9], grad[9], chi[9], relax[9];

  moments_sweep(o);

  for (int z = 0; z < o->n[2]; ++z)
    for (int y = 0; y < o->n[1]; ++y)
      for (int x = 0; x < o->n[0]; ++x) {
        const int p[3] = {x, y, z};
        const long s = site_index(o, x, y, z);
        const double *f = &o->f[s * Q];
        const double *A = &o->A[s * DD];
        const double *u = &o->u[s * 3];
        double F[3];
        total_force(o, x, y, z, F);

        /* tau_p = (eta_p / lambda)(A - I), Sec. 2.1 */
        for (int a = 0; a < D; ++a)
          for (int b = 0; b < D; ++b)
            tau_p[T(D, a, b)] =
                o->eta_p / o->lambda * (A[T(D, a, b)] - (a == b ? 1.0 : 0.0));

        fB_site(L, o->tau_f, tau_p, fB);
        if (o->scheme)
          for (int i = 0; i < Q; ++i) fB[i] = 0.0;  /* reading R8 */
        forcing_site(L, o->tau_f, F, u, Fi);
        const double pr = pressure_site(L, o->tau_f, f, u, Fi[0], fB[0]);
        feq_site(L, pr, u, feq);

        /* grad u and chi = -P(A)/lambda + A.grad u + (grad u)^T.A, with
         * P(A) = A - I for Oldroyd-B (Sec. 2.3) or the model of reading R9 */
        for (int a = 0; a < D; ++a)
          for (int b = 0; b < D; ++b) grad[T(D, a, b)] = grad_component(o, p, a, b);
        relax_term(o, A, relax);
        for (int a = 0; a < D; ++a)
          for (int b = 0; b < D; ++b) {
            double v = -relax[T(D, a, b)] / o->lambda;
            for (int g = 0; g < D; ++g) {
              v += A[T(D, a, g)] * grad[T(D, g, b)];
              v += grad[T(D, g, a)] * A[T(D, g, b)];
            }
            chi[T(D, a, b)] = v;
          }
        double *chi_old = &o->chi_old[s * DD];
        if (o->first)
          for (int ab = 0; ab < DD; ++ab) chi_old[ab] = chi[ab];

        /* f: collide and stream */
        for (int i = 0; i < Q; ++i) {
          const double post = f[i] - (f[i] - feq[i]) / o->tau_f + fB[i] + Fi[i];
          int j;
          const long d = stream_dest(o, p, i, &j);
          o->f_new[d * Q + j] = post;
        }

        /* h: collide and stream.  h^eq_i = w_i A (1 + c_i.u / c_s^2) for
         * i >= 1; the rest direction takes what the zeroth moment leaves,
         * h^eq_0 = A - sum_{i>=1} h^eq_i (reading R10). */
        for (int ab = 0; ab < DD; ++ab) {
          const double *h = &o->h[(s * DD + ab) * Q];
          double heq[19];
          double moving = 0.0;
          for (int i = 1; i < Q; ++i) {
            heq[i] = L->w[i] * A[ab] * (1.0 + dot3(L->c[i], u) / CS2);
            moving += heq[i];
          }
          heq[0] = A[ab] - moving;
          for (int i = 0; i < Q; ++i) {
            const double cu = dot3(L->c[i], u);
            const double phi =
                L->w[i] * (1.0 + (1.0 - 0.5 / o->tau_h) * cu / CS2);
            const double post = h[i] - (h[i] - heq[i]) / o->tau_h + phi * chi[ab] +
                                0.5 * phi * (chi[ab] - chi_old[ab]);
            int j;
            const long d = stream_dest(o, p, i, &j);
            o->h_new[(d * DD + ab) * Q + j] = post;
          }
        }
        for (int ab = 0; ab < DD; ++ab) chi_old[ab] = chi[ab];
      }

  double *tmp = o->f; o->f = o->f_new; o->f_new = tmp;
  tmp = o->h; o->h = o->h_new; o->h_new = tmp;
  o->first = 0;
  o->t += 1;
}

void orc_step(orc *o, long nsteps) {
  for (long k = 0; k < nsteps; ++k) step_once(o);
}

/* Macroscopic fields at the current time.
 * U: [N][D]; P: [N]; A and TAU_P: [N][DD] (full tensors, row-major). */
int orc_fields(orc *o, int which, double *out) {
  const lattice_t *L = &o->L;
  const int Q = o->Q, D = o->D, DD = o->DD;
  double fB[19], Fi[19], tau_p[9];
  moments_sweep(o);
  for (int z = 0; z < o->n[2]; ++z)
    for (int y = 0; y < o->n[1]; ++y)
      for (int x = 0; x < o->n[0]; ++x) {
        const long s = site_index(o, x, y, z);
        const double *A = &o->A[s * DD];
        const double *u = &o->u[s * 3];
        for (int a = 0; a < D; ++a)
          for (int b = 0; b < D; ++b)
            tau_p[T(D, a, b)] =
                o->eta_p / o->lambda * (A[T(D, a, b)] - (a == b ? 1.0 : 0.0));
        switch (which) {
          case ORC_FIELD_U:
            for (int a = 0; a < D; ++a) out[s * D + a] = u[a];
            break;
          case ORC_FIELD_P: {
            double F[3];
            total_force(o, x, y, z, F);
            fB_site(L, o->tau_f, tau_p, fB);
            if (o->scheme)
              for (int i = 0; i < Q; ++i) fB[i] = 0.0;
            forcing_site(L, o->tau_f, F, u, Fi);
            out[s] = pressure_site(L, o->tau_f, &o->f[s * Q], u, Fi[0], fB[0]);
            break;
          }
          case ORC_FIELD_A:
            for (int ab = 0; ab < DD; ++ab) out[s * DD + ab] = A[ab];
            break;
          case ORC_FIELD_TAU_P:
            for (int ab = 0; ab < DD; ++ab) out[s * DD + ab] = tau_p[ab];
            break;
          default:
            return -1;
        }
      }
  return 0;
}

/* ---------------------------------------------------------------------------
 * High-Wi repair of the conformation (reading R11).  Eigen-decomposition of
 * a symmetric D x D matrix by cyclic Jacobi rotations (each rotation zeroes
 * one off-diagonal entry; sweeps until the off-diagonal part is below 1e-300
 * or 50 sweeps), then A' = V max(Lambda, eps) V^T.
 * ------------------------------------------------------------------------- */
static void sym_eig(int D, const double *A, double *lam, double *V) {
  double a[3][3], v[3][3];
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      a[r][c] = A[T(D, r, c)];
      v[r][c] = r == c ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0;
    for (int r = 0; r < D; ++r)
      for (int c = r + 1; c < D; ++c) off += a[r][c] * a[r][c];
    if (off < 1e-300) break;
    for (int p = 0; p < D; ++p)
      for (int q = p + 1; q < D; ++q) {
        if (a[p][q] == 0.0) continue;
        /* rotation angle: tan(2 theta) = 2 a_pq / (a_qq - a_pp) */
        const double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < D; ++k) {   /* A <- A J (columns p, q) */
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = cs * akp - sn * akq;
          a[k][q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < D; ++k) {   /* A <- J^T A (rows p, q) */
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = cs * apk - sn * aqk;
          a[q][k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < D; ++k) {   /* V <- V J */
          const double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = cs * vkp - sn * vkq;
          v[k][q] = sn * vkp + cs * vkq;
        }
      }
  }
  for (int k = 0; k < D; ++k) {
    lam[k] = a[k][k];
    for (int r = 0; r < D; ++r) V[T(D, r, k)] = v[r][k];   /* column k */
  }
}

/* Every node whose A = sum_i h_i has its smallest eigenvalue below eps (or a
 * non-finite entry: left as it is and counted) gets A' = V max(Lambda, eps)
 * V^T, by adding w_i (A' - A) to each of its stress populations; returns
 * the number of nodes changed. */
long orc_repair(orc *o, double eps) {
  const lattice_t *L = &o->L;
  const int Q = o->Q, D = o->D, DD = o->DD;
  long count = 0;
  for (long s = 0; s < o->N; ++s) {
    double A[9], lam[3], V[9];
    int finite = 1;
    for (int ab = 0; ab < DD; ++ab) {
      double acc = 0.0;
      for (int i = 0; i < Q; ++i) acc += o->h[(s * DD + ab) * Q + i];
      A[ab] = acc;
      finite &= isfinite(acc);
    }
    if (!finite) {
      ++count;
      continue;
    }
    sym_eig(D, A, lam, V);
    double lmin = lam[0];
    for (int k = 1; k < D; ++k) lmin = lam[k] < lmin ? lam[k] : lmin;
    if (lmin >= eps) continue;
    ++count;
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        double An = 0.0;
        for (int k = 0; k < D; ++k)
          An += V[T(D, a, k)] * (lam[k] > eps ? lam[k] : eps) * V[T(D, b, k)];
        const double dA = An - A[T(D, a, b)];
        for (int i = 0; i < Q; ++i) o->h[(s * DD + T(D, a, b)) * Q + i] += L->w[i] * dA;
      }
  }
  return count;
}

/* Raw state access: f [N][Q], h [N][DD][Q], chi_old [N][DD]. */
void orc_get_state(const orc *o, double *f, double *h, double *chi_old,
                   int *first) {
  if (f) memcpy(f, o->f, sizeof(double) * o->N * o->Q);
  if (h) memcpy(h, o->h, sizeof(double) * o->N * o->DD * o->Q);
  if (chi_old) memcpy(chi_old, o->chi_old, sizeof(double) * o->N * o->DD);
  if (first) *first = o->first;
}

void orc_set_state(orc *o, const double *f, const double *h,
                   const double *chi_old, int first, long t) {
  if (f) memcpy(o->f, f, sizeof(double) * o->N * o->Q);
  if (h) memcpy(o->h, h, sizeof(double) * o->N * o->DD * o->Q);
  if (chi_old) memcpy(o->chi_old, chi_old, sizeof(double) * o->N * o->DD);
  o->first = first;
  o->t = t;
}

/* ---------------------------------------------------------------------------
 * Exported per-site building blocks, for the tests.
 * ------------------------------------------------------------------------- */
int orc_lattice(int lattice, int *Q, int *D, int *c, double *w, int *opp) {
  lattice_t L;
  if (lattice_get(lattice, &L) != 0) return -1;
  *Q = L.Q; *D = L.D;
  for (int i = 0; i < L.Q; ++i) {
    for (int a = 0; a < 3; ++a) c[i * 3 + a] = L.c[i][a];
    w[i] = L.w[i];
    opp[i] = L.opp[i];
  }
  return 0;
}

int orc_feq(int lattice, double p, const double *u, double *out) {
  lattice_t L;
  if (lattice_get(lattice, &L) != 0) return -1;
  feq_site(&L, p, u, out);
  return 0;
}

int orc_forcing(int lattice, double tau_f, const double *F, const double *u,
                double *out) {
  lattice_t L;
  if (lattice_get(lattice, &L) != 0) return -1;
  forcing_site(&L, tau_f, F, u, out);
  return 0;
}

/* tau_p: full D x D tensor, row-major. */
int orc_fB(int lattice, double tau_f, const double *tau_p, double *out) {
  lattice_t L;
  if (lattice_get(lattice, &L) != 0) return -1;
  fB_site(&L, tau_f, tau_p, out);
  return 0;
}

/* The printed f^B coefficient matrices themselves (9x4 scaled by -1/72, and
 * 19x13), for the pseudo-inverse check. */
int orc_fB_matrix(int lattice, double *out) {
  if (lattice == ORC_D2Q9) {
    for (int i = 0; i < 9; ++i)
      for (int k = 0; k < 4; ++k) out[i * 4 + k] = FB9[i][k] / 72.0;
    return 0;
  }
  if (lattice == ORC_D3Q19) {
    for (int i = 0; i < 19; ++i)
      for (int k = 0; k < 13; ++k) out[i * 13 + k] = FB19[i][k];
    return 0;
  }
  return -1;
}

double orc_pressure(int lattice, double tau_f, const double *f,
                    const double *u, double F0, double fB0) {
  lattice_t L;
  if (lattice_get(lattice, &L) != 0) return NAN;
  return pressure_site(&L, tau_f, f, u, F0, fB0);
}

void orc_force_at(const orc *o, int x, int y, int z, long t, double *F) {
  force_at(o, x, y, z, t, F);
}
