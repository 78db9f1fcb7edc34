"""Seeded synthetic workloads shaped like the paper's four test flows.

This module holds only problem statements: parameters, initial fields and
instance lists.  It contains none of the lattice Boltzmann arithmetic and is
shared by the tests (for the oracle and the CUDA library alike) and by the
benchmark.  Nothing here touches a GPU.

Lattice units throughout: dx = dt = 1, c_s^2 = 1/3, tau = 3 nu + 1/2.

Array conventions: grids are ``(ny, nx)`` in 2D and ``(nz, ny, nx)`` in 3D
(x fastest); velocity has the space dimension last; the conformation tensor
``A`` is a full ``D x D`` tensor on the last two axes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

D2Q9 = 9
D3Q19 = 19

FORCE_NONE = 0
FORCE_CONST = 1
FORCE_FOUR_ROLL = 2
FORCE_COSINE = 3

TAU_H = 0.501  # Sec. 3: relaxation parameter of the stress LB


def tau_from_nu(nu: float) -> float:
    """Sec. 2.2: tau_f = nu_s / c_s^2 + 1/2 (dt = 1)."""
    return 3.0 * nu + 0.5


def nu_from_tau(tau: float) -> float:
    return (tau - 0.5) / 3.0


@dataclass
class Problem:
    """Everything needed to create and initialise one simulation."""
    name: str
    lattice: int
    nx: int
    ny: int
    nz: int = 1
    tau_s: float = 0.8
    eta_p: float = 0.0
    lam: float = 1.0
    force_kind: int = FORCE_NONE
    F0: tuple = (0.0, 0.0, 0.0)
    k: float = 0.0
    omega: float = 0.0
    walls: int = 0
    u0: np.ndarray | None = None
    p0: np.ndarray | None = None
    A0: np.ndarray | None = None
    meta: dict = field(default_factory=dict)
    # constitutive model: 0 Oldroyd-B (the paper's), 1 Giesekus, 2 linear
    # PTT, 3 exponential PTT; mpar is alpha (Giesekus) or eps (PTT)
    model: int = 0
    mpar: float = 0.0

    @property
    def D(self) -> int:
        return 2 if self.lattice == D2Q9 else 3

    @property
    def shape(self):
        return (self.ny, self.nx) if self.D == 2 else (self.nz, self.ny, self.nx)

    @property
    def sites(self) -> int:
        return self.nx * self.ny * (self.nz if self.D == 3 else 1)

    def oracle_kwargs(self) -> dict:
        return dict(nx=self.nx, ny=self.ny, nz=self.nz, tau_s=self.tau_s,
                    eta_p=self.eta_p, lam=self.lam, force_kind=self.force_kind,
                    F0=self.F0, k=self.k, omega=self.omega, walls=self.walls,
                    model=self.model, mpar=self.mpar)


def _coords(shape):
    return np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")


# ---------------------------------------------------------------------------
# Sec. 3.1: simplified four-roll mill
# ---------------------------------------------------------------------------

def four_roll(n: int = 64, Wi: float = 0.1, beta: float = 0.5, U0: float = 0.01,
              tau_s: float = 0.8, at_rest: bool = True) -> Problem:
    """Periodic n x n box, body force 2 nu_s U0 k^2 (sin kx cos ky, -cos kx sin ky),
    k = 2 pi / n; Wi = lambda U0 k; beta = nu_s / (nu_s + nu_p)."""
    nu_s = nu_from_tau(tau_s)
    nu_p = nu_s * (1.0 - beta) / beta
    k = 2.0 * math.pi / n
    lam = Wi / (U0 * k)
    amp = 2.0 * nu_s * U0 * k * k
    pr = Problem("four_roll", D2Q9, n, n, 1, tau_s, nu_p, lam, FORCE_FOUR_ROLL,
                 (amp, 0.0, 0.0), k, 0.0, 0)
    if not at_rest:
        y, x = _coords((n, n))
        u = np.stack([U0 * np.sin(k * x) * np.cos(k * y),
                      -U0 * np.cos(k * x) * np.sin(k * y)], axis=-1)
        pr.u0 = u
    pr.meta = dict(U0=U0, Wi=Wi, beta=beta, nu_s=nu_s, nu_p=nu_p)
    return pr


# ---------------------------------------------------------------------------
# Sec. 3.2: planar Poiseuille flow
# ---------------------------------------------------------------------------

def poiseuille(L: int = 32, nx: int = 8, Wi: float = 1.0, beta: float = 0.1,
               Re: float = 1.0, tau_s: float = 0.8) -> Problem:
    """Channel of L nodes between halfway-bounce-back walls on y (walls at
    y = 0 and y = L, node j at y = j + 1/2), periodic in x, constant force
    g_x = 8 (nu_s + nu_p) U0 / L^2 (Sec. 3.2), U0 = Re (nu_s + nu_p) / L,
    lambda = Wi L / U0."""
    nu_s = nu_from_tau(tau_s)
    nu_p = nu_s * (1.0 - beta) / beta
    nu = nu_s + nu_p
    U0 = Re * nu / L
    lam = Wi * L / U0
    g = 8.0 * nu * U0 / L ** 2
    pr = Problem("poiseuille", D2Q9, nx, L, 1, tau_s, nu_p, lam, FORCE_CONST,
                 (g, 0.0, 0.0), 0.0, 0.0, 0b10)
    pr.meta = dict(U0=U0, Wi=Wi, beta=beta, nu_s=nu_s, nu_p=nu_p, g=g, L=L)
    return pr


def poiseuille_steady(pr: Problem):
    """Closed-form steady Oldroyd-B channel solution (Sec. 3.2), on the nodes:
    u_x = g y (L - y) / (2 nu), A_xy = lambda u_x', A_yy = 1,
    A_xx = 1 + 2 (lambda u_x')^2.  Returns (u_x[L], A_xx[L], A_xy[L])."""
    m = pr.meta
    L = m["L"]
    nu = m["nu_s"] + m["nu_p"]
    y = np.arange(L) + 0.5
    u = m["g"] / (2.0 * nu) * y * (L - y)
    du = m["g"] / (2.0 * nu) * (L - 2.0 * y)
    return u, 1.0 + 2.0 * (pr.lam * du) ** 2, pr.lam * du


# ---------------------------------------------------------------------------
# Sec. 3.3: Womersley channel
# ---------------------------------------------------------------------------

def womersley(L: int = 64, nx: int = 4, gamma: float = 3.070, beta: float = 0.5,
              Wi: float = 0.5, U: float = 0.01, tau_s: float = 0.8,
              newtonian: bool = False) -> Problem:
    """Channel of L nodes between walls on y, driven by
    g_x = 8 (nu_s + nu_p) U / L^2 cos(omega t), with the Womersley number
    gamma = (L/2) sqrt(omega / nu_s) fixing omega (Sec. 3.3)."""
    nu_s = nu_from_tau(tau_s)
    nu_p = 0.0 if newtonian else nu_s * (1.0 - beta) / beta
    omega = nu_s * (2.0 * gamma / L) ** 2
    lam = Wi * L / U
    amp = 8.0 * (nu_s + nu_p) * U / L ** 2
    pr = Problem("womersley", D2Q9, nx, L, 1, tau_s, nu_p, lam, FORCE_COSINE,
                 (amp, 0.0, 0.0), 0.0, omega, 0b10)
    pr.meta = dict(U=U, Wi=Wi, beta=beta, nu_s=nu_s, nu_p=nu_p, gamma=gamma,
                   period=2.0 * math.pi / omega, L=L, amp=amp)
    return pr


# ---------------------------------------------------------------------------
# Sec. 3.4: three-dimensional Taylor-Green vortex
# ---------------------------------------------------------------------------

def taylor_green_3d(n: int = 128, U0: float = 0.02, Re: float = 100.0,
                    Wi: float = 1.0, beta: float = 0.5, theta: float = math.pi / 2,
                    length: str = "2pi", fields: bool = True, out_u=None,
                    out_p=None) -> Problem:
    """Periodic n^3 box, initial velocity and pressure of Sec. 3.4 (theta =
    pi/2), zero initial polymer stress.  The characteristic length is
    L = n / (2 pi) (the box spans 2 pi) or L = n; nu = U0 L / Re, lambda =
    Wi L / U0, nu_s = beta nu.

    The fields are formed one z-plane at a time from per-axis sine and cosine
    tables, so building them holds nothing beyond the outputs (u: n^3 x 3,
    p: n^3 doubles).  ``out_u`` / ``out_p`` (C-contiguous float64 arrays of
    those shapes, e.g. page-locked host buffers) receive them in place;
    ``fields=False`` leaves u0 and p0 unset."""
    L = n / (2.0 * math.pi) if length == "2pi" else float(n)
    nu = U0 * L / Re
    nu_s = beta * nu
    nu_p = nu - nu_s
    tau_s = tau_from_nu(nu_s)
    lam = Wi * L / U0
    pr = Problem("taylor_green_3d", D3Q19, n, n, n, tau_s, nu_p, lam,
                 FORCE_NONE, (0.0, 0.0, 0.0), 0.0, 0.0, 0)
    pr.meta = dict(U0=U0, Re=Re, Wi=Wi, beta=beta, nu_s=nu_s, nu_p=nu_p, L=L)
    if fields:
        pr.u0, pr.p0 = taylor_green_3d_fields(n, U0, theta, out_u, out_p)
    return pr


def taylor_green_3d_fields(n: int, U0: float = 0.02, theta: float = math.pi / 2,
                           out_u=None, out_p=None):
    """Initial velocity and pressure of the Sec. 3.4 vortex on the n^3 nodes
    (x = k i, k = 2 pi / n): u = (2 U0 / sqrt 3) [sin(theta + 2 pi/3) sin x cos y cos z,
    sin(theta - 2 pi/3) cos x sin y cos z, sin(theta) cos x cos y sin z] and the
    pressure that balances it.  Returns (u [n, n, n, 3], p [n, n, n])."""
    k = 2.0 * math.pi / n
    t = k * np.arange(n, dtype=np.float64)
    s1, c1 = np.sin(t), np.cos(t)
    c2 = np.cos(2 * t)
    a = 2.0 * U0 / math.sqrt(3.0)
    ax = a * math.sin(theta + 2.0 * math.pi / 3.0)
    ay = a * math.sin(theta - 2.0 * math.pi / 3.0)
    az = a * math.sin(theta)
    u = np.empty((n, n, n, 3)) if out_u is None else out_u
    p = np.empty((n, n, n)) if out_p is None else out_p
    if u.shape != (n, n, n, 3) or p.shape != (n, n, n):
        raise ValueError("out_u / out_p have the wrong shape")
    X, Y = s1[None, :], s1[:, None]          # sin over x (last axis) and y
    CX, CY = c1[None, :], c1[:, None]
    C2X, C2Y = c2[None, :], c2[:, None]
    for iz in range(n):
        sz, cz, c2z = s1[iz], c1[iz], c2[iz]
        u[iz, :, :, 0] = ax * X * CY * cz
        u[iz, :, :, 1] = ay * CX * Y * cz
        u[iz, :, :, 2] = az * CX * CY * sz
        p[iz] = U0 ** 2 * ((C2X * C2Y + 2 * c2z) / 12.0
                           + (C2X * c2z + 2 * C2Y) / 48.0
                           + (C2Y * c2z + 2 * C2X) / 48.0)
    return u, p


def taylor_green_2d(n: int = 64, U0: float = 0.01, tau_s: float = 0.8,
                    eta_p: float = 0.0, lam: float = 1.0) -> Problem:
    """Periodic 2D Taylor-Green vortex u = U0 (sin kx cos ky, -cos kx sin ky),
    p = U0^2/4 (cos 2kx + cos 2ky), k = 2 pi / n: an exact Navier-Stokes
    solution decaying as exp(-2 nu k^2 t)."""
    k = 2.0 * math.pi / n
    y, x = _coords((n, n))
    u = np.stack([U0 * np.sin(k * x) * np.cos(k * y),
                  -U0 * np.cos(k * x) * np.sin(k * y)], axis=-1)
    p = 0.25 * U0 ** 2 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    pr = Problem("taylor_green_2d", D2Q9, n, n, 1, tau_s, eta_p, lam)
    pr.u0, pr.p0 = u, p
    pr.meta = dict(U0=U0, k=k, nu_s=nu_from_tau(tau_s))
    return pr


# ---------------------------------------------------------------------------
# Random smooth states for parity and invariant tests
# ---------------------------------------------------------------------------

def random_smooth(lattice: int, shape, seed: int = 0, U: float = 0.02,
                  dA: float = 0.3, modes: int = 3):
    """A few random Fourier modes (periodic on the grid) for u, p and a
    symmetric positive-definite A = I + small symmetric perturbation."""
    rng = np.random.default_rng(seed)
    D = 2 if lattice == D2Q9 else 3
    grids = _coords(shape)
    ks = [2.0 * math.pi / n for n in shape]

    def field_():
        out = np.zeros(shape)
        for _ in range(modes):
            ph = rng.uniform(0, 2 * math.pi)
            amp = rng.normal()
            arg = ph
            for g, kk in zip(grids, ks):
                arg = arg + rng.integers(-2, 3) * kk * g
            out += amp * np.cos(arg)
        return out / modes

    u = np.stack([U * field_() for _ in range(D)], axis=-1)
    p = 0.5 * U * U * field_()
    A = np.zeros(shape + (D, D))
    for a in range(D):
        A[..., a, a] = 1.0 + dA * np.abs(field_())
        for b in range(a + 1, D):
            v = 0.3 * dA * field_()
            A[..., a, b] = v
            A[..., b, a] = v
    return u, p, A


# ---------------------------------------------------------------------------
# Batched instances: uneven D2Q9 grids, mixed four-roll and Poiseuille
# ---------------------------------------------------------------------------

def batch_instances(count: int = 512, seed: int = 0, nmin: int = 32,
                    nmax: int = 512, U0: float = 0.01, tau_s: float = 0.8):
    """Square n x n D2Q9 instances, n log-uniform in [nmin, nmax], a fair coin
    between four-roll (periodic) and Poiseuille (walls on y), Wi ~ U[0.1, 2],
    beta ~ U[0.1, 0.9]."""
    rng = np.random.default_rng(seed)
    out = []
    nu_s = nu_from_tau(tau_s)
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        Wi = float(rng.uniform(0.1, 2.0))
        beta = float(rng.uniform(0.1, 0.9))
        if rng.random() < 0.5:
            pr = four_roll(n=n, Wi=Wi, beta=beta, U0=U0, tau_s=tau_s)
        else:
            nu_p = nu_s * (1.0 - beta) / beta
            nu = nu_s + nu_p
            lam = Wi * n / U0
            g = 8.0 * nu * U0 / n ** 2
            pr = Problem("poiseuille", D2Q9, n, n, 1, tau_s, nu_p, lam, FORCE_CONST,
                         (g, 0.0, 0.0), 0.0, 0.0, 0b10)
            pr.meta = dict(U0=U0, Wi=Wi, beta=beta, nu_s=nu_s, nu_p=nu_p, g=g, L=n)
        out.append(pr)
    return out
