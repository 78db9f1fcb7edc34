"""Pins of the FP64 oracle's time stepping against closed forms and invariants
that the paper and the continuum equations fix (Sec. 2.1-2.3, Sec. 3)."""
import cmath
import math

import numpy as np
import pytest

import oracle as O
from paper_2506_13072_gb300 import workloads as W


def make(pr, tau_h=None):
    o = O.Oracle(pr.lattice, tau_h=tau_h, **pr.oracle_kwargs())
    o.init(u=pr.u0, p=pr.p0, A=pr.A0)
    return o


# ---------------------------------------------------------------------------
# Conservation (Sec. 2.2 moment conditions; f^B carries no mass or momentum)
# ---------------------------------------------------------------------------

def _momentum(o):
    f, _, _, _ = o.get_state()
    c, _, _ = O.lattice(o.lat)
    return f.sum(axis=0), f @ c[:, : o.D].astype(float)


def test_mass_and_momentum_periodic_four_roll():
    """Periodic box: sum_i f stays 0 (sum f^eq = 0 and the initial state is an
    equilibrium) and the population momentum grows by sum_x F each step, which
    is 0 for the four-roll force on a whole number of periods."""
    pr = W.four_roll(n=16, Wi=0.5, beta=0.5)
    u, p, A = W.random_smooth(O.D2Q9, pr.shape, seed=7)
    pr.u0, pr.p0, pr.A0 = u, p, A
    o = make(pr)
    m0, P0 = _momentum(o)
    assert abs(m0.sum()) < 1e-15
    for _ in range(5):
        o.step(40)
        m, P = _momentum(o)
        assert abs(m.sum()) < 1e-13
        assert np.abs(P.sum(axis=0) - P0.sum(axis=0)).max() < 1e-15


def test_momentum_grows_by_force_3d():
    """D3Q19, constant force, periodic: total momentum after n steps is
    P0 + n N F exactly (up to rounding)."""
    pr = W.Problem("c", W.D3Q19, 6, 5, 4, 0.9, 0.05, 40.0, W.FORCE_CONST, (1e-5, -2e-5, 3e-5))
    u, p, A = W.random_smooth(O.D3Q19, pr.shape, seed=8)
    pr.u0, pr.p0, pr.A0 = u, p, A
    o = make(pr)
    _, P0 = _momentum(o)
    o.step(30)
    m, P = _momentum(o)
    assert abs(m.sum()) < 1e-13
    want = P0.sum(axis=0) + 30 * pr.sites * np.array(pr.F0)
    assert np.abs(P.sum(axis=0) - want).max() < 1e-14


def test_conformation_stays_symmetric():
    pr = W.four_roll(n=12, Wi=0.5, beta=0.5)
    u, p, A = W.random_smooth(O.D2Q9, pr.shape, seed=9)
    pr.u0, pr.p0, pr.A0 = u, p, A
    o = make(pr)
    o.step(100)
    A = o.A()
    assert np.abs(A[..., 0, 1] - A[..., 1, 0]).max() < 1e-14
    pr3 = W.Problem("s", W.D3Q19, 5, 4, 6, 0.8, 0.1, 20.0)
    pr3.u0, pr3.p0, pr3.A0 = W.random_smooth(O.D3Q19, pr3.shape, seed=10)
    o3 = make(pr3)
    o3.step(40)
    A3 = o3.A()
    assert np.abs(A3 - np.swapaxes(A3, -1, -2)).max() < 1e-14


# ---------------------------------------------------------------------------
# Uniform relaxation: the stress LB reduces to Adams-Bashforth 2 (Sec. 2.3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_uniform_relaxation_is_ab2(lat):
    """With u = 0 and uniform A, summing the h evolution over i gives
    A^{n+1} = A^n + chi^n + (chi^n - chi^{n-1})/2 with chi = -(A - I)/lambda:
    the two-step Adams-Bashforth rule (first step Euler) for
    dA/dt = -(A - I)/lambda."""
    D = 2 if lat == O.D2Q9 else 3
    lam = 7.0
    A0 = np.eye(D) + np.array([[0.6, 0.2, 0.1], [0.2, -0.3, 0.05], [0.1, 0.05, 0.4]])[:D, :D]
    shape = (3, 2) if D == 2 else (2, 3, 2)
    o = O.Oracle(lat, shape[-1], shape[-2], 1 if D == 2 else shape[0], tau_s=0.7,
                 eta_p=0.3, lam=lam)
    o.init(A=np.broadcast_to(A0, shape + (D, D)))
    e_prev = A0 - np.eye(D)
    e = e_prev - e_prev / lam   # Euler first step
    o.step(1)
    assert np.abs(o.A() - (np.eye(D) + e)).max() < 1e-14
    assert np.abs(o.u()).max() < 1e-16
    for _ in range(30):
        e, e_prev = e - 1.5 * e / lam + 0.5 * e_prev / lam, e
        o.step(1)
        assert np.abs(o.A() - (np.eye(D) + e)).max() < 1e-13
    # and AB2 tracks the exact exponential to O(dt^2 / lambda^2)
    assert np.abs(e - (A0 - np.eye(D)) * math.exp(-31 / lam)).max() < 5e-3


# ---------------------------------------------------------------------------
# Newtonian limit: 2D Taylor-Green vortex decays as exp(-2 nu k^2 t)
# ---------------------------------------------------------------------------

def _tg_rate_error(n):
    pr = W.taylor_green_2d(n=n, U0=0.01, tau_s=0.8)
    o = make(pr)
    u0 = o.u()
    T = int(400 * (n / 64) ** 2)
    o.step(T)
    u = o.u()
    ratio = (u * u0).sum() / (u0 * u0).sum()
    rate = -math.log(ratio) / T
    # the shape is preserved (an exact Navier-Stokes solution)
    assert np.abs(u - ratio * u0).max() < 1e-4 * pr.meta["U0"]
    return rate / (2.0 * pr.meta["nu_s"] * pr.meta["k"] ** 2) - 1.0


def test_taylor_green_newtonian_decay():
    """Decay rate 2 nu k^2 with nu = (tau - 1/2)/3 (Sec. 2.2), to second
    order in the lattice spacing."""
    e32, e64 = _tg_rate_error(32), _tg_rate_error(64)
    assert abs(e64) < 2e-3
    assert math.log2(abs(e32 / e64)) > 1.9


# ---------------------------------------------------------------------------
# Linear viscoelastic shear wave (Oldroyd-B linearised about rest)
# ---------------------------------------------------------------------------

def _shear_wave_amplitude(t, U0, K, nu_s, eta_p, lam):
    """u_x = U(t) sin(K y), tau_xy = S(t) cos(K y):
    U' = -nu_s K^2 U - K S,  S' = -S / lambda + eta_p K U / lambda,
    U(0) = U0, S(0) = 0.  Roots of lambda s^2 + (1 + lambda nu_s K^2) s
    + (nu_s + eta_p) K^2 = 0."""
    a, b, c = lam, 1.0 + lam * nu_s * K * K, (nu_s + eta_p) * K * K
    disc = cmath.sqrt(b * b - 4 * a * c)
    s1, s2 = (-b + disc) / (2 * a), (-b - disc) / (2 * a)
    d0 = -nu_s * K * K * U0
    c1 = (d0 - s2 * U0) / (s1 - s2)
    c2 = U0 - c1
    return (c1 * cmath.exp(s1 * t) + c2 * cmath.exp(s2 * t)).real


@pytest.mark.parametrize("lam", [50.0, 400.0])
def test_viscoelastic_shear_wave(lam):
    n, U0, tau = 64, 1e-4, 0.8
    nu_s = W.nu_from_tau(tau)
    eta_p = 0.15
    K = 2 * math.pi / n
    pr = W.Problem("sw", W.D2Q9, 1, n, 1, tau, eta_p, lam)
    y = np.arange(n, dtype=float)
    pr.u0 = np.stack([U0 * np.sin(K * y), 0 * y], -1)[:, None, :]
    o = make(pr)
    errs = []
    for k in range(8):
        o.step(250)
        ux = o.u()[:, 0, 0]
        Ut = 2.0 / n * (ux * np.sin(K * y)).sum()
        want = _shear_wave_amplitude(o.t, U0, K, nu_s, eta_p, lam)
        errs.append(abs(Ut - want))
    assert max(errs) < 1e-2 * U0
    # a wrong sign of the polymer coupling would show as growth
    assert abs(Ut) < U0


# ---------------------------------------------------------------------------
# Planar Poiseuille flow (Sec. 3.2)
# ---------------------------------------------------------------------------

def _poiseuille_run(L, Wi=1.0, beta=0.1, newtonian=False, nl=12):
    pr = W.poiseuille(L=L, nx=1, Wi=Wi, beta=beta)
    if newtonian:
        pr.eta_p = 0.0
        pr.meta["nu_p"] = 0.0
        pr.F0 = (8.0 * pr.meta["nu_s"] * pr.meta["U0"] / L ** 2, 0.0, 0.0)
        pr.meta["g"] = pr.F0[0]
    ua, Axx, Axy = W.poiseuille_steady(pr)
    # start from the closed form so that only the discretisation error remains
    pr.u0 = np.stack([ua, 0 * ua], -1)[:, None, :]
    A = np.zeros((L, 1, 2, 2))
    A[:, 0, 0, 0], A[:, 0, 0, 1], A[:, 0, 1, 0], A[:, 0, 1, 1] = Axx, Axy, Axy, 1.0
    pr.A0 = A
    o = make(pr)
    o.step(int(nl * pr.lam) if not newtonian else 20 * L * L)
    u = o.u()[:, 0, 0]
    Am = o.A()[:, 0]

    def gre(a, b):  # Sec. 3.2, global relative error
        return np.abs(a - b).sum() / np.abs(b).sum()

    return gre(u, ua), gre(Am[:, 0, 1], Axy), gre(Am[:, 0, 0], Axx), np.abs(Am[:, 1, 1] - 1).max()


def test_poiseuille_newtonian_second_order():
    e16 = _poiseuille_run(16, newtonian=True)[0]
    e32 = _poiseuille_run(32, newtonian=True)[0]
    assert e32 < 1e-3
    assert math.log2(e16 / e32) > 1.95


def test_poiseuille_oldroyd_b_steady():
    """Steady u_x, A_xy = lambda u', A_xx = 1 + 2 (lambda u')^2, A_yy = 1
    (Sec. 3.2, with the A_xx numerator read as in the reading list)."""
    gu, gxy, gxx, yy = _poiseuille_run(32, Wi=1.0, beta=0.1)
    assert gu < 4e-3
    assert gxy < 1.5e-3
    assert gxx < 1.5e-2
    assert yy < 1e-5


def _waters_king_centre(t_star, El, beta, terms=400):
    """Sec. 3.2 transient series at y* = 1/2 (Waters and King)."""
    s = 0.0
    for n in range(1, terms + 1):
        N = (2 * n - 1) * math.pi
        S = 1.0 - (2.0 - beta) * N * N * El
        a = 1.0 + beta * El * N * N
        b2 = a * a - 4.0 * N * N * El
        if b2 >= 0:
            b = math.sqrt(b2)
            aN, bN = 1 + S / b, 1 - S / b
            p, q = (-a + b) / (2 * El), (-a - b) / (2 * El)
            G = 0.5 * (aN * math.exp(p * t_star) + bN * math.exp(q * t_star))
        else:
            b = math.sqrt(-b2)
            G = math.exp(-a / (2 * El) * t_star) * (math.cos(b / (2 * El) * t_star)
                                                    + S / b * math.sin(b / (2 * El) * t_star))
        s += math.sin(N * 0.5) / N ** 3 * G
    return 1.0 - 32.0 * s


def test_poiseuille_transient_waters_king():
    """Start-up from rest, Re = 1, Wi = 1, beta = 0.1: centre-line velocity
    against the series of Sec. 3.2 (t* = t nu / L^2 = t U0 / L at Re = 1)."""
    L = 32
    pr = W.poiseuille(L=L, nx=1, Wi=1.0, beta=0.1)
    o = make(pr)
    U0 = pr.meta["U0"]
    El = pr.meta["Wi"] / 1.0
    nu = pr.meta["nu_s"] + pr.meta["nu_p"]
    worst = 0.0
    for _ in range(20):
        o.step(128)
        u = o.u()[:, 0, 0]
        uc = 0.5 * (u[L // 2 - 1] + u[L // 2])
        want = _waters_king_centre(o.t * nu / L ** 2, El, 0.1)
        worst = max(worst, abs(uc / U0 - want))
    assert worst < 2e-2


# ---------------------------------------------------------------------------
# Womersley flow (Sec. 3.3)
# ---------------------------------------------------------------------------

def _womersley_profile(y_nodes, L, amp, omega, nu, t):
    """Re{ A/(i omega) [1 - cosh(kappa (2y/L - 1)) / cosh(kappa)] e^{i omega t} }
    with kappa^2 = i omega (L/2)^2 / nu (Sec. 3.3; nu may be complex)."""
    kappa = cmath.sqrt(1j * omega * (L / 2) ** 2 / nu)
    out = []
    for y in y_nodes:
        eta = 2.0 * y / L - 1.0
        v = amp / (1j * omega) * (1 - cmath.cosh(kappa * eta) / cmath.cosh(kappa)) \
            * cmath.exp(1j * omega * t)
        out.append(v.real)
    return np.array(out)


@pytest.mark.parametrize("newtonian,Wi,tol", [(True, 0.0, 1e-2), (False, 0.5, 2e-2),
                                              (False, 2.0, 2e-2)])
def test_womersley(newtonian, Wi, tol):
    """Newtonian: the closed form of Sec. 3.3.  Oldroyd-B: the flow is
    unidirectional, so the momentum equation stays linear and the same
    closed form holds with the complex viscosity nu_s + nu_p / (1 + i omega
    lambda)."""
    L = 64
    pr = W.womersley(L=L, nx=1, gamma=3.070, beta=0.5, Wi=max(Wi, 1e-3), newtonian=newtonian)
    o = make(pr)
    T = pr.meta["period"]
    nu = pr.meta["nu_s"] if newtonian else \
        pr.meta["nu_s"] + pr.meta["nu_p"] / (1 + 1j * pr.omega * pr.lam)
    settle = 3 if newtonian else max(3, int(math.ceil(8 * pr.lam / T)))
    o.step(int(settle * T))
    y = np.arange(L) + 0.5
    amp = pr.meta["amp"]
    scale = np.abs(_womersley_profile(y, L, amp, pr.omega, nu, 0.0)).max()
    worst = 0.0
    for k in range(8):
        o.step(int(T / 8))
        u = o.u()[:, 0, 0]
        # u is reported with the half-force shift at the step's own time
        want = _womersley_profile(y, L, amp, pr.omega, nu, o.t)
        worst = max(worst, np.abs(u - want).max() / scale)
    assert worst < tol


# ---------------------------------------------------------------------------
# Four-roll mill, low-Wi limit (Sec. 3.1)
# ---------------------------------------------------------------------------

def test_four_roll_low_wi_amplitude():
    """As Wi -> 0 the polymer acts as extra viscosity; the forced cellular
    flow then has amplitude 2 nu_s U0 k^2 / (2 (nu_s + nu_p) k^2) = beta U0."""
    pr = W.four_roll(n=32, Wi=0.01, beta=0.5, U0=0.01)
    o = make(pr)
    o.step(3000)
    u = o.u()
    k = pr.k
    y, x = np.meshgrid(np.arange(32.0), np.arange(32.0), indexing="ij")
    shape = np.sin(k * x) * np.cos(k * y)
    amp = (u[..., 0] * shape).sum() / (shape * shape).sum()
    assert amp == pytest.approx(0.5 * 0.01, rel=1e-2)
