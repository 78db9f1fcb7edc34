"""Pins of the oracle's other constitutive models (reading R9 in the oracle's
header; the paper names Giesekus and Phan-Thien-Tanner in Sec. 1 and leaves
them to future work in Sec. 4).  Only the relaxation part P(A) of the stress
source chi of Sec. 2.3 changes, so each pin fixes P through a state whose
evolution has a closed form:

* zero model parameter: the Oldroyd-B step, bit for bit;
* a uniform conformation at rest relaxes by an ODE with a closed-form
  solution (logistic for Giesekus and linear PTT, the exponential integral
  for exponential PTT), which the stress LB follows to second order in
  dt / lambda (the d(chi)/dt term makes the update Adams-Bashforth 2);
* steady channel flow: the textbook steady-shear solutions (Giesekus's
  viscosity and normal-stress functions; the PTT cubic with a Newtonian
  solvent) integrated across the channel.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import brentq
from scipy.special import expi

import oracle as O
from paper_2506_13072_gb300 import workloads as W

GIE, PTTL, PTTE = O.MODEL_GIESEKUS, O.MODEL_PTT_LINEAR, O.MODEL_PTT_EXP


def _oracle(pr, **kw):
    o = O.Oracle(pr.lattice, **{**pr.oracle_kwargs(), **kw})
    o.init(u=pr.u0, p=pr.p0, A=pr.A0)
    return o


# ---------------------------------------------------------------------------
# zero parameter: Oldroyd-B
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("model", [GIE, PTTL, PTTE])
@pytest.mark.parametrize("lat", [W.D2Q9, W.D3Q19])
def test_zero_parameter_is_oldroyd_b(model, lat):
    if lat == W.D2Q9:
        pr = W.four_roll(n=12, Wi=0.5, beta=0.5)
    else:
        pr = W.taylor_green_3d(n=6, Wi=0.5, beta=0.5)
    pr.u0, pr.p0, pr.A0 = W.random_smooth(pr.lattice, pr.shape, seed=5, U=0.03, dA=0.4)
    a = _oracle(pr)
    b = _oracle(pr, model=model, mpar=0.0)
    a.step(20)
    b.step(20)
    for x, y in zip(a.get_state()[:3], b.get_state()[:3]):
        assert np.array_equal(x, y)


def test_model_validation():
    pr = W.four_roll(n=8)
    with pytest.raises(ValueError):
        O.Oracle(pr.lattice, **{**pr.oracle_kwargs(), "model": 4})
    with pytest.raises(ValueError):
        O.Oracle(pr.lattice, **{**pr.oracle_kwargs(), "model": GIE, "mpar": -0.1})


# ---------------------------------------------------------------------------
# uniform relaxation at rest: dM/dt = -P(M)/lambda, M = A - I
# ---------------------------------------------------------------------------

def _logistic(y0, a, s):
    """y' = -(y + a y^2) in s = t / lambda."""
    e = math.exp(-s)
    return y0 * e / (1.0 + a * y0 * (1.0 - e))


def _exact_relaxation(model, par, M0, s):
    if model == GIE:
        # M, M.M commute: every eigenvalue follows the logistic law
        mu, V = np.linalg.eigh(M0)
        return (V * np.array([_logistic(m, par, s) for m in mu])) @ V.T
    T = np.trace(M0)
    if model == PTTL:
        # M = c M0 with c' = -(1 + par T c) c, c(0) = 1
        return _logistic(1.0, par * T, s) * M0
    # exponential PTT: c' = -exp(k c) c, k = par T, so that
    # Ei(-k c) - Ei(-k) = -s (d/dc Ei(-k c) = exp(-k c) / c)
    k = par * T
    c = brentq(lambda c: expi(-k * c) - expi(-k) + s, 1e-12, 1.0, xtol=1e-15, rtol=1e-15)
    return c * M0


def _uniform_run(lat, model, par, M0, lam, steps):
    D = 2 if lat == W.D2Q9 else 3
    n = (4, 4, 1) if D == 2 else (3, 3, 3)
    o = O.Oracle(lat, n[0], n[1], n[2], tau_s=0.8, eta_p=0.05, lam=lam,
                 model=model, mpar=par)
    shape = o.shape
    o.init(A=np.broadcast_to(np.eye(D) + M0, shape + (D, D)).copy())
    o.step(steps)
    A = o.A().reshape(-1, D, D)
    assert np.abs(A - A[0]).max() < 1e-13           # stays uniform
    return A[0] - np.eye(D)


M2 = np.array([[0.6, 0.3], [0.3, -0.2]])
M3 = np.array([[0.5, 0.2, -0.1], [0.2, -0.3, 0.15], [-0.1, 0.15, 0.4]])


@pytest.mark.parametrize("model,par", [(GIE, 0.3), (PTTL, 0.4), (PTTE, 0.4)])
@pytest.mark.parametrize("lat", [W.D2Q9, W.D3Q19])
def test_uniform_relaxation_closed_form(lat, model, par):
    M0 = M2 if lat == W.D2Q9 else M3
    lam, steps = 200.0, 400
    got = _uniform_run(lat, model, par, M0, lam, steps)
    want = _exact_relaxation(model, par, M0, steps / lam)
    # second order in dt / lambda: the error is ~(dt/lambda)^2 |M0|
    err = np.abs(got - want).max()
    assert err < 1e-5 * np.abs(M0).max(), err
    # and the Oldroyd-B law (P = M) is far from it
    ob = math.exp(-steps / lam) * M0
    assert np.abs(ob - want).max() > 50 * err


@pytest.mark.parametrize("model,par", [(GIE, 0.3), (PTTL, 0.4), (PTTE, 0.4)])
def test_uniform_relaxation_second_order(model, par):
    """Halving dt / lambda divides the error by 4."""
    errs = []
    for lam in (100.0, 200.0):
        steps = int(2 * lam)
        got = _uniform_run(W.D2Q9, model, par, M2, lam, steps)
        errs.append(np.abs(got - _exact_relaxation(model, par, M2, 2.0)).max())
    assert 3.6 < errs[0] / errs[1] < 4.4, errs


# ---------------------------------------------------------------------------
# steady channel flow
# ---------------------------------------------------------------------------

def _giesekus_shear(al, Wi):
    """Steady simple shear of the Giesekus model at Wi = lambda du/dy > 0:
    (eta_p / eta_p0, M_xy, M_xx, M_yy) from the textbook closed form
    (Giesekus 1982; Bird, Armstrong, Hassager): with
    Lambda^2 = (sqrt(1 + 16 al (1 - al) Wi^2) - 1) / (8 al (1 - al) Wi^2) and
    f = (1 - Lambda) / (1 + (1 - 2 al) Lambda),
    eta_p / eta_p0 = (1 - f)^2 / (1 + (1 - 2 al) f),
    Psi_1 / (2 eta_p0 lambda) = f (1 - al f) / (al Wi^2 (1 - f)),
    Psi_2 / (eta_p0 lambda) = -f / Wi^2."""
    if Wi < 1e-6:
        return 1.0, Wi, 2.0 * Wi * Wi, 0.0
    q = 8.0 * al * (1.0 - al) * Wi * Wi
    Lm = math.sqrt((math.sqrt(1.0 + 2.0 * q) - 1.0) / q)
    f = (1.0 - Lm) / (1.0 + (1.0 - 2.0 * al) * Lm)
    eta = (1.0 - f) ** 2 / (1.0 + (1.0 - 2.0 * al) * f)
    n1 = 2.0 * f * (1.0 - al * f) / (al * (1.0 - f))   # lambda N1 / eta_p0
    myy = -f                                             # lambda N2 / eta_p0
    return eta, eta * Wi, n1 + myy, myy


def _ptt_shear_a(model, eps, lam_sigma, eta_s, eta_p):
    """Steady simple shear of PTT (no slip parameter) under total shear
    stress sigma: M_yy = 0, M_xx = 2 a^2 with a = M_xy, and
    lambda sigma = eta_s f a + eta_p a, f = 1 + eps M_xx (linear) or
    exp(eps M_xx); lambda du/dy = f a."""
    def f_of(a):
        return 1.0 + 2.0 * eps * a * a if model == PTTL else math.exp(2.0 * eps * a * a)
    if model == PTTL:
        # 2 eps eta_s a^3 + (eta_s + eta_p) a - lambda sigma = 0 (one real root)
        r = np.roots([2.0 * eps * eta_s, 0.0, eta_s + eta_p, -lam_sigma])
        a = float(r[np.argmin(np.abs(r.imag))].real)
    else:
        hi = abs(lam_sigma) / eta_p + 1.0
        a = brentq(lambda a: eta_s * f_of(a) * a + eta_p * a - lam_sigma, -hi, hi,
                   xtol=1e-15, rtol=1e-15)
    return a, f_of(a)


def _channel_exact(pr, model, par):
    """u_x, M_xx, M_xy, M_yy on the nodes y = j + 1/2 of the channel
    [0, L] under the body force g (total shear stress g (L/2 - y))."""
    m = pr.meta
    L, g, lam = m["L"], m["g"], pr.lam
    eta_s, eta_p = m["nu_s"], pr.eta_p

    def local(y):
        sig = g * (L / 2.0 - y)
        if model == GIE:
            # sigma = eta_s gd + eta_p0 gd eta(lambda gd): monotone in gd
            s = abs(sig)
            hi = s / eta_s * 1.01 + 1e-300
            gd = brentq(lambda gd: eta_s * gd + eta_p * gd * _giesekus_shear(par, lam * gd)[0] - s,
                        0.0, hi, xtol=1e-18, rtol=1e-15) if s > 0 else 0.0
            _, mxy, mxx, myy = _giesekus_shear(par, lam * gd)
            sgn = 1.0 if sig >= 0 else -1.0
            return sgn * gd, mxx, sgn * mxy, myy
        a, f = _ptt_shear_a(model, par, lam * sig, eta_s, eta_p)
        return f * a / lam, 2.0 * a * a, a, 0.0

    y = np.arange(L) + 0.5
    u = np.array([quad(lambda t: local(t)[0], 0.0, yy, epsabs=1e-16, epsrel=1e-12)[0]
                  for yy in y])
    M = np.array([local(yy)[1:] for yy in y])
    return u, M[:, 0], M[:, 1], M[:, 2]


def _channel_run(model, par, L=32, Wi=1.0, beta=0.1, nl=12):
    pr = W.poiseuille(L=L, nx=1, Wi=Wi, beta=beta)
    pr.model, pr.mpar = model, par
    u, mxx, mxy, myy = _channel_exact(pr, model, par)
    # start from the closed form so that only the discretisation error remains
    pr.u0 = np.stack([u, 0 * u], -1)[:, None, :]
    A = np.zeros((L, 1, 2, 2))
    A[:, 0, 0, 0], A[:, 0, 0, 1], A[:, 0, 1, 0], A[:, 0, 1, 1] = 1 + mxx, mxy, mxy, 1 + myy
    pr.A0 = A
    o = _oracle(pr)
    o.step(int(nl * pr.lam))
    Am = o.A()[:, 0] - np.eye(2)

    def gre(a, b):  # Sec. 3.2, global relative error
        return np.abs(a - b).sum() / np.abs(b).sum()

    return (gre(o.u()[:, 0, 0], u), gre(Am[:, 0, 1], mxy), gre(Am[:, 0, 0], mxx),
            np.abs(Am[:, 1, 1] - myy).max() / np.abs(mxx).max(), (u, mxx, mxy, myy))


@pytest.mark.parametrize("model,par", [(GIE, 0.2), (PTTL, 0.25), (PTTE, 0.25)])
def test_channel_steady_closed_form(model, par):
    gu, gxy, gxx, yy, exact = _channel_run(model, par)
    assert gu < 4e-3, gu
    assert gxy < 3e-3, gxy
    assert gxx < 2e-2, gxx
    assert yy < 2e-3, yy
    # the model matters here: Oldroyd-B's closed form is far from it
    pr = W.poiseuille(L=32, nx=1, Wi=1.0, beta=0.1)
    uob = W.poiseuille_steady(pr)[0]
    assert np.abs(uob - exact[0]).sum() / np.abs(exact[0]).sum() > 10 * gu


def test_giesekus_closed_form_limits():
    """The Giesekus shear functions reduce to Oldroyd-B (eta = eta_p0,
    M_xy = Wi, M_xx = 2 Wi^2, M_yy = 0) as alpha -> 0."""
    for Wi in (0.2, 1.0, 3.0):
        eta, mxy, mxx, myy = _giesekus_shear(1e-5, Wi)
        assert abs(eta - 1) < 1e-3 and abs(mxy - Wi) < 1e-3 * Wi
        assert abs(mxx - 2 * Wi * Wi) < 1e-3 * Wi * Wi and abs(myy) < 1e-3
