"""Pins of the oracle's "original" scheme, the one the paper compares its
method with (Sec. 1 and Tables 1-2): the polymer stress divergence enters the
momentum equation as a body force evaluated by finite differences, with no
fluctuation term f^B (reading R8 in the oracle's header).

Each pin holds for the scheme independently of the oracle's code: an
independent numpy step (brute force, tiny grids), the Newtonian limit in
which both schemes are the same LB, global momentum (a central-difference
divergence sums to zero on a periodic grid), and the steady Poiseuille
closed form of Sec. 3.2, which both schemes must reach."""
import numpy as np

import oracle as O
from paper_2506_13072_gb300 import workloads as W

from test_oracle_bruteforce import _compare
from test_oracle_physics import _momentum

ORIG = O.SCHEME_ORIGINAL


def test_original_bruteforce_d2q9_walls():
    pr = W.Problem("bf", W.D2Q9, 8, 7, 1, 0.8, 0.2, 15.0, W.FORCE_CONST, (2e-5, -1e-5, 0.0),
                   walls=0b10)
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D2Q9, pr.shape, seed=21, U=0.03, dA=0.5)
    _compare(pr, 25, ORIG)


def test_original_bruteforce_d2q9_periodic_four_roll():
    pr = W.four_roll(n=8, Wi=0.5, beta=0.5, U0=0.02)
    pr.nx, pr.ny = 7, 5
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D2Q9, pr.shape, seed=22, U=0.03, dA=0.5)
    _compare(pr, 25, ORIG)


def test_original_bruteforce_d3q19_walls_x_z():
    pr = W.Problem("bf3", W.D3Q19, 5, 4, 3, 0.75, 0.1, 13.0, W.FORCE_CONST,
                   (1e-5, 2e-5, -1e-5), walls=0b101)
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D3Q19, pr.shape, seed=23, U=0.03, dA=0.4)
    _compare(pr, 12, ORIG)


def test_original_bruteforce_d3q19_periodic():
    pr = W.Problem("bf3p", W.D3Q19, 4, 5, 3, 0.8, 0.15, 11.0, W.FORCE_NONE, (0.0, 0.0, 0.0))
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D3Q19, pr.shape, seed=24, U=0.03, dA=0.4)
    _compare(pr, 12, ORIG)


def test_newtonian_limit_is_the_present_scheme():
    """eta_p = 0: no stress, no divergence and no f^B; the two schemes are the
    same LB step, to the last bit."""
    pr = W.Problem("n", W.D2Q9, 9, 8, 1, 0.7, 0.0, 10.0, W.FORCE_CONST, (1e-5, 0.0, 0.0),
                   walls=0b10)
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D2Q9, pr.shape, seed=25, U=0.02, dA=0.3)
    a = O.Oracle(pr.lattice, **pr.oracle_kwargs())
    b = O.Oracle(pr.lattice, scheme=ORIG, **pr.oracle_kwargs())
    a.init(u=pr.u0, p=pr.p0, A=pr.A0)
    b.init(u=pr.u0, p=pr.p0, A=pr.A0)
    a.step(40)
    b.step(40)
    fa, ha, _, _ = a.get_state()
    fb, hb, _, _ = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb)


def test_original_momentum_periodic():
    """Periodic box, constant external force: the population momentum grows
    by N F per step; the stress divergence adds nothing in total."""
    pr = W.Problem("c", W.D3Q19, 6, 5, 4, 0.9, 0.2, 20.0, W.FORCE_CONST, (1e-5, -2e-5, 3e-5))
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D3Q19, pr.shape, seed=26, dA=0.5)
    o = O.Oracle(pr.lattice, scheme=ORIG, **pr.oracle_kwargs())
    o.init(u=pr.u0, p=pr.p0, A=pr.A0)
    _, P0 = _momentum(o)
    o.step(30)
    m, P = _momentum(o)
    assert abs(m.sum()) < 1e-13
    want = P0.sum(axis=0) + 30 * pr.sites * np.array(pr.F0)
    assert np.abs(P.sum(axis=0) - want).max() < 1e-14


def test_original_differs_from_present():
    """With polymer stress the schemes are different discretisations of the
    same equations: a dropped divergence (or an f^B left in) would make them
    equal, a wrong sign or index far apart.  On this coarse random field
    (16^2, short wavelengths, large stress) they differ by about 2 % of the
    peak velocity after 20 steps; the closed-form pin below checks their
    agreement where the solution is resolved."""
    pr = W.four_roll(n=16, Wi=0.5, beta=0.5)
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D2Q9, pr.shape, seed=27, U=0.01, dA=0.5)
    a = O.Oracle(pr.lattice, **pr.oracle_kwargs())
    b = O.Oracle(pr.lattice, scheme=ORIG, **pr.oracle_kwargs())
    for o in (a, b):
        o.init(u=pr.u0, p=pr.p0, A=pr.A0)
        o.step(20)
    d = np.abs(a.u() - b.u()).max()
    assert 1e-9 < d < 5e-2 * np.abs(a.u()).max()


def test_original_poiseuille_steady():
    """Sec. 3.2 steady state: u_x, A_xy = lambda u', A_xx = 1 + 2 (lambda u')^2,
    A_yy = 1, reached from the closed form with the same bounds as the
    present scheme's test."""
    L = 32
    pr = W.poiseuille(L=L, nx=1, Wi=1.0, beta=0.1)
    ua, Axx, Axy = W.poiseuille_steady(pr)
    pr.u0 = np.stack([ua, 0 * ua], -1)[:, None, :]
    A = np.zeros((L, 1, 2, 2))
    A[:, 0, 0, 0], A[:, 0, 0, 1], A[:, 0, 1, 0], A[:, 0, 1, 1] = Axx, Axy, Axy, 1.0
    pr.A0 = A
    o = O.Oracle(pr.lattice, scheme=ORIG, **pr.oracle_kwargs())
    o.init(u=pr.u0, p=pr.p0, A=pr.A0)
    o.step(int(12 * pr.lam))
    u = o.u()[:, 0, 0]
    Am = o.A()[:, 0]

    def gre(a, b):
        return np.abs(a - b).sum() / np.abs(b).sum()

    assert gre(u, ua) < 4e-3
    assert gre(Am[:, 0, 1], Axy) < 1.5e-3
    assert gre(Am[:, 0, 0], Axx) < 1.5e-2
    assert np.abs(Am[:, 1, 1] - 1).max() < 1e-5
