"""Pins of the FP64 oracle's per-site building blocks against what the paper
and the mathematics fix: printed lattices and matrices, the moment identities
of Sec. 2.2, the pseudo-inverse of Appendix A recomputed from the lattice
velocities, and the pressure relation of Appendix B."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


# ---------------------------------------------------------------------------
# Lattices
# ---------------------------------------------------------------------------

def test_d2q9_matches_printed_lattice():
    c, w, opp = O.lattice(O.D2Q9)
    for r in _rows("d2q9_lattice.txt"):
        i = int(r[0])
        assert tuple(c[i, :2]) == (int(r[1]), int(r[2]))
        assert c[i, 2] == 0
        assert w[i] == pytest.approx(float(Fraction(r[3])), abs=1e-17)


def test_d3q19_matches_printed_velocities():
    c, _, _ = O.lattice(O.D3Q19)
    for r in _rows("d3q19_velocities.txt"):
        i = int(r[0])
        assert tuple(c[i]) == (int(r[1]), int(r[2]), int(r[3]))


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_lattice_isotropy(lat):
    """Weights must make the lattice 4th-order isotropic with c_s^2 = 1/3
    (this is what fixes the unprinted D3Q19 weights)."""
    c, w, opp = O.lattice(lat)
    D = 2 if lat == O.D2Q9 else 3
    c = c[:, :D].astype(float)
    I = np.eye(D)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-16
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * I, atol=1e-16)
    assert np.abs(np.einsum("i,ia,ib,ig->abg", w, c, c, c)).max() < 1e-16
    m4 = np.einsum("i,ia,ib,ig,id->abgd", w, c, c, c, c)
    iso = CS2 ** 2 * (np.einsum("ab,gd->abgd", I, I) + np.einsum("ag,bd->abgd", I, I)
                      + np.einsum("ad,bg->abgd", I, I))
    assert np.allclose(m4, iso, atol=1e-16)
    for i in range(len(w)):
        assert np.all(c[opp[i]] == -c[i])


# ---------------------------------------------------------------------------
# Equilibrium and forcing moments (Sec. 2.2, the moment conditions)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_feq_moments(lat):
    rng = np.random.default_rng(1)
    c, _, _ = O.lattice(lat)
    D = 2 if lat == O.D2Q9 else 3
    c = c[:, :D].astype(float)
    for _ in range(20):
        u = rng.normal(scale=0.05, size=D)
        p = rng.normal(scale=0.01)
        f = O.feq(lat, p, u)
        assert abs(f.sum()) < 1e-16
        assert np.allclose(c.T @ f, u, atol=1e-16, rtol=0)
        m2 = np.einsum("i,ia,ib->ab", f, c, c)
        assert np.allclose(m2, np.outer(u, u) + p * np.eye(D), atol=1e-16, rtol=0)
        m3 = np.einsum("i,ia,ib,ig->abg", f, c, c, c)
        I = np.eye(D)
        want = CS2 * (np.einsum("ab,g->abg", I, u) + np.einsum("ag,b->abg", I, u)
                      + np.einsum("bg,a->abg", I, u))
        assert np.allclose(m3, want, atol=1e-16, rtol=0)


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_forcing_moments(lat):
    rng = np.random.default_rng(2)
    c, _, _ = O.lattice(lat)
    D = 2 if lat == O.D2Q9 else 3
    c = c[:, :D].astype(float)
    for tau in (0.55, 0.8, 1.7):
        u = rng.normal(scale=0.05, size=D)
        F = rng.normal(scale=1e-4, size=D)
        Fi = O.forcing(lat, tau, F, u)
        k = 1.0 - 0.5 / tau
        assert abs(Fi.sum()) < 1e-18
        assert np.allclose(c.T @ Fi, k * F, atol=1e-19, rtol=0)
        m2 = np.einsum("i,ia,ib->ab", Fi, c, c)
        assert np.allclose(m2, k * (np.outer(F, u) + np.outer(u, F)), atol=1e-19, rtol=0)


# ---------------------------------------------------------------------------
# f^B: pseudo-inverse of the constraint system (Appendix A)
# ---------------------------------------------------------------------------

def _constraint_matrix_2d():
    """Rows in the order of Appendix A: yx, xx, xy, yy, mass, m_x, m_y."""
    c, _, _ = O.lattice(O.D2Q9)
    cx, cy = c[:, 0].astype(float), c[:, 1].astype(float)
    return np.stack([cy * cx, cx * cx, cx * cy, cy * cy, np.ones(9), cx, cy])


def _constraint_matrix_3d():
    """Rows: xx, yy, zz, xy, xz, yx, yz, zx, zy, m_x, m_y, m_z, mass."""
    c, _, _ = O.lattice(O.D3Q19)
    c = c.astype(float)
    x, y, z = c[:, 0], c[:, 1], c[:, 2]
    return np.stack([x * x, y * y, z * z, x * y, x * z, y * x, y * z, z * x, z * y,
                     x, y, z, np.ones(19)])


def test_d2q9_pinv_matches_printed():
    C = _constraint_matrix_2d()
    P = np.linalg.pinv(C)
    printed = np.array(_rows("d2q9_pinv_x72.txt"), dtype=float) / 72.0
    assert np.abs(P - printed).max() < 1e-12
    assert np.abs(O.fB_matrix(O.D2Q9) - P[:, :4]).max() < 1e-12


def test_d3q19_pinv_matches_oracle_matrix():
    C = _constraint_matrix_3d()
    P = np.linalg.pinv(C)
    assert np.abs(O.fB_matrix(O.D3Q19) - P).max() < 1e-12


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_fB_constraints(lat):
    """Sum f^B = 0, sum c f^B = 0, sum c c f^B = -tau_p / tau_f (Sec. 2.2)."""
    rng = np.random.default_rng(3)
    c, _, _ = O.lattice(lat)
    D = 2 if lat == O.D2Q9 else 3
    c = c[:, :D].astype(float)
    C = _constraint_matrix_2d() if lat == O.D2Q9 else _constraint_matrix_3d()
    P = np.linalg.pinv(C)
    for tau_f in (0.6, 0.8, 1.3):
        t = rng.normal(size=(D, D))
        t = t + t.T
        fb = O.fB(lat, tau_f, t)
        assert abs(fb.sum()) < 1e-14
        assert np.abs(c.T @ fb).max() < 1e-14
        assert np.allclose(np.einsum("i,ia,ib->ab", fb, c, c), -t / tau_f, atol=1e-14)
        if lat == O.D2Q9:
            b = -np.array([t[1, 0], t[0, 0], t[0, 1], t[1, 1], 0, 0, 0]) / tau_f
        else:
            b = -np.array([t[0, 0], t[1, 1], t[2, 2], t[0, 1], t[0, 2], t[1, 0], t[1, 2],
                           t[2, 0], t[2, 1], 0, 0, 0, 0]) / tau_f
        assert np.allclose(fb, P @ b, atol=1e-14)


def test_fB_d2q9_compact_form_example():
    """Worked example of the printed D2Q9 matrix: tau_xx = 1, others 0,
    tau_f = 1 gives f^B = -(1/72)(-24, 12, -24, 12, -24, 12, 12, 12, 12)."""
    fb = O.fB(O.D2Q9, 1.0, np.array([[1.0, 0.0], [0.0, 0.0]]))
    want = -np.array([-24, 12, -24, 12, -24, 12, 12, 12, 12]) / 72.0
    assert np.allclose(fb, want, atol=1e-16)


# ---------------------------------------------------------------------------
# Pressure relation (Appendix B)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_pressure_inverts_appendix_b(lat):
    """For populations with sum f = 0 (Sec. 2.2), the pressure formula returns
    the p for which f_0 - f_0^eq(p, u) = tau_f (f_0^B + F_0)."""
    rng = np.random.default_rng(4)
    Q = O.qsize(lat)
    D = 2 if lat == O.D2Q9 else 3
    for tau_f in (0.6, 0.8, 1.5):
        f = rng.normal(scale=0.01, size=Q)
        f[0] = -f[1:].sum()
        u = rng.normal(scale=0.05, size=D)
        F0, fB0 = rng.normal(scale=1e-3), rng.normal(scale=1e-3)
        p = O.pressure(lat, tau_f, f, u, F0, fB0)
        lhs = f[0] - O.feq(lat, p, u)[0]
        assert lhs == pytest.approx(tau_f * (fB0 + F0), abs=1e-16)


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_pressure_of_equilibrium(lat):
    """With no force and no stress, the pressure of f = f^eq(p, u) is p."""
    rng = np.random.default_rng(5)
    D = 2 if lat == O.D2Q9 else 3
    for _ in range(10):
        u = rng.normal(scale=0.05, size=D)
        p = rng.normal(scale=0.01)
        f = O.feq(lat, p, u)
        assert O.pressure(lat, 0.8, f, u, 0.0, 0.0) == pytest.approx(p, abs=1e-16)
