"""The conformation check (fvlb_conformation): number of nodes where A is not
positive definite, smallest eigenvalue, largest tr A.  The definition is
the eigenvalues of the symmetric tensor A (Sec. 2.1), computed here by
LAPACK (numpy.linalg.eigvalsh) on seeded inputs or on the FP64 oracle's
fields; the count is an integer decision and must match exactly (the inputs
keep every eigenvalue at least 0.05 away from 0)."""
import numpy as np
import pytest

import oracle as O
from paper_2506_13072_gb300 import workloads as W

from gpu_common import fvlb

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1


def _tensors(shape, D, seed, frac_bad=0.05):
    """Symmetric tensors V diag(lam) V^T with random rotations; eigenvalues in
    [0.05, 3], one of them in [-0.5, -0.05] at a random frac_bad of nodes."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    lam = rng.uniform(0.05, 3.0, (n, D))
    bad = rng.random(n) < frac_bad
    lam[bad, 0] = -rng.uniform(0.05, 0.5, bad.sum())
    V, _ = np.linalg.qr(rng.normal(size=(n, D, D)))
    A = np.einsum("nab,nb,ncb->nac", V, lam, V)
    return A.reshape(shape + (D, D)), lam.reshape(shape + (D,))


def _expect(A):
    D = A.shape[-1]
    A = A.reshape(-1, D, D)
    ok = np.isfinite(A).all(axis=(1, 2))
    ev = np.full(len(A), np.nan)
    ev[ok] = np.linalg.eigvalsh(A[ok])[:, 0]
    not_spd = int((~ok).sum() + (ev[ok] <= 0).sum())
    tr = np.trace(A, axis1=1, axis2=2)
    return not_spd, ev[ok].min(), tr[ok].max()


def _sim(lat, shape, prec, walls=0):
    F = fvlb()
    if lat == W.D2Q9:
        ny, nx = shape
        return F.Simulation(F.FVLB_D2Q9, nx, ny, 1, 0.8, 0.1, 10.0, walls=walls, precision=prec)
    nz, ny, nx = shape
    return F.Simulation(F.FVLB_D3Q19, nx, ny, nz, 0.8, 0.1, 10.0, walls=walls, precision=prec)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("lat,shape", [(W.D2Q9, (37, 53)), (W.D2Q9, (1, 1)),
                                       (W.D3Q19, (9, 17, 23)), (W.D3Q19, (1, 1, 5))])
def test_conformation_seeded(lat, shape, prec):
    D = 2 if lat == W.D2Q9 else 3
    A, lam = _tensors(shape, D, seed=sum(shape) + prec, frac_bad=0.05 if np.prod(shape) > 5 else 0.5)
    s = _sim(lat, shape, prec)
    s.init_fields(A=A)
    got = s.conformation()
    n_bad, emin, trmax = _expect(A)
    assert got["not_spd"] == n_bad
    # FP32 storage rounds A - I to ~1e-7 relative; FP64 to ~1e-16
    tol = 1e-12 if prec == FP64 else 2e-6
    scale = np.abs(A).max()
    assert abs(got["min_eig"] - emin) <= tol * scale
    assert abs(got["max_trA"] - trmax) <= tol * scale * D
    s.close()


@pytest.mark.parametrize("lat", [W.D2Q9, W.D3Q19])
def test_conformation_degenerate(lat):
    """A = I (rest), diagonal A, a doubly repeated eigenvalue, a non-finite
    node: the special cases of the closed forms."""
    D = 2 if lat == W.D2Q9 else 3
    shape = (4, 4) if D == 2 else (2, 2, 4)
    s = _sim(lat, shape, FP64)
    s.init_fields()
    got = s.conformation()
    assert got["not_spd"] == 0 and got["min_eig"] == 1.0 and got["max_trA"] == D
    n = int(np.prod(shape))
    A = np.broadcast_to(np.eye(D), (n, D, D)).copy()
    A[1] = np.diag(np.arange(1, D + 1) * 0.5)                 # diagonal
    A[2] = np.diag([2.0] * (D - 1) + [-0.25])                 # diagonal, indefinite
    v = np.ones(D) / np.sqrt(D)
    A[3] = 0.7 * np.eye(D) + 1.3 * np.outer(v, v)             # eigenvalue 0.7 repeated
    A[4, 0, 0] = np.nan                                       # non-finite node
    s.init_fields(A=A.reshape(shape + (D, D)))
    got = s.conformation()
    assert got["not_spd"] == 2
    assert abs(got["min_eig"] - (-0.25)) <= 1e-14
    A[4] = np.eye(D)
    want = _expect(A)
    assert abs(got["max_trA"] - want[2]) <= 1e-13
    s.close()


def test_conformation_four_roll_high_wi():
    """The four-roll mill at Wi = 5 (Sec. 3.1): after 1500 steps of the
    FP64 path the check equals the eigenvalues of the oracle's A."""
    from gpu_common import gpu_sim, oracle_sim

    pr = W.four_roll(n=64, Wi=5.0, beta=0.5, U0=0.01)
    s = gpu_sim(pr, FP64)
    o = oracle_sim(pr)
    s.step(1500)
    o.step(1500)
    got = s.conformation()
    n_bad, emin, trmax = _expect(o.A())
    assert got["not_spd"] == n_bad
    assert abs(got["min_eig"] - emin) <= 1e-10 * abs(emin)
    assert abs(got["max_trA"] - trmax) <= 1e-10 * trmax
    s.close()
