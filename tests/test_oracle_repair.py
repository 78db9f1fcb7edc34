"""Pins of the oracle's high-Wi repair (reading R11 of fvlb_oracle.c): a node
whose conformation A = sum_i h_i has an eigenvalue below a floor eps gets the
eigenvalues clipped at eps with its eigenvectors kept, applied as
h_i += w_i (A' - A).  Checked against the closed form of a rotated diagonal
tensor and against LAPACK (numpy.linalg.eigh) node by node."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2506_13072_gb300 import workloads as W


def _rotation(D, seed):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(D, D)))
    return q * np.sign(np.diag(r))


def _oracle(lat, shape, A):
    D = 2 if lat == O.D2Q9 else 3
    o = O.Oracle(lat, shape[-1], shape[-2], 1 if D == 2 else shape[0], tau_s=0.8, eta_p=0.2,
                 lam=20.0)
    rng = np.random.default_rng(5)
    u = 0.01 * rng.normal(size=shape + (D,))
    o.init(u=u, A=A)
    return o


@pytest.mark.parametrize("lat,eigs", [(O.D2Q9, (-0.3, 1.5)), (O.D3Q19, (-0.2, 0.5, 2.0)),
                                      (O.D3Q19, (-0.4, -0.1, 3.0))])
def test_repair_closed_form(lat, eigs):
    D = len(eigs)
    R = _rotation(D, 11)
    A0 = R @ np.diag(eigs) @ R.T
    shape = (4, 3) if D == 2 else (2, 3, 4)
    o = _oracle(lat, shape, np.broadcast_to(A0, shape + (D, D)))
    f0, h0, _, _ = o.get_state()
    c, w, _ = O.lattice(lat)
    eps = 0.05
    n = o.repair(eps)
    assert n == int(np.prod(shape))
    want = R @ np.diag(np.maximum(eigs, eps)) @ R.T
    assert np.abs(o.A() - want).max() < 1e-14
    f1, h1, _, _ = o.get_state()
    # the flow populations are untouched and the stress populations change by
    # w_i (A' - A): no other moment of h moves
    assert np.array_equal(f0, f1)
    dh = h1 - h0
    assert np.abs(dh - np.einsum("i,sk->ski", w, (want - A0).reshape(1, D * D))).max() < 1e-15
    assert np.abs(np.einsum("ski,ia->ska", dh, c[:, :D].astype(float))).max() < 1e-15


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_repair_leaves_spd_nodes_alone(lat):
    D = 2 if lat == O.D2Q9 else 3
    shape = (5, 4) if D == 2 else (3, 4, 5)
    _, _, A = W.random_smooth(lat, shape, seed=3, dA=0.5)
    o = _oracle(lat, shape, A)
    before = o.get_state()[1].copy()
    assert o.repair(1e-3) == 0
    assert np.array_equal(o.get_state()[1], before)


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_repair_matches_lapack(lat):
    """Seeded tensors V diag(lambda) V^T with eigenvalues in [0.05, 3] and one
    of them in [-0.5, -0.05] at about a fifth of the nodes."""
    D = 2 if lat == O.D2Q9 else 3
    shape = (6, 5) if D == 2 else (3, 4, 5)
    rng = np.random.default_rng(17)
    N = int(np.prod(shape))
    A = np.zeros((N, D, D))
    for s in range(N):
        lam = rng.uniform(0.05, 3.0, size=D)
        if rng.random() < 0.2:
            lam[rng.integers(D)] = rng.uniform(-0.5, -0.05)
        V = _rotation(D, 100 + s)
        A[s] = V @ np.diag(lam) @ V.T
    o = _oracle(lat, shape, A.reshape(shape + (D, D)))
    eps = 0.1
    Ain = o.A().reshape(N, D, D)
    ev, vec = np.linalg.eigh(Ain)
    want = np.einsum("nak,nk,nbk->nab", vec, np.maximum(ev, eps), vec)
    bad = ev.min(-1) < eps
    want[~bad] = Ain[~bad]
    n = o.repair(eps)
    assert n == int(bad.sum())
    assert np.abs(o.A().reshape(N, D, D) - want).max() < 1e-13
    # and the repaired state steps on
    o.step(5)
    assert np.isfinite(o.A()).all()
