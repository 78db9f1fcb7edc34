"""fvlb_repair_conformation (high-Wi repair) against the oracle's repair
(reading R11 of fvlb_oracle.c): eigenvalues of A below a floor clipped with
the eigenvectors kept, applied as w_i (A' - A) on the stress populations.

1. Seeded tensors with negative eigenvalues at about a fifth of the nodes:
   the repaired-node count is exact and A matches the oracle's.
2. The four-roll mill at Wi = 5 (Sec. 3.1) on a coarse 16^2 grid loses the
   positive definiteness of A near step 900 without repair; repaired after
   every step, it keeps A >= eps at every node, and the FP64 path follows
   the oracle doing the same (u, tau_p within 1e-12, counts equal)."""
import numpy as np
import pytest

from paper_2506_13072_gb300 import workloads as W

from gpu_common import compact, fvlb, gpu_sim, oracle_sim, rel_l2, tau_floor

pytestmark = pytest.mark.gpu

FP64, FP32, FP16 = 0, 1, 2


def _rotation(D, seed):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(D, D)))
    return q * np.sign(np.diag(r))


def _tensors(lat, shape, seed):
    D = 2 if lat == W.D2Q9 else 3
    rng = np.random.default_rng(seed)
    N = int(np.prod(shape))
    A = np.zeros((N, D, D))
    for s in range(N):
        lam = rng.uniform(0.05, 3.0, size=D)
        if rng.random() < 0.2:
            lam[rng.integers(D)] = rng.uniform(-0.5, -0.05)
        V = _rotation(D, 1000 * seed + s)
        A[s] = V @ np.diag(lam) @ V.T
    return A.reshape(shape + (D, D))


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (FP32, 2e-6), (FP16, 2e-3)])
@pytest.mark.parametrize("lat,shape", [(W.D2Q9, (9, 13)), (W.D3Q19, (5, 6, 7))])
def test_repair_matches_oracle(prec, tol, lat, shape):
    D = 2 if lat == W.D2Q9 else 3
    nx, ny = shape[-1], shape[-2]
    pr = W.Problem("rp", lat, nx, ny, shape[0] if D == 3 else 1, 0.8, 0.2, 20.0)
    pr.u0, pr.p0, _ = W.random_smooth(lat, shape, seed=7, U=0.01)
    pr.A0 = _tensors(lat, shape, seed=3)
    s = gpu_sim(pr, prec)
    o = oracle_sim(pr)
    eps = 0.1
    n_gpu = s.repair_conformation(eps)
    n_orc = o.repair(eps)
    # a node within rounding of the floor could fall either way in the
    # reduced precisions; none of these seeded nodes is that close
    assert n_gpu == n_orc > 0
    A_ref = compact(o.A())
    assert np.abs(s.A() - A_ref).max() <= tol * np.abs(A_ref).max()
    # every eigenvalue is now at least eps, up to the rounding of the stored
    # state (a clipped eigenvalue sits at eps, and re-summing the stored
    # populations puts it a rounding error to either side)
    rnd = {FP64: 1e-12, FP32: 1e-5, FP16: 2e-2}[prec]
    assert s.conformation()["min_eig"] >= eps * (1 - rnd)
    s.step(10)
    o.step(10)
    if prec == FP64:
        assert rel_l2(s.u(), o.u(), 1e-30) <= 1e-12
        assert rel_l2(s.tau_p(), compact(o.tau_p()), tau_floor(pr, compact(o.A()), o.u(), 10)) <= 1e-12
    s.close()


def test_repair_keeps_four_roll_wi5_positive_definite():
    pr = W.four_roll(n=16, Wi=5.0, beta=0.5, U0=0.01)
    F = fvlb()
    # without repair: A loses positive definiteness at some nodes
    s = gpu_sim(pr, FP64)
    lost = 0
    for _ in range(40):
        s.step(25)
        lost = max(lost, s.conformation()["not_spd"])
    s.close()
    assert lost > 0
    # repaired after every step: the GPU follows the oracle's repair
    eps = 1e-3
    s = gpu_sim(pr, FP64)
    o = oracle_sim(pr)
    total = 0
    for t in range(1000):
        s.step(1)
        o.step(1)
        n_gpu = s.repair_conformation(eps)
        n_orc = o.repair(eps)
        assert n_gpu == n_orc, (t, n_gpu, n_orc)
        total += n_gpu
    assert total > 0
    c = s.conformation()
    assert c["not_spd"] == 0 and c["min_eig"] >= eps * (1 - 1e-12)
    assert rel_l2(s.u(), o.u(), 1e-30) <= 1e-12
    assert rel_l2(s.tau_p(), compact(o.tau_p()), tau_floor(pr, compact(o.A()), o.u(), 1000)) <= 1e-12
    s.close()


def test_repair_rejects_bad_eps():
    F = fvlb()
    pr = W.four_roll(n=8, Wi=0.5, beta=0.5)
    s = gpu_sim(pr, FP64)
    for eps in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(F.FvlbError):
            s.repair_conformation(eps)
    s.close()
