"""Parity of the CUDA library's original scheme (the one the paper compares
its method with, Sec. 1 and Tables 1-2: the polymer stress divergence as a
finite-difference body force, no f^B) with the FP64 oracle's original
scheme, through the C ABI.  Tolerances as for the present scheme: FP64
1e-12, FP32 1e-5 (relative L2 per field, norms of gpu_common.compare)."""
import numpy as np
import pytest

from paper_2506_13072_gb300 import workloads as W

from gpu_common import compare, fvlb, gpu_sim, oracle_sim, rel_l2

pytestmark = pytest.mark.gpu

FP64, FP32, FP16 = 0, 1, 2
TOL = {FP64: 1e-12, FP32: 1e-5}
ORIG = 1


def _random(pr, seed, U=0.02, dA=0.4):
    pr.u0, pr.p0, pr.A0 = W.random_smooth(pr.lattice, pr.shape, seed=seed, U=U, dA=dA)
    return pr


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_original_four_roll(prec, kernel):
    pr = _random(W.four_roll(n=64, Wi=0.5, beta=0.5), seed=31, U=0.01, dA=0.3)
    compare(pr, 200, prec, TOL[prec], kernel=kernel, chunks=2, scheme=ORIG)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_original_poiseuille_walls(prec, kernel):
    pr = W.poiseuille(L=32, nx=8, Wi=1.0, beta=0.1)
    compare(pr, 400, prec, TOL[prec], kernel=kernel, chunks=2, scheme=ORIG)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_original_taylor_green_3d(prec, kernel):
    pr = W.taylor_green_3d(n=32, U0=0.02, Re=100, Wi=1.0, beta=0.5)
    compare(pr, 40, prec, TOL[prec], kernel=kernel, chunks=2, scheme=ORIG)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("lat,shape,walls", [
    (W.D2Q9, (33, 17), 0b10), (W.D2Q9, (7, 5), 0b11),
    (W.D3Q19, (37, 19, 11), 0b100), (W.D3Q19, (5, 4, 6), 0b011)])
@pytest.mark.parametrize("kernel", [0, 1])
def test_original_ragged(prec, lat, shape, walls, kernel):
    if lat == W.D2Q9:
        nx, ny = shape
        pr = W.Problem("r", W.D2Q9, nx, ny, 1, 0.7, 0.15, 11.0, W.FORCE_CONST,
                       (1e-5, -2e-5, 0.0), walls=walls)
    else:
        nx, ny, nz = shape
        pr = W.Problem("r3", W.D3Q19, nx, ny, nz, 0.75, 0.1, 13.0, W.FORCE_CONST,
                       (1e-5, 2e-5, -1e-5), walls=walls)
    _random(pr, seed=sum(shape) + walls)
    compare(pr, 30, prec, TOL[prec], kernel=kernel, chunks=2, scheme=ORIG)


def test_original_16bit_storage():
    """FP16 deviation storage under the original scheme: the same bounds as
    the present scheme's FP16 four-roll form (u 1e-3, tau_p 2e-3)."""
    pr = W.four_roll(n=64, Wi=0.5, beta=0.5)
    w = compare(pr, 1000, FP16, 1.0, chunks=4, fields=("u", "tau_p"), scheme=ORIG)
    assert w["u"] <= 1e-3 and w["tau_p"] <= 2e-3, w


def test_original_diagnostics_match_oracle():
    """FP64 diagnostics use the same total force as the step: kinetic energy
    (u includes half the stress divergence) equals the oracle's."""
    F = fvlb()
    pr = _random(W.four_roll(n=32, Wi=0.5, beta=0.5), seed=33, U=0.02, dA=0.5)
    s = gpu_sim(pr, FP64, scheme=ORIG)
    o = oracle_sim(pr, ORIG)
    s.step(25)
    o.step(25)
    d = s.reduce()
    u = o.u()
    ke = 0.5 * (u * u).sum(-1).mean()   # the diagnostics report the mean per node
    assert abs(d["KE"] - ke) <= 1e-12 * ke
    s.close()


def test_schemes_switch_between_steps():
    """The scheme can change between steps: present, then original, equals
    the oracle doing the same."""
    pr = _random(W.four_roll(n=32, Wi=0.5, beta=0.5), seed=34)
    s = gpu_sim(pr, FP64)
    s.step(10)
    s.set_scheme(ORIG)
    s.step(10)
    a = oracle_sim(pr)
    a.step(10)
    f, h, chi, first = a.get_state()
    import oracle as O
    b = O.Oracle(pr.lattice, scheme=ORIG, **pr.oracle_kwargs())
    b.set_state(f, h, chi, first, a.t)
    b.step(10)
    assert rel_l2(s.u(), b.u(), 1e-30) <= 1e-12
    s.close()


def test_scheme_validation():
    """The original scheme's wall stencil needs 3 nodes across a wall; the
    checks run on the host before any device work."""
    import ctypes

    F = fvlb()
    h = ctypes.c_void_p()
    assert F.lib.fvlb_create(ctypes.byref(h), 9, 8, 2, 1, 0.8, 0.1, 10.0, None) == F.FVLB_OK
    try:
        assert F.lib.fvlb_set_scheme(h, 7) == F.FVLB_EINVAL
        assert F.lib.fvlb_set_walls(h, 0b10) == F.FVLB_OK          # 2 nodes: fine for f^B
        assert F.lib.fvlb_set_scheme(h, F.FVLB_SCHEME_ORIGINAL) == F.FVLB_EINVAL
        assert F.lib.fvlb_set_walls(h, 0) == F.FVLB_OK
        assert F.lib.fvlb_set_scheme(h, F.FVLB_SCHEME_ORIGINAL) == F.FVLB_OK
        assert F.lib.fvlb_set_walls(h, 0b10) == F.FVLB_EINVAL      # now 3 are needed
        assert F.lib.fvlb_set_scheme(h, F.FVLB_SCHEME_PRESENT) == F.FVLB_OK
    finally:
        F.lib.fvlb_destroy(h)


@pytest.mark.parametrize("prec", [FP32, FP16])
def test_original_full_size_launch_shapes(prec):
    """The fused original scheme in the 256^3 D3Q19 and 2048^2 D2Q9 launch
    shapes of the benchmark, by periodic tiling of 16^3 and 32^2 oracle runs."""
    from gpu_common import tiled_check

    tol = TOL[FP32] if prec == FP32 else 2e-3
    small = _random(W.taylor_green_3d(n=16, Wi=1.0, beta=0.5), seed=35)
    tiled_check(small, 16, 6, prec, tol, scheme=ORIG)
    small2 = _random(W.four_roll(n=32, Wi=0.5, beta=0.5), seed=36)
    tiled_check(small2, 64, 12, prec, tol, scheme=ORIG)
