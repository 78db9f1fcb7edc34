"""Parity of the CUDA library's other constitutive models (Giesekus, linear
and exponential Phan-Thien-Tanner; the relaxation part of the stress source
chi of Sec. 2.3) with the FP64 oracle's, through the C ABI.  Tolerances as
for Oldroyd-B: FP64 1e-12, FP32 1e-5 (relative L2 per field, the norms of
gpu_common.compare); FP16 storage as the Oldroyd-B FP16 form."""
import ctypes

import numpy as np
import pytest

from paper_2506_13072_gb300 import workloads as W

from gpu_common import compare, fvlb, tiled_check

pytestmark = pytest.mark.gpu

FP64, FP32, FP16 = 0, 1, 2
TOL = {FP64: 1e-12, FP32: 1e-5}
GIE, PTTL, PTTE = 1, 2, 3
MODELS = [(GIE, 0.3), (PTTL, 0.4), (PTTE, 0.4)]


def _random(pr, seed, U=0.02, dA=0.5):
    pr.u0, pr.p0, pr.A0 = W.random_smooth(pr.lattice, pr.shape, seed=seed, U=U, dA=dA)
    return pr


def _with(pr, model, par):
    pr.model, pr.mpar = model, par
    return pr


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("model,par", MODELS)
def test_models_four_roll(model, par, prec, kernel):
    pr = _random(W.four_roll(n=64, Wi=1.0, beta=0.5), seed=41, U=0.01)
    compare(_with(pr, model, par), 200, prec, TOL[prec], kernel=kernel, chunks=2)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("model,par", MODELS)
def test_models_poiseuille_walls(model, par, prec):
    pr = W.poiseuille(L=32, nx=8, Wi=1.0, beta=0.1)
    compare(_with(pr, model, par), 400, prec, TOL[prec], chunks=2)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("model,par", MODELS)
def test_models_taylor_green_3d(model, par, prec, kernel):
    pr = _random(W.taylor_green_3d(n=32, U0=0.02, Re=100, Wi=1.0, beta=0.5), seed=42)
    compare(_with(pr, model, par), 40, prec, TOL[prec], kernel=kernel, chunks=2)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("model,par", MODELS)
@pytest.mark.parametrize("lat,shape,walls", [
    (W.D2Q9, (33, 17), 0b10), (W.D3Q19, (37, 19, 11), 0b100), (W.D3Q19, (5, 4, 6), 0b011)])
def test_models_ragged(lat, shape, walls, model, par, prec):
    if lat == W.D2Q9:
        nx, ny = shape
        pr = W.Problem("r", W.D2Q9, nx, ny, 1, 0.7, 0.15, 11.0, W.FORCE_CONST,
                       (1e-5, -2e-5, 0.0), walls=walls)
    else:
        nx, ny, nz = shape
        pr = W.Problem("r3", W.D3Q19, nx, ny, nz, 0.75, 0.1, 13.0, W.FORCE_CONST,
                       (1e-5, 2e-5, -1e-5), walls=walls)
    _random(pr, seed=sum(shape) + walls, dA=0.6)
    compare(_with(pr, model, par), 30, prec, TOL[prec], chunks=2)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("model,par", MODELS)
def test_models_original_scheme(model, par, kernel):
    pr = _random(W.four_roll(n=32, Wi=1.0, beta=0.5), seed=43)
    compare(_with(pr, model, par), 100, FP64, 1e-12, kernel=kernel, chunks=2, scheme=1)


@pytest.mark.parametrize("model,par", MODELS)
def test_models_16bit_storage(model, par):
    """FP16 deviation storage: the Oldroyd-B FP16 four-roll bounds."""
    pr = _with(W.four_roll(n=64, Wi=0.5, beta=0.5), model, par)
    w = compare(pr, 1000, FP16, 1.0, chunks=4, fields=("u", "tau_p"))
    assert w["u"] <= 1e-3 and w["tau_p"] <= 2e-3, w


@pytest.mark.parametrize("model,par", [(GIE, 0.3), (PTTE, 0.4)])
def test_models_full_size_launch_shapes(model, par):
    """1024^2 D2Q9 and 128^3 D3Q19 FP32 launch shapes, checked by periodic
    tiling of 32^2 and 16^3 oracle runs (every node compared)."""
    small = _with(_random(W.four_roll(n=32, Wi=1.0, beta=0.5), seed=44), model, par)
    tiled_check(small, 32, 20, FP32, 1e-5)
    small3 = _with(_random(W.taylor_green_3d(n=16, Wi=1.0, beta=0.5), seed=45), model, par)
    tiled_check(small3, 8, 10, FP32, 1e-5)


def test_model_validation():
    F = fvlb()
    h = ctypes.c_void_p()
    assert F.lib.fvlb_create(ctypes.byref(h), 9, 8, 8, 1, 0.8, 0.1, 10.0, None) == F.FVLB_OK
    try:
        assert F.lib.fvlb_set_model(h, 4, 0.1) == F.FVLB_EINVAL
        assert F.lib.fvlb_set_model(h, GIE, -0.1) == F.FVLB_EINVAL
        assert F.lib.fvlb_set_model(h, GIE, 1.5) == F.FVLB_EINVAL
        assert F.lib.fvlb_set_model(h, PTTE, float("nan")) == F.FVLB_EINVAL
        assert F.lib.fvlb_set_model(h, PTTE, 0.2) == F.FVLB_OK
        assert F.lib.fvlb_set_model(h, 0, 0.0) == F.FVLB_OK
    finally:
        F.lib.fvlb_destroy(h)


def test_model_switch_between_steps():
    """Oldroyd-B for 10 steps, then Giesekus, equals the oracle doing the same."""
    import oracle as O

    from gpu_common import gpu_sim, oracle_sim, rel_l2

    pr = _random(W.four_roll(n=32, Wi=1.0, beta=0.5), seed=46)
    s = gpu_sim(pr, FP64)
    s.step(10)
    s.set_model(GIE, 0.3)
    s.step(10)
    a = oracle_sim(pr)
    a.step(10)
    f, h, chi, first = a.get_state()
    b = O.Oracle(pr.lattice, **{**pr.oracle_kwargs(), "model": GIE, "mpar": 0.3})
    b.set_state(f, h, chi, first, a.t)
    b.step(10)
    assert rel_l2(s.u(), b.u(), 1e-30) <= 1e-12
    assert rel_l2(s.A(), compact_A(b.A()), 1.0) <= 1e-12
    s.close()


def compact_A(A):
    from gpu_common import compact

    return compact(A)
