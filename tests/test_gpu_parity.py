"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 over a whole field, per field, norms as defined in
gpu_common.compare):
  FP64 storage and arithmetic        1e-12 over horizons of <= 1000 steps
  FP32 storage and arithmetic        1e-5  over horizons of <= 1000 steps
                                     (4000 steps: test_long_run_drift)
  16-bit deviation storage           per form and flow, see the tests below
"""
import numpy as np
import pytest

from paper_2506_13072_gb300 import workloads as W

from gpu_common import compare, fvlb, gpu_sim, oracle_sim, rel_l2, tiled_problem, compact

pytestmark = pytest.mark.gpu

FP64, FP32, FP16, BF16 = 0, 1, 2, 3
TOL = {FP64: 1e-12, FP32: 1e-5, FP16: 1e-3, BF16: 1e-3}
KERNELS = [0, 1]  # fused, split


def _with_random(pr, seed, U=0.02, dA=0.4):
    pr.u0, pr.p0, pr.A0 = W.random_smooth(pr.lattice, pr.shape, seed=seed, U=U, dA=dA)
    return pr


# ---------------------------------------------------------------------------
# D2Q9
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("Wi", [0.1, 0.5])
def test_four_roll_64_fp64(kernel, Wi):
    """Simplified four-roll mill, 64^2 periodic, from rest, FP64."""
    pr = W.four_roll(n=64, Wi=Wi, beta=0.5)
    compare(pr, 300, FP64, TOL[FP64], kernel=kernel, chunks=3)




@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("L", [32, 128])
def test_poiseuille_startup(prec, L):
    """Planar Poiseuille start-up, walls on y, 8 periodic columns, 1000 steps."""
    pr = W.poiseuille(L=L, nx=8, Wi=1.0, beta=0.1)
    compare(pr, 1000, prec, TOL[prec], chunks=4, fields=("u", "tau_p", "A"))


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_womersley_cosine_force(prec):
    pr = W.womersley(L=64, nx=4, gamma=3.070, beta=0.5, Wi=0.5)
    compare(pr, 1000, prec, TOL[prec], chunks=3, fields=("u", "tau_p", "A"))


@pytest.mark.parametrize("name,prec,steps,bound", [
    ("poiseuille32", FP32, 4000, 1e-5), ("womersley64", FP32, 4000, 1e-4),
    ("poiseuille128", FP64, 2000, 1e-12), ("womersley64", FP64, 4000, 1e-12)])
def test_long_run_drift(name, prec, steps, bound):
    """Over thousands of steps rounding accumulates coherently (slow flows
    round the same way every step).  FP64 stays within 1e-12 and the FP32
    channel within 1e-5 over 4000 steps; the oscillating Womersley flow in
    FP32 drifts to 8e-5 in u (5e-5 in tau_p) by step 4000, held to 1e-4."""
    pr = {"poiseuille32": lambda: W.poiseuille(L=32, nx=8, Wi=1.0, beta=0.1),
          "poiseuille128": lambda: W.poiseuille(L=128, nx=8, Wi=1.0, beta=0.1),
          "womersley64": lambda: W.womersley(L=64, nx=4, gamma=3.070, beta=0.5, Wi=0.5)}[name]()
    compare(pr, steps, prec, bound, chunks=4, fields=("u", "tau_p"))


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("shape,walls", [((7, 5), 0b01), ((33, 17), 0b10), ((1, 9), 0b10),
                                         ((5, 1), 0), ((1, 1), 0), ((200, 3), 0b11)])
def test_ragged_d2q9(kernel, prec, shape, walls):
    """Ragged and degenerate grids (one-node-wide, single node, several
    tiles plus a ragged tail), random smooth state, both wall layouts."""
    nx, ny = shape
    pr = W.Problem("r", W.D2Q9, nx, ny, 1, 0.7, 0.15, 11.0, W.FORCE_CONST, (1e-5, -2e-5, 0.0),
                   walls=walls)
    _with_random(pr, seed=nx * 100 + ny)
    compare(pr, 60, prec, TOL[prec], kernel=kernel, chunks=2)


# 16-bit storage (flow populations as scaled deviations from the velocity
# part of the receiving node's equilibrium, FP32 rest stress populations
# carrying the rounding residuals).  Measured worst rel-L2 against the FP64
# oracle (u / tau_p), over 1000 (four-roll) and 4000 (channel) steps:
#   FP16 nearest      four-roll 2.4e-5 / 5.7e-4, Poiseuille 32 8.2e-4 / 7.5e-4,
#                     Poiseuille 128 1.5e-5 / 4.8e-4, Womersley 6.9e-5 / 7.6e-4,
#                     Womersley (gamma 5.3, Wi 2) 3.1e-5 / 8.6e-4
#   FP16 stochastic   the same within 1e-3 except tau_p in the channels
#                     (2.35e-3 Poiseuille 32, 1.28e-3 Womersley)
#   BF16 (both)       u 9e-5 .. 9.8e-3, tau_p 4.3e-3 .. 1.2e-2
# FP16 with nearest rounding is the form that meets 1e-3 in every flow; the
# bounds below are 1e-3 for it and the measured errors (rounded up) for the
# others.
FP16SR, BF16SR = 4, 5
REDUCED = {
    # (form, flow): (steps, u bound, tau_p bound)
    (FP16, "four_roll"): (1000, 1e-3, 1e-3),
    (FP16, "poiseuille32"): (4000, 1e-3, 1e-3),
    (FP16, "poiseuille128"): (4000, 1e-3, 1e-3),
    (FP16, "womersley64"): (4000, 1e-3, 1e-3),
    (FP16, "womersley64_wi2"): (4000, 1e-3, 1e-3),
    (FP16SR, "four_roll"): (1000, 1e-3, 1e-3),
    (FP16SR, "poiseuille128"): (4000, 1e-3, 1e-3),
    (FP16SR, "poiseuille32"): (4000, 1.2e-3, 3.5e-3),
    (FP16SR, "womersley64"): (4000, 1e-3, 1.6e-3),
    (BF16, "four_roll"): (1000, 5e-4, 6e-3),
    (BF16, "poiseuille32"): (4000, 1.2e-2, 8e-3),
    (BF16, "poiseuille128"): (4000, 2e-4, 6e-3),
    (BF16, "womersley64"): (4000, 1.5e-3, 9e-3),
    (BF16SR, "four_roll"): (1000, 5e-4, 8e-3),
    (BF16SR, "poiseuille128"): (4000, 2e-4, 9e-3),
    (BF16SR, "womersley64"): (4000, 1.2e-3, 1.3e-2),
}


@pytest.mark.parametrize("prec,flow", sorted(REDUCED))
def test_reduced_precision(prec, flow):
    steps, bu, bt = REDUCED[(prec, flow)]
    if flow == "four_roll":
        pr = W.four_roll(n=64, Wi=0.5, beta=0.5)
    elif flow == "poiseuille32":
        pr = W.poiseuille(L=32, nx=8, Wi=1.0, beta=0.1)
    elif flow == "poiseuille128":
        pr = W.poiseuille(L=128, nx=8, Wi=1.0, beta=0.1)
    elif flow == "womersley64_wi2":
        pr = W.womersley(L=64, nx=4, gamma=5.317, beta=0.5, Wi=2.0)
    else:
        pr = W.womersley(L=64, nx=4, gamma=3.070, beta=0.5, Wi=0.5)
    w = compare(pr, steps, prec, 1.0, chunks=4, fields=("u", "tau_p"))
    assert w["u"] <= bu and w["tau_p"] <= bt, w


# ---------------------------------------------------------------------------
# D3Q19
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_taylor_green_32(kernel, prec):
    pr = W.taylor_green_3d(n=32, U0=0.02, Re=100, Wi=1.0, beta=0.5)
    compare(pr, 40, prec, TOL[prec], kernel=kernel, chunks=2)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("shape,walls", [((37, 19, 11), 0b100), ((5, 4, 6), 0b010),
                                         ((33, 9, 3), 0b101), ((1, 1, 7), 0), ((8, 1, 1), 0),
                                         ((40, 7, 5), 0b010), ((24, 5, 9), 0b100),
                                         ((68, 3, 4), 0b001)])
def test_ragged_d3q19(kernel, prec, shape, walls):
    """Ragged and degenerate grids; nx a multiple of 4 (8, 40, 24, 68) puts
    the FP32 fused step on its bulk tensor copies, whose 64-node boxes run
    past the row (and the grid) there."""
    nx, ny, nz = shape
    pr = W.Problem("r3", W.D3Q19, nx, ny, nz, 0.75, 0.1, 13.0, W.FORCE_CONST,
                   (1e-5, 2e-5, -1e-5), walls=walls)
    _with_random(pr, seed=nx + 7 * ny + 31 * nz)
    compare(pr, 20, prec, TOL[prec], kernel=kernel, chunks=2)


@pytest.mark.parametrize("prec,bu,bt", [(FP16, 1e-3, 1e-3), (FP16SR, 1e-3, 1e-3),
                                         (BF16, 1.5e-3, 4e-3), (BF16SR, 2e-3, 5e-3)])
def test_reduced_precision_taylor_green(prec, bu, bt):
    pr = W.taylor_green_3d(n=32, U0=0.02, Re=100, Wi=1.0, beta=0.5)
    w = compare(pr, 200, prec, 1.0, chunks=2, fields=("u", "tau_p"))
    assert w["u"] <= bu and w["tau_p"] <= bt, w


# 16-bit storage on ragged grids.  A warp whose 32 nodes are all in the grid
# with nx a multiple of 8 copies whole rows in 16-byte chunks; otherwise,
# with nx even, the fused kernel stages the populations of each pair of
# neighbouring nodes with 4-byte copies shared by the pair's two lanes (a
# tile's ragged tail leaves part of a warp without nodes); with nx odd it
# loads them directly.  An exchanged or misplaced chunk or half of a pair
# gives errors of order one; the bounds are those of the 16-bit forms above
# (FP16 1e-3; BF16 with stochastic rounding, measured 1.1e-2 / 7e-3 on
# these random states).
RAGGED16 = [((34, 5, 6), 0b001), ((37, 4, 5), 0b010), ((66, 3, 4), 0), ((40, 5, 4), 0b100),
            ((66, 9), 0b01), ((33, 17), 0b10), ((130, 5), 0), ((136, 9), 0b01)]


@pytest.mark.parametrize("prec,bu,bt", [(FP16, 1e-3, 1e-3), (BF16SR, 1.5e-2, 1.5e-2)])
@pytest.mark.parametrize("shape,walls", RAGGED16)
def test_ragged_16bit(prec, bu, bt, shape, walls):
    if len(shape) == 3:
        nx, ny, nz = shape
        pr = W.Problem("r3", W.D3Q19, nx, ny, nz, 0.75, 0.1, 13.0, W.FORCE_CONST,
                       (1e-5, 2e-5, -1e-5), walls=walls)
    else:
        nx, ny = shape
        pr = W.Problem("r", W.D2Q9, nx, ny, 1, 0.7, 0.15, 11.0, W.FORCE_CONST,
                       (1e-5, -2e-5, 0.0), walls=walls)
    _with_random(pr, seed=sum(shape) + walls)
    w = compare(pr, 20, prec, 1.0, chunks=2, fields=("u", "tau_p"))
    assert w["u"] <= bu and w["tau_p"] <= bt, w


# The fused step stages each warp's populations either with bulk tensor
# copies (one per array group, nx a multiple of 16 bytes' worth of nodes) or
# with per-lane cp.async copies (FVLB_STAGE_TMA=0 forces these); the two
# must give bitwise the same state.
@pytest.mark.parametrize("prec", [FP32, FP16, BF16])
@pytest.mark.parametrize("shape,walls", [((40, 6, 5), 0b010), ((64, 4, 3), 0), ((96, 7), 0b10),
                                         ((136, 5), 0)])
def test_stage_copies_bitwise(prec, shape, walls, monkeypatch):
    if len(shape) == 3:
        nx, ny, nz = shape
        pr = W.Problem("r3", W.D3Q19, nx, ny, nz, 0.75, 0.1, 13.0, W.FORCE_CONST,
                       (1e-5, 2e-5, -1e-5), walls=walls)
    else:
        nx, ny = shape
        pr = W.Problem("r", W.D2Q9, nx, ny, 1, 0.7, 0.15, 11.0, W.FORCE_CONST,
                       (1e-5, -2e-5, 0.0), walls=walls)
    _with_random(pr, seed=sum(shape) + 3 * walls)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("FVLB_STAGE_TMA", flag)
        s = gpu_sim(pr, prec)
        s.step(12)
        out.append(np.concatenate([s.u().ravel(), s.tau_p().ravel(), s.p().ravel()]))
        s.close()
    assert np.array_equal(out[0], out[1])


# ---------------------------------------------------------------------------
# Full-size launch configurations, checked through periodic tiling: a
# problem whose fields repeat with the period of a small grid evolves as the
# small grid's solution tiled, so the oracle on the small grid gives every
# site of the large one.
# ---------------------------------------------------------------------------

def _tiled_check(small, reps, steps, prec, tol, kernel=0):
    big = tiled_problem(small, reps)
    s = gpu_sim(big, prec, kernel)
    o = oracle_sim(small)
    s.step(steps)
    o.step(steps)
    D = small.D
    tile = (reps,) * D
    ref_u = np.tile(o.u(), tile + (1,))
    ref_t = np.tile(compact(o.tau_p()), tile + (1,))
    eu = rel_l2(s.u(), ref_u, 1e-12)
    et = rel_l2(s.tau_p(), ref_t, 1e-12)
    s.close()
    assert eu <= tol and et <= tol, (eu, et)


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_full_size_d3q19_256(prec):
    """256^3 D3Q19 (the benchmark's grid and launch shape) against the
    oracle on a 16^3 period."""
    small = W.Problem("t", W.D3Q19, 16, 16, 16, 0.52, 0.004, 800.0)
    _with_random(small, seed=3, U=0.02, dA=0.3)
    _tiled_check(small, 16, 6, prec, TOL[prec])


@pytest.mark.parametrize("prec", [FP32, FP16])
def test_full_size_d2q9_1024(prec):
    small = W.four_roll(n=32, Wi=0.5, beta=0.5)
    _with_random(small, seed=4)
    _tiled_check(small, 32, 20, prec, TOL[prec])


@pytest.mark.parametrize("prec", [FP32, FP16])
def test_full_size_d2q9_2048(prec):
    """2048^2 D2Q9, the grid and launch shape of the benchmark's D2Q9 forms."""
    small = W.four_roll(n=32, Wi=0.5, beta=0.5)
    _with_random(small, seed=6)
    _tiled_check(small, 64, 12, prec, TOL[prec])


@pytest.mark.parametrize("prec", [FP16, BF16])
def test_full_size_d3q19_256_16bit(prec):
    """256^3 D3Q19 with 16-bit deviation storage (the benchmark's forms);
    bounds of the 16-bit Taylor-Green forms (u and tau_p together)."""
    small = W.Problem("t", W.D3Q19, 16, 16, 16, 0.52, 0.004, 800.0)
    _with_random(small, seed=5, U=0.02, dA=0.3)
    _tiled_check(small, 16, 6, prec, 1e-3 if prec == FP16 else 5e-3)


# ---------------------------------------------------------------------------
# Invariants, diagnostics, checkpoints
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [FP64, FP32])
def test_diagnostics_match_oracle(prec):
    pr = W.taylor_green_3d(n=24, U0=0.02, Re=100, Wi=1.0, beta=0.5)
    s = gpu_sim(pr, prec)
    o = oracle_sim(pr)
    s.step(30)
    o.step(30)
    d = s.reduce()
    u = o.u()
    f, h, chi, _ = o.get_state()
    KE = 0.5 * (u * u).sum(-1).mean()
    tp = o.tau_p()
    PE = 0.5 * np.trace(tp, axis1=-2, axis2=-1).mean()
    tol = 1e-12 if prec == FP64 else 1e-5
    assert d["KE"] == pytest.approx(KE, rel=tol)
    assert d["PE"] == pytest.approx(PE, rel=10 * tol, abs=1e-20)
    # mass and momentum: rounding of the stored populations, relative to
    # their magnitudes (at tau_s = 0.501 the mass mode is barely damped)
    eps = 1e-12 if prec == FP64 else 1e-6
    assert abs(d["mass"] - f.sum()) < eps * np.abs(f).sum()
    c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1],
                  [0, 0, -1], [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1],
                  [-1, 0, -1], [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1],
                  [0, -1, 1]], float)
    P = f @ c
    assert np.abs(d["momentum"] - P.sum(0)).max() < eps * np.abs(P).sum()
    assert d["nonfinite"] == 0
    assert d["umax"] == pytest.approx(np.sqrt((u * u).sum(-1)).max(), rel=tol)
    s.close()


def test_momentum_invariant_periodic():
    """Four-roll force sums to zero over whole periods: the GPU keeps the
    total population momentum fixed (up to rounding) over many steps."""
    pr = W.four_roll(n=128, Wi=0.5, beta=0.5)
    _with_random(pr, seed=5)
    s = gpu_sim(pr, FP64)
    d0 = s.reduce()
    s.step(500)
    d1 = s.reduce()
    assert abs(d1["mass"]) < 1e-12
    # rounding only: relative to the total momentum
    scale = np.abs(d0["momentum"]).max() + 1.0
    assert np.abs(d1["momentum"] - d0["momentum"]).max() < 1e-13 * scale
    s.close()


@pytest.mark.parametrize("prec", [FP64, FP16])
def test_checkpoint_resume_bitwise(prec):
    pr = W.four_roll(n=48, Wi=0.5, beta=0.5)
    _with_random(pr, seed=6)
    a = gpu_sim(pr, prec)
    a.step(17)
    blob = a.save_state()
    a.step(23)
    ua, Aa = a.u(), a.A()
    b = gpu_sim(pr, prec)
    b.load_state(blob)
    assert b.t == 17
    b.step(23)
    assert np.array_equal(b.u(), ua) and np.array_equal(b.A(), Aa)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [FP32, FP16])
def test_deterministic_on_concurrent_streams(prec):
    """No atomics and no order-dependent sums: two handles stepping the same
    problem at once on two streams end in the same bytes as one handle on
    the default stream."""
    import torch

    pr = W.taylor_green_3d(n=32, U0=0.02, Re=100, Wi=1.0, beta=0.5)
    _with_random(pr, seed=8)
    F = fvlb()
    ref = gpu_sim(pr, prec)
    ref.step(30)
    want = ref.save_state()
    ref.close()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sims = []
    for st in streams:
        s = F.Simulation.from_problem(pr, precision=prec, stream=st)
        s.init_fields(pr.u0, pr.p0, pr.A0)
        sims.append(s)
    for _ in range(30):
        for s in sims:
            s.step(1)
    for s in sims:
        assert np.array_equal(s.save_state(), want)
        s.close()


def test_fused_and_split_agree():
    pr = W.taylor_green_3d(n=40, U0=0.02, Re=100, Wi=1.0, beta=0.5)
    a = gpu_sim(pr, FP32, kernel=0)
    b = gpu_sim(pr, FP32, kernel=1)
    a.step(25)
    b.step(25)
    assert rel_l2(a.u(), b.u(), 1e-12) < 1e-6
    a.close()
    b.close()


def test_nonfinite_is_reported():
    """A state with a NaN (injected through the checkpoint image on the host)
    makes fvlb_reduce return FVLB_EUNSTABLE."""
    F = fvlb()
    pr = W.four_roll(n=16, Wi=0.5, beta=0.5)
    s = gpu_sim(pr, FP64)
    blob = s.save_state()
    payload = blob[64:].view(np.float64)   # header is 64 bytes; f_0 comes first
    payload[3] = np.nan
    s.load_state(blob)
    with pytest.raises(F.FvlbError) as e:
        s.reduce()
    assert e.value.code == F.FVLB_EUNSTABLE
    s.close()


def test_allocation_failure_is_reported():
    """A device allocator that fails (injected through the allocator hooks)
    surfaces as FVLB_ENOMEM, and the handle stays usable for destruction."""
    import ctypes

    F = fvlb()
    fail_alloc = F.ALLOC_FN(lambda n, ctx: None)
    noop_free = F.FREE_FN(lambda p, ctx: None)
    assert F.lib.fvlb_set_allocator(fail_alloc, noop_free, None) == F.FVLB_OK
    try:
        s = F.Simulation(F.FVLB_D2Q9, 16, 16, 1, 0.8, 0.1, 10.0)
        with pytest.raises(F.FvlbError) as e:
            s.step(1)
        assert e.value.code == F.FVLB_ENOMEM
        s.close()
    finally:
        F._alloc_refs = None
        F.use_torch_allocator()
