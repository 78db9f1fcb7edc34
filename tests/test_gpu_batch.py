"""Batched persistent step (fvlb_batch_*): many D2Q9 problems of uneven size
and parameters in one launch per step, against the FP64 oracle instance by
instance, and against the single-grid library."""
import numpy as np
import pytest

from paper_2506_13072_gb300 import workloads as W

from gpu_common import compact, fvlb, tau_floor, oracle_sim, rel_l2

pytestmark = pytest.mark.gpu


def _mixed_problems(seed=21):
    probs = []
    a = W.four_roll(n=16, Wi=0.5, beta=0.5)
    a.u0, a.p0, a.A0 = W.random_smooth(W.D2Q9, a.shape, seed=seed)
    probs.append(a)
    b = W.poiseuille(L=24, nx=20, Wi=1.0, beta=0.1)
    probs.append(b)
    c = W.womersley(L=20, nx=12, gamma=3.0, beta=0.5, Wi=0.5)
    c.u0, c.p0, c.A0 = W.random_smooth(W.D2Q9, c.shape, seed=seed + 1, U=0.01)
    probs.append(c)
    d = W.Problem("r", W.D2Q9, 37, 5, 1, 0.7, 0.15, 11.0, W.FORCE_CONST, (1e-5, -2e-5, 0.0),
                  walls=0b01)
    d.u0, d.p0, d.A0 = W.random_smooth(W.D2Q9, d.shape, seed=seed + 2)
    probs.append(d)
    e = W.Problem("one", W.D2Q9, 1, 1, 1, 0.9, 0.1, 5.0)
    e.u0, e.p0, e.A0 = W.random_smooth(W.D2Q9, e.shape, seed=seed + 3)
    probs.append(e)
    f = W.Problem("c", W.D2Q9, 33, 33, 1, 0.8, 0.05, 30.0, W.FORCE_CONST, (2e-6, 1e-6, 0.0))
    f.u0, f.p0, f.A0 = W.random_smooth(W.D2Q9, f.shape, seed=seed + 4)
    probs.append(f)
    return probs


def _batch(probs, prec):
    F = fvlb()
    bt = F.Batch(probs, precision=prec)
    for i, pr in enumerate(probs):
        if pr.u0 is not None or pr.A0 is not None:
            bt.init_fields(i, pr.u0, pr.p0, pr.A0)
    return bt


@pytest.mark.parametrize("prec,tol,steps", [(0, 1e-12, 45), (1, 1e-5, 45)])
def test_batch_matches_oracle(prec, tol, steps):
    """45 steps: the first direct, 18 autotuning steps over 9 tile shapes,
    then two-step graph replays and a direct remainder."""
    F = fvlb()
    probs = _mixed_problems()
    bt = _batch(probs, prec)
    bt.step(steps)
    bt.synchronize()
    info = bt.info()
    assert info["gx"] in (1, 2, 4) and info["rows"] in (8, 16, 32)
    assert info["tuned_ms_per_step"] > 0
    assert bt.t == steps
    for i, pr in enumerate(probs):
        o = oracle_sim(pr)
        o.step(steps)
        ru = o.u()
        eu = rel_l2(bt.fields(i, F.FVLB_FIELD_U), ru, 1e-30)
        et = rel_l2(bt.fields(i, F.FVLB_FIELD_TAU_P), compact(o.tau_p()), tau_floor(pr, compact(o.A()), o.u(), steps))
        assert eu <= tol and et <= tol, (i, pr.name, eu, et)
    bt.close()


def test_batch_equals_single_grid_runs():
    """Each instance of an FP32 batch evolves as the same problem run alone
    (same node update, different tiling)."""
    F = fvlb()
    probs = _mixed_problems(seed=31)
    bt = _batch(probs, F.FVLB_FP32)
    bt.step(40)
    for i, pr in enumerate(probs):
        s = F.Simulation.from_problem(pr, precision=F.FVLB_FP32)
        s.init_fields(pr.u0, pr.p0, pr.A0)
        s.step(40)
        assert rel_l2(bt.fields(i, F.FVLB_FIELD_U), s.u(), 1e-30) < 1e-6
        assert rel_l2(bt.fields(i, F.FVLB_FIELD_A), s.A(), 1e-30) < 1e-6
        s.close()
    bt.close()


def test_batch_fp16_config_shaped():
    """The batched form as the benchmark runs it (FP16 deviation storage), on
    instances drawn from the benchmark's own list (512 square grids, n
    log-uniform in [32, 512], four-roll or Poiseuille, seed 0): the six
    smallest four-roll and six smallest Poiseuille instances, against the
    oracle in u and tau_p at the 16-bit bound 1e-3."""
    F = fvlb()
    allp = W.batch_instances(count=512, seed=0)
    fr = sorted((p for p in allp if p.name == "four_roll"), key=lambda p: p.nx)[:6]
    po = sorted((p for p in allp if p.name == "poiseuille"), key=lambda p: p.nx)[:6]
    probs = fr + po
    bt = F.Batch(probs, precision=F.FVLB_FP16_DEV)
    steps = 300
    bt.step(steps)
    for i, pr in enumerate(probs):
        o = oracle_sim(pr)
        o.step(steps)
        eu = rel_l2(bt.fields(i, F.FVLB_FIELD_U), o.u(), 1e-30)
        et = rel_l2(bt.fields(i, F.FVLB_FIELD_TAU_P), compact(o.tau_p()),
                    tau_floor(pr, compact(o.A()), o.u(), steps))
        assert eu <= 1e-3 and et <= 1e-3, (i, pr.name, pr.nx, eu, et)
    bt.close()


def test_batch_rejects_bad_specs():
    F = fvlb()
    bad = W.Problem("bad", W.D2Q9, 8, 8, 1, 0.5, 0.1, 1.0)
    with pytest.raises(F.FvlbError):
        F.Batch([bad])
