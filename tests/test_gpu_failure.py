"""Failure detection without a GPU fault: the periodic finiteness check
(fvlb_set_check_interval / fvlb_status).  The failure is made on the host:
a NaN in the uploaded initial velocity of one node, which the initial
equilibrium carries into that node's populations."""
import numpy as np
import pytest

from paper_2506_13072_gb300 import workloads as W

from gpu_common import fvlb

pytestmark = pytest.mark.gpu


def _sim(prec):
    F = fvlb()
    pr = W.four_roll(n=32, Wi=0.5, beta=0.5)
    pr.u0, pr.p0, pr.A0 = W.random_smooth(pr.lattice, pr.shape, seed=7)
    s = F.Simulation.from_problem(pr, precision=prec)
    return F, pr, s


@pytest.mark.parametrize("prec", [0, 1])
def test_periodic_check_clean_run(prec):
    F, pr, s = _sim(prec)
    s.init_fields(pr.u0, pr.p0, pr.A0)
    s.set_check_interval(5)
    s.step(53)
    assert s.status(wait=True) == F.FVLB_OK
    s.step(7)
    assert s.status(wait=True) == F.FVLB_OK
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_periodic_check_detects_non_finite(prec):
    F, pr, s = _sim(prec)
    u0 = pr.u0.copy()
    u0[5, 9, 0] = np.nan
    s.init_fields(u0, pr.p0, pr.A0)
    s.set_check_interval(5)
    try:
        s.step(12)          # the check at step 5 may already be collected here
    except F.FvlbError as e:
        assert e.code == F.FVLB_EUNSTABLE
    assert s.status(wait=True) == F.FVLB_EUNSTABLE
    assert "step 5" in F.last_error(s.h)
    with pytest.raises(F.FvlbError) as ei:
        s.step(1)
    assert ei.value.code == F.FVLB_EUNSTABLE
    # a new state clears it
    s.init_fields(pr.u0, pr.p0, pr.A0)
    assert s.status(wait=True) == F.FVLB_OK
    s.step(20)
    assert s.status(wait=True) == F.FVLB_OK
    assert s.reduce()["nonfinite"] == 0
    s.close()


def test_check_interval_validation_and_off():
    F, pr, s = _sim(1)
    assert F.lib.fvlb_set_check_interval(s.h, -1) == F.FVLB_EINVAL
    u0 = pr.u0.copy()
    u0[0, 0, 1] = np.inf
    s.init_fields(u0, pr.p0, pr.A0)
    s.set_check_interval(0)          # off: nothing is checked
    s.step(10)
    assert s.status(wait=True) == F.FVLB_OK
    assert s.reduce(check_finite=False)["nonfinite"] > 0
    s.close()
