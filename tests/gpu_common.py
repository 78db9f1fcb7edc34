"""Helpers shared by the GPU tests: run the CUDA library and the FP64 oracle
on the same seeded problem and compare them."""
import numpy as np

import oracle as O
from paper_2506_13072_gb300 import workloads as W

_fvlb = None


def fvlb():
    """The binding, with device memory routed through torch's allocator."""
    global _fvlb
    if _fvlb is None:
        import torch

        torch.cuda.init()
        from paper_2506_13072_gb300 import fvlb as F

        F.use_torch_allocator()
        _fvlb = F
    return _fvlb


def rel_l2(x, ref, floor):
    """||x - ref||_2 / ||ref||_2, or / floor when ||ref|| is below it."""
    d = np.linalg.norm(np.ravel(x) - np.ravel(ref))
    n = np.linalg.norm(np.ravel(ref))
    return d / max(n, floor)


def p_floor(u_ref):
    """Norm floor of the pressure error: 0.1 ||u||.  p is of size |u|^2 but
    is recovered from a sum of populations of size |u|, so where the flow
    is slow its absolute error is set by the rounding of those populations;
    below 0.1 ||u|| the relative error of p is measured against 0.1 ||u||."""
    return 0.1 * np.linalg.norm(u_ref) + 1e-30


def tau_floor(pr, A_ref, u_ref=None, steps=1):
    """Norm floor of the polymer-stress error.  tau_p = (eta_p/lambda)(A - I)
    is recovered from stress populations of size w_i (|A - I| + 3 |u| |A|),
    on the oracle's side from h ~ w_i A:
      - FP64 resolves A to about 2 eps |A| per step (the oracle sums 9 or 19
        populations of size w_i |A| and subtracts I), a random walk of
        4e-16 sqrt(steps) |A|;
      - the velocity part 3 |u| |A| of the populations bounds how well either
        side resolves A - I, as |u| does for the pressure (p_floor): below
        0.3 |u| |A| the error is measured against that scale.
    Where the stress is not small against these, the error is relative to
    ||tau_p|| itself."""
    A2 = np.asarray(A_ref).reshape(-1, np.shape(A_ref)[-1])
    nA = np.linalg.norm(A2)
    f = 4e-16 * np.sqrt(max(steps, 1)) * nA
    if u_ref is not None:
        u2 = np.asarray(u_ref).reshape(A2.shape[0], -1)
        f = max(f, 0.3 * np.linalg.norm(np.linalg.norm(u2, axis=1) * np.linalg.norm(A2, axis=1)))
    return pr.eta_p / pr.lam * f + 1e-300


def compact(A):
    return fvlb().full_to_compact(A)


def gpu_sim(pr, precision, kernel=0, scheme=0):
    F = fvlb()
    s = F.Simulation.from_problem(pr, precision=precision, kernel=kernel, scheme=scheme)
    s.init_fields(pr.u0, pr.p0, pr.A0)
    return s


def oracle_sim(pr, scheme=0):
    o = O.Oracle(pr.lattice, scheme=scheme, **pr.oracle_kwargs())
    o.init(u=pr.u0, p=pr.p0, A=pr.A0)
    return o


def compare(pr, steps, precision, tol, kernel=0, chunks=1, fields=("u", "p", "tau_p", "A"),
            scheme=0):
    """Advance both sides `steps` steps (in `chunks` pieces) and return the
    worst relative L2 error per field; assert each is <= tol.  scheme 1: the
    original scheme on both sides."""
    s = gpu_sim(pr, precision, kernel, scheme)
    o = oracle_sim(pr, scheme)
    worst = {k: 0.0 for k in fields}
    per = steps // chunks
    done = 0
    for c in range(chunks):
        n = per if c < chunks - 1 else steps - per * (chunks - 1)
        s.step(n)
        o.step(n)
        done += n
        got = dict(u=s.u(), p=s.p(), tau_p=s.tau_p(), A=s.A())
        ref = dict(u=o.u(), p=o.p(), tau_p=compact(o.tau_p()), A=compact(o.A()))
        floors = dict(u=1e-30, p=p_floor(ref["u"]),
                      tau_p=tau_floor(pr, ref["A"], ref["u"], done), A=1.0)
        for k in fields:
            worst[k] = max(worst[k], rel_l2(got[k], ref[k], floors[k]))
    s.close()
    bad = {k: v for k, v in worst.items() if not v <= tol}
    assert not bad, f"rel-L2 above {tol}: {worst}"
    return worst


def tiled_problem(pr_small, reps):
    """The same problem on a grid `reps` times larger per axis, with the
    initial fields tiled; a periodic problem whose fields have the small
    grid's period evolves as the small one tiled."""
    import copy

    pr = copy.deepcopy(pr_small)
    D = pr.D
    pr.nx *= reps
    pr.ny *= reps
    if D == 3:
        pr.nz *= reps
    tile = (reps,) * D
    pr.u0 = np.tile(pr_small.u0, tile + (1,))
    pr.p0 = np.tile(pr_small.p0, tile)
    pr.A0 = np.tile(pr_small.A0, tile + (1, 1))
    return pr


def tiled_check(small, reps, steps, prec, tol, kernel=0, scheme=0):
    """The GPU on `small` tiled `reps` times per axis against the oracle on
    `small` (periodic problems only); asserts rel-L2 of u and tau_p <= tol."""
    big = tiled_problem(small, reps)
    s = gpu_sim(big, prec, kernel, scheme)
    o = oracle_sim(small, scheme)
    s.step(steps)
    o.step(steps)
    tile = (reps,) * small.D
    ref_u = np.tile(o.u(), tile + (1,))
    ref_t = np.tile(compact(o.tau_p()), tile + (1,))
    eu = rel_l2(s.u(), ref_u, 1e-12)
    et = rel_l2(s.tau_p(), ref_t, 1e-12)
    s.close()
    assert eu <= tol and et <= tol, (eu, et)
    return eu, et
