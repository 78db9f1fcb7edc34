"""Brute-force cross-check of the oracle on tiny grids.

The numpy step below is written independently of the oracle, directly from the
tensor forms of the paper's equations: f^eq and F_i by the tensor contractions
of Sec. 2.2 (not their expanded scalar forms), f^B as the least-norm solution
of the moment constraints solved here with numpy's pseudo-inverse (not the
printed matrices), chi by einsum over full tensors, streaming by np.roll with
bounce-back rows patched afterwards.  Both sides follow the readings listed in
the oracle's header."""
import numpy as np
import pytest

import oracle as O
from paper_2506_13072_gb300 import workloads as W

CS2 = 1.0 / 3.0


class NumpyLB:
    """scheme 0: the present method; 1: the original one (div tau_p as a body
    force, no f^B), the divergence by np.roll central differences with the
    two wall rows replaced by one-sided second-order differences."""

    def __init__(self, pr, scheme=0):
        self.pr = pr
        self.scheme = scheme
        self.D = pr.D
        c, w, opp = O.lattice(pr.lattice)   # lattice tables are pinned separately
        self.c = c[:, : self.D].astype(float)
        self.ci = c[:, : self.D]
        self.w = w
        self.opp = opp
        self.Q = len(w)
        self.shape = pr.shape  # (ny, nx) or (nz, ny, nx); numpy axes reversed vs x,y,z
        D = self.D
        # least-norm f^B: constraints sum f = 0, sum c f = 0, sum c_a c_b f = -tau/tau_f
        rows = [np.ones(self.Q)] + [self.c[:, a] for a in range(D)] + \
               [self.c[:, a] * self.c[:, b] for a in range(D) for b in range(D)]
        self.Cmat = np.stack(rows)
        self.P = np.linalg.pinv(self.Cmat)
        self.tau_h = W.TAU_H

    def axis(self, a):
        """numpy axis of space direction a (x is the last axis)."""
        return len(self.shape) - 1 - a

    def force(self, t):
        pr, D = self.pr, self.D
        F = np.zeros(self.shape + (D,))
        if pr.force_kind == W.FORCE_CONST:
            F[...] = np.array(pr.F0[:D])
        elif pr.force_kind == W.FORCE_COSINE:
            F[...] = np.array(pr.F0[:D]) * np.cos(pr.omega * t)
        elif pr.force_kind == W.FORCE_FOUR_ROLL:
            g = np.meshgrid(*[np.arange(n, dtype=float) for n in self.shape], indexing="ij")
            x, y = g[-1], g[-2]
            F[..., 0] = pr.F0[0] * np.sin(pr.k * x) * np.cos(pr.k * y)
            F[..., 1] = -pr.F0[0] * np.cos(pr.k * x) * np.sin(pr.k * y)
        return F

    def init(self, u, p, A):
        D = self.D
        u = np.zeros(self.shape + (D,)) if u is None else u
        p = np.zeros(self.shape) if p is None else p
        A = np.broadcast_to(np.eye(D), self.shape + (D, D)).copy() if A is None else A
        self.f = self.feq(p, u)
        cu = np.einsum("ia,...a->...i", self.c, u)
        self.h = np.einsum("i,...ab,...i->...abi", self.w, A, 1 + cu / CS2)
        self.chi_old = np.zeros(self.shape + (D, D))
        self.first = True
        self.t = 0

    def feq(self, p, u):
        D = self.D
        lam = self.w / CS2
        lam[0] = (self.w[0] - 1) / CS2
        Qt = np.einsum("ia,ib->iab", self.c, self.c) - CS2 * np.eye(D)
        uu = np.einsum("...a,...b->...ab", u, u)
        cu = np.einsum("ia,...a->...i", self.c, u)
        return (lam * p[..., None] + self.w * (cu / CS2 + np.einsum("...ab,iab->...i", uu, Qt)
                                               / (2 * CS2 ** 2)))

    def grad(self, u):
        """g[..., a, b] = d_a u_b; central, one-sided next to walls."""
        D = self.D
        g = np.zeros(self.shape + (D, D))
        for a in range(D):
            ax = self.axis(a)
            n = self.shape[ax]
            d = 0.5 * (np.roll(u, -1, axis=ax) - np.roll(u, 1, axis=ax))
            if (self.pr.walls >> a) & 1:
                sl = [slice(None)] * len(self.shape)

                def take(j):
                    s = list(sl)
                    s[ax] = j
                    return tuple(s)
                d[take(0)] = u[take(0)] + u[take(1)] / 3.0
                d[take(n - 1)] = -(u[take(n - 1)] + u[take(n - 2)] / 3.0)
            g[..., a, :] = d
        return g

    def div(self, tau):
        """d[..., b] = sum_a d_a tau[..., a, b]."""
        D = self.D
        d = np.zeros(self.shape + (D,))
        for a in range(D):
            ax = self.axis(a)
            n = self.shape[ax]
            if n == 1:
                continue
            t = tau[..., a, :]
            g = 0.5 * (np.roll(t, -1, axis=ax) - np.roll(t, 1, axis=ax))
            if (self.pr.walls >> a) & 1:
                def row(j):
                    return np.take(t, j, axis=ax)
                lo = 0.5 * (-3 * row(0) + 4 * row(1) - row(2))
                hi = -0.5 * (-3 * row(n - 1) + 4 * row(n - 2) - row(n - 3))
                idx = [slice(None)] * (len(self.shape) + 1)
                idx[ax] = 0
                g[tuple(idx)] = lo
                idx[ax] = n - 1
                g[tuple(idx)] = hi
            d += g
        return d

    def stream(self, post):
        """post[..., i] -> populations after streaming with wrap / bounce-back."""
        out = np.zeros_like(post)
        for i in range(self.Q):
            v = post[..., i]
            for a in range(self.D):
                v = np.roll(v, self.ci[i, a], axis=self.axis(a))
            out[..., i] = v
        for a in range(self.D):
            if not (self.pr.walls >> a) & 1:
                continue
            ax = self.axis(a)
            n = self.shape[ax]
            for i in range(self.Q):
                ca = self.ci[i, a]
                if ca == 0:
                    continue
                j = 0 if ca > 0 else n - 1     # nodes whose upstream neighbour is a wall
                s = [slice(None)] * len(self.shape)
                s[ax] = j
                s = tuple(s)
                out[s + (i,)] = post[s + (self.opp[i],)]
        return out

    def step(self):
        pr, D = self.pr, self.D
        c, w = self.c, self.w
        I = np.eye(D)
        F = self.force(self.t)
        f, h = self.f, self.h
        A = h.sum(axis=-1)
        tau_p = pr.eta_p / pr.lam * (A - I)
        if self.scheme:
            F = F + self.div(tau_p)
        u = np.einsum("...i,ia->...a", f, c) + 0.5 * F
        b = np.concatenate([np.zeros(self.shape + (1 + D,)),
                            (-tau_p / pr.tau_s).reshape(self.shape + (D * D,))], axis=-1)
        fB = np.einsum("iq,...q->...i", self.P, b)
        if self.scheme:
            fB = np.zeros_like(fB)
        Qt = np.einsum("ia,ib->iab", c, c) - CS2 * I
        Fu = np.einsum("...a,...b->...ab", F, u)
        Fi = w * (1 - 0.5 / pr.tau_s) * (np.einsum("ia,...a->...i", c, F) / CS2
                                         + np.einsum("...ab,iab->...i", Fu + np.swapaxes(Fu, -1, -2), Qt)
                                         / (2 * CS2 ** 2))
        s0 = w[0] * (-1.5 * (u * u).sum(-1))
        p = CS2 / (1 - w[0]) * (f[..., 1:].sum(-1) + s0 + pr.tau_s * Fi[..., 0]
                                + pr.tau_s * fB[..., 0])
        fpost = f - (f - self.feq(p, u)) / pr.tau_s + fB + Fi
        g = self.grad(u)
        M = A - I
        trM = np.trace(M, axis1=-2, axis2=-1)[..., None, None]
        relax = {0: lambda: M,
                 1: lambda: M + pr.mpar * np.einsum("...ag,...gb->...ab", M, M),
                 2: lambda: (1 + pr.mpar * trM) * M,
                 3: lambda: np.exp(pr.mpar * trM) * M}[pr.model]()
        chi = -relax / pr.lam + np.einsum("...ag,...gb->...ab", A, g) \
            + np.einsum("...ga,...gb->...ab", g, A)
        if self.first:
            self.chi_old = chi.copy()
        cu = np.einsum("ia,...a->...i", c, u)
        heq = np.einsum("i,...ab,...i->...abi", w, A, 1 + cu / CS2)
        phi = w * (1 + (1 - 0.5 / self.tau_h) * cu / CS2)
        src = np.einsum("...ab,...i->...abi", chi, phi)
        old = np.einsum("...ab,...i->...abi", self.chi_old, phi)
        hpost = h - (h - heq) / self.tau_h + src + 0.5 * (src - old)
        self.chi_old = chi
        self.first = False
        self.f = self.stream(fpost)
        hs = hpost.reshape(self.shape + (D * D, self.Q))
        self.h = np.stack([self.stream(hs[..., k, :]) for k in range(D * D)],
                          axis=-2).reshape(hpost.shape)
        self.t += 1

    def fields(self):
        F = self.force(self.t)
        A = self.h.sum(-1)
        if self.scheme:
            F = F + self.div(self.pr.eta_p / self.pr.lam * (A - np.eye(self.D)))
        u = np.einsum("...i,ia->...a", self.f, self.c) + 0.5 * F
        return u, A


def _compare(pr, steps, scheme=0):
    o = O.Oracle(pr.lattice, scheme=scheme, **pr.oracle_kwargs())
    o.init(u=pr.u0, p=pr.p0, A=pr.A0)
    nb = NumpyLB(pr, scheme)
    nb.init(pr.u0, pr.p0, pr.A0)
    for _ in range(steps):
        nb.step()
    o.step(steps)
    u, A = nb.fields()
    f, h, chi, _ = o.get_state()
    assert np.abs(o.u() - u).max() <= 1e-12 * np.abs(u).max()
    assert np.abs(o.A() - A).max() <= 1e-12 * np.abs(A).max()
    assert np.abs(f - nb.f.reshape(f.shape)).max() <= 1e-12 * np.abs(f).max()
    hn = nb.h.reshape(h.shape)
    assert np.abs(h - hn).max() <= 1e-12 * np.abs(hn).max()


def test_bruteforce_d2q9_walls_const_force():
    pr = W.Problem("bf", W.D2Q9, 8, 8, 1, 0.8, 0.2, 15.0, W.FORCE_CONST, (2e-5, -1e-5, 0.0),
                   walls=0b10)
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D2Q9, pr.shape, seed=11, U=0.03, dA=0.5)
    _compare(pr, 25)


def test_bruteforce_d2q9_periodic_four_roll_ragged():
    pr = W.four_roll(n=8, Wi=0.5, beta=0.5, U0=0.02)
    pr.nx, pr.ny = 7, 5            # ragged, non-square
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D2Q9, pr.shape, seed=12, U=0.03, dA=0.5)
    _compare(pr, 25)


def test_bruteforce_d2q9_cosine_walls_x():
    pr = W.Problem("bf", W.D2Q9, 6, 4, 1, 0.7, 0.1, 9.0, W.FORCE_COSINE, (3e-5, 1e-5, 0.0),
                   omega=0.3, walls=0b01)
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D2Q9, pr.shape, seed=13, U=0.03, dA=0.5)
    _compare(pr, 20)


@pytest.mark.parametrize("walls", [0, 0b010, 0b101])
def test_bruteforce_d3q19(walls):
    pr = W.Problem("bf3", W.D3Q19, 5, 4, 6, 0.75, 0.15, 12.0, W.FORCE_CONST,
                   (1e-5, 2e-5, -1e-5), walls=walls)
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D3Q19, pr.shape, seed=14, U=0.03, dA=0.5)
    _compare(pr, 12)


@pytest.mark.parametrize("model,par", [(O.MODEL_GIESEKUS, 0.3), (O.MODEL_PTT_LINEAR, 0.4),
                                       (O.MODEL_PTT_EXP, 0.4)])
@pytest.mark.parametrize("lat", [W.D2Q9, W.D3Q19])
def test_bruteforce_models(lat, model, par):
    """Other constitutive models (reading R9 of the oracle): the relaxation
    part of chi, by full-tensor einsum, in a walled random flow."""
    if lat == W.D2Q9:
        pr = W.Problem("bf", W.D2Q9, 7, 6, 1, 0.8, 0.2, 6.0, W.FORCE_CONST, (2e-5, -1e-5, 0.0),
                       walls=0b10)
    else:
        pr = W.Problem("bf3", W.D3Q19, 5, 4, 6, 0.75, 0.15, 6.0, W.FORCE_CONST,
                       (1e-5, 2e-5, -1e-5), walls=0b001)
    pr.model, pr.mpar = model, par
    pr.u0, pr.p0, pr.A0 = W.random_smooth(lat, pr.shape, seed=21, U=0.03, dA=0.6)
    _compare(pr, 15)


# ---------------------------------------------------------------------------
# Extended precision: the same tensor forms in long double with weights that
# sum to 1 (exact fractions), against the FP64 oracle on a slow, strongly
# stressed channel, where A - I is a small part of A.  With the FP64 weights
# (which sum to 1 - 5.6e-17) in an equilibrium w_i A, every collision would
# scale A by about 1 - 1.1e-16 (1/tau_h ~ 2), a drift of 2e-13 (64 nodes,
# 1000 steps) and 5e-12 (128 nodes, 300 steps) in A - I; the oracle's rest
# equilibrium taken from the zeroth-moment condition (its reading R10)
# removes it.
# ---------------------------------------------------------------------------

class NumpyLBLong(NumpyLB):
    """NumpyLB in long double: exact-fraction weights, the least-norm f^B
    operator refined in long double (Newton-Schulz iteration on the FP64
    pseudo-inverse), force tables in long double."""

    def __init__(self, pr):
        super().__init__(pr)
        LD = np.longdouble
        self.c = self.c.astype(LD)
        if self.Q == 9:
            w = [LD(4) / 9] + [LD(1) / 9] * 4 + [LD(1) / 36] * 4
        else:
            w = [LD(1) / 3] + [LD(1) / 18] * 6 + [LD(1) / 36] * 12
        self.w = np.array(w, dtype=LD)
        Cm = self.Cmat.astype(LD)
        P = self.P.astype(LD)
        for _ in range(3):
            P = 2 * P - P @ Cm @ P
        self.P = P

    def init(self, u, p, A):
        super().init(u, p, A)
        LD = np.longdouble
        self.f = self.f.astype(LD)
        self.h = self.h.astype(LD)
        self.chi_old = self.chi_old.astype(LD)

    def force(self, t):
        return super().force(t).astype(np.longdouble)


@pytest.mark.parametrize("L,steps,bound", [(64, 1000, 1e-13), (128, 300, 2e-12)])
def test_oracle_against_extended_precision(L, steps, bound):
    pr = W.poiseuille(L=L, nx=4, Wi=1.0, beta=0.1)
    nb = NumpyLBLong(pr)
    nb.init(pr.u0, pr.p0, pr.A0)
    for _ in range(steps):
        nb.step()
    o = O.Oracle(pr.lattice, **pr.oracle_kwargs())
    o.init(u=pr.u0, p=pr.p0, A=pr.A0)
    o.step(steps)
    u, A = nb.fields()
    I = np.eye(2)
    T = np.asarray(A - I, dtype=np.float64)
    err = np.linalg.norm((o.A() - I) - T) / np.linalg.norm(T)
    assert err < bound, err
    assert np.linalg.norm(o.u() - np.asarray(u, np.float64)) / np.linalg.norm(np.asarray(u, np.float64)) < 1e-13
