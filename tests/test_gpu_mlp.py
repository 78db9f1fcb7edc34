"""The learned stress closure on the GPU: inference on the tensor cores and
the training kernels' gradients against the FP64 reference network
(oracle/mlp.py), the training pairs against the oracle's fields, and a
trained network applied in the step, judged against the FP64 oracle."""
import time

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_2506_13072_gb300 import workloads as W

from gpu_common import compact, fvlb, tau_floor, gpu_sim, oracle_sim, rel_l2, tiled_problem

pytestmark = pytest.mark.gpu


def _f16(a):
    """Round to the nearest IEEE half (ties to even), kept in float64."""
    return np.asarray(a, np.float64).astype(np.float16).astype(np.float64)


def _forward_f16(p, x):
    """The reference forward pass with operands rounded to FP16 as the
    tensor-core path does (weights, and each layer's input)."""
    h = _f16(x)
    h = M.gelu(h @ _f16(p["W1"]).T + p["b1"])
    h = M.gelu(_f16(h) @ _f16(p["W2"]).T + p["b2"])
    return _f16(h) @ _f16(p["W3"]).T + p["b3"]


@pytest.mark.parametrize("lattice", [9, 19])
def test_tensor_core_inference(lattice):
    F = fvlb()
    nin, nout = M.dims(lattice)
    p = M.init_params(lattice, seed=5)
    rng = np.random.default_rng(6)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    net = F.Mlp(lattice, capacity=16)
    net.set_params(F.mlp_flatten(p))
    p32 = F.mlp_unflatten(net.params(), nin, nout)
    x = rng.normal(size=(1000, nin)).astype(np.float32)   # 1000: ragged last warp
    y = net.infer(x).astype(np.float64)
    exact, _ = M.forward(p32, x.astype(np.float64))
    assert rel_l2(y, exact, 1e-30) < 3e-2
    assert rel_l2(y, _forward_f16(p32, x), 1e-30) < 5e-3
    net.close()


@pytest.mark.parametrize("lattice,delta", [(9, 0.0), (19, 0.0), (9, 0.05)])
def test_training_gradient(lattice, delta):
    F = fvlb()
    nin, nout = M.dims(lattice)
    p = M.init_params(lattice, seed=7)
    rng = np.random.default_rng(8)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    net = F.Mlp(lattice, capacity=16)
    net.set_params(F.mlp_flatten(p))
    net.set_loss(delta)
    p32 = F.mlp_unflatten(net.params(), nin, nout)
    x = rng.normal(size=(200, nin)).astype(np.float32)
    t = rng.normal(size=(200, nout)).astype(np.float32)
    loss, g = net.grad(x, t)
    lref, gref = M.loss_and_grad(p32, x.astype(np.float64), t.astype(np.float64), delta)
    assert loss == pytest.approx(lref, rel=1e-5)
    gg = F.mlp_unflatten(g, nin, nout)
    for k in gref:
        assert rel_l2(gg[k], gref[k], 1e-30) < 1e-4, k
    net.close()


def test_collected_pairs_match_oracle_fields():
    """Inputs (lambda grad u, A - I, dt/lambda) and targets lambda chi of the
    sampled nodes, against the oracle's fields of the same state."""
    F = fvlb()
    pr = W.poiseuille(L=16, nx=12, Wi=1.0, beta=0.1)
    pr.u0, pr.p0, pr.A0 = W.random_smooth(W.D2Q9, pr.shape, seed=9, U=0.02, dA=0.4)
    s = gpu_sim(pr, F.FVLB_FP64)
    o = oracle_sim(pr)
    s.step(20)
    o.step(20)
    net = F.Mlp(W.D2Q9, capacity=4096)
    net.collect(s, stride=5)
    x, y = net.pairs()
    u, A = o.u(), o.A()
    ny, nx = pr.shape
    lam = pr.lam
    for j in range(x.shape[0]):
        site = (j * 5) % (nx * ny)
        iy, ix = divmod(site, nx)
        gr = np.zeros((2, 2))
        gr[0] = 0.5 * (u[iy, (ix + 1) % nx] - u[iy, (ix - 1) % nx])
        if iy == 0:
            gr[1] = u[iy, ix] + u[iy + 1, ix] / 3
        elif iy == ny - 1:
            gr[1] = -(u[iy, ix] + u[iy - 1, ix] / 3)
        else:
            gr[1] = 0.5 * (u[iy + 1, ix] - u[iy - 1, ix])
        Ad = A[iy, ix] - np.eye(2)
        want_x = np.concatenate([lam * gr.ravel(), [Ad[0, 0], Ad[0, 1], Ad[1, 1]], [1 / lam]])
        assert np.allclose(x[j], want_x, rtol=1e-5, atol=1e-7), j
        G = lam * gr
        Af = A[iy, ix]
        chi = -Ad + Af @ G + G.T @ Af
        assert np.allclose(y[j], [chi[0, 0], chi[0, 1], chi[1, 1]], rtol=1e-5, atol=1e-7), j
    net.close()
    s.close()


def _train_2d(F, seed=0):
    net = F.Mlp(W.D2Q9, capacity=1 << 20, seed=seed)
    for pr in (W.four_roll(n=64, Wi=0.5, beta=0.5), W.four_roll(n=64, Wi=0.1, beta=0.5),
               W.poiseuille(L=32, nx=8, Wi=1.0, beta=0.1),
               W.womersley(L=64, nx=4, gamma=3.070, beta=0.5, Wi=0.5)):
        s = gpu_sim(pr, F.FVLB_FP32)
        for _ in range(8):
            s.step(500)
            net.collect(s, stride=3)
        s.close()
    net.set_loss(1e-3)   # relative error per pair (floor 1e-3)
    for steps, batch, lr in ((10000, 1024, 2e-3), (10000, 2048, 5e-4), (10000, 4096, 1e-4)):
        loss = net.train(steps, batch=batch, lr=lr)
    return net, loss


@pytest.fixture(scope="module")
def net2d():
    F = fvlb()
    net, loss = _train_2d(F)
    yield net, loss
    net.close()


def _train_3d(F, seed=0):
    """The 3D network as the benchmark trains it: pairs from Taylor-Green
    32^3 runs of the plain method (Wi 1 and 0.2), relative loss."""
    net = F.Mlp(W.D3Q19, capacity=1 << 20, seed=seed)
    for Wi in (1.0, 0.2):
        small = W.taylor_green_3d(n=32, U0=0.02, Re=100, Wi=Wi, beta=0.5)
        s = gpu_sim(small, F.FVLB_FP32)
        for _ in range(8):
            s.step(100)
            net.collect(s, stride=5)
        s.close()
    net.set_loss(1e-3)
    for steps, batch, lr in ((10000, 1024, 2e-3), (10000, 2048, 5e-4), (10000, 4096, 1e-4)):
        net.train(steps, batch=batch, lr=lr)
    return net


@pytest.fixture(scope="module")
def net3d():
    F = fvlb()
    net = _train_3d(F)
    yield net
    net.close()


def _closure_run(pr, net, steps, tol=1e-2):
    F = fvlb()
    s = gpu_sim(pr, F.FVLB_FP32)
    s.set_closure(net, tol=tol)
    s.step(steps)
    st = s.closure_stats()
    served = st["network"] / max(1, st["network"] + st["fallback"])
    assert st["network"] + st["fallback"] == steps * pr.sites
    return s, served


def test_learned_closure_taylor_green_3d(net3d):
    """D3Q19 Taylor-Green 32^3, Wi 1 (the 3D network's own flow), 300 steps
    with the closure against the FP64 oracle's plain method: within 1e-3 in
    u and tau_p, with the fraction of node updates the network served."""
    pr = W.taylor_green_3d(n=32, U0=0.02, Re=100, Wi=1.0, beta=0.5)
    s, served = _closure_run(pr, net3d, 300)
    o = oracle_sim(pr)
    o.step(300)
    eu = rel_l2(s.u(), o.u(), 1e-30)
    et = rel_l2(s.tau_p(), compact(o.tau_p()), tau_floor(pr, compact(o.A()), o.u(), 300))
    s.close()
    print(f"3D closure, TGV 32^3: served {served:.4f}, rel-L2 u {eu:.2e} tau_p {et:.2e}")
    assert eu < 1e-3 and et < 1e-3, (eu, et, served)


def test_learned_closure_taylor_green_256_tiled(net3d):
    """The benchmark's closure launch shape, 256^3: the Taylor-Green field of
    a 32^3 box repeated 8 times per axis evolves as the 32^3 solution tiled,
    so the oracle on 32^3 gives every node (closure and fallback nodes
    alike are node-local)."""
    small = W.taylor_green_3d(n=32, U0=0.02, Re=100, Wi=1.0, beta=0.5)
    small.A0 = np.broadcast_to(np.eye(3), small.shape + (3, 3)).copy()
    big = tiled_problem(small, 8)
    s, served = _closure_run(big, net3d, 20)
    o = oracle_sim(small)
    o.step(20)
    eu = rel_l2(s.u(), np.tile(o.u(), (8, 8, 8, 1)), 1e-30)
    et = rel_l2(s.tau_p(), np.tile(compact(o.tau_p()), (8, 8, 8, 1)), 1e-30)
    s.close()
    assert eu < 1e-3 and et < 1e-3, (eu, et, served)


def test_learned_closure_four_roll_1024(net2d):
    """D2Q9 four-roll mill 1024^2 (k = 2 pi / 1024, the config's closure
    grid), from the forced velocity field, 40 steps with the closure against
    the FP64 oracle's plain method on the full grid."""
    net, _ = net2d
    pr = W.four_roll(n=1024, Wi=0.5, beta=0.5, at_rest=False)
    s, served = _closure_run(pr, net, 40)
    o = oracle_sim(pr)
    o.step(40)
    eu = rel_l2(s.u(), o.u(), 1e-30)
    et = rel_l2(s.tau_p(), compact(o.tau_p()), tau_floor(pr, compact(o.A()), o.u(), 40))
    s.close()
    print(f"2D closure, four-roll 1024^2: served {served:.4f}, rel-L2 u {eu:.2e} tau_p {et:.2e}")
    assert eu < 1e-3 and et < 1e-3, (eu, et, served)


def test_learned_closure_in_the_step(net2d):
    """Trained on pairs from the plain method (four-roll, Poiseuille,
    Womersley trajectories), the network stands in for chi in a four-roll
    run; nodes whose network chi is off by more than 1e-2 relative use the
    analytic chi.  The run stays within 1e-3 of the FP64 oracle, and the test
    reports what the network gains: the fraction of nodes it serves and the
    throughput ratio against the analytic step."""
    F = fvlb()
    net, loss = net2d
    assert loss < 3e-2, loss          # relative mean squared error of the last minibatch
    pr = W.four_roll(n=64, Wi=0.5, beta=0.5)
    s = gpu_sim(pr, F.FVLB_FP32)
    s.set_closure(net, tol=1e-2)
    o = oracle_sim(pr)
    s.step(1000)
    o.step(1000)
    st = s.closure_stats()
    eu = rel_l2(s.u(), o.u(), 1e-30)
    et = rel_l2(s.tau_p(), compact(o.tau_p()), tau_floor(pr, compact(o.A()), o.u(), 1000))
    served = st["network"] / max(1, st["network"] + st["fallback"])
    assert st["network"] + st["fallback"] == 1000 * pr.sites
    assert served > 0.3, served
    assert eu < 1e-3 and et < 1e-3, (eu, et, served)
    # throughput with and without the network on a larger grid
    big = W.four_roll(n=1024, Wi=0.5, beta=0.5)
    rates = {}
    for use in (False, True):
        b = gpu_sim(big, F.FVLB_FP32)
        if use:
            b.set_closure(net, tol=1e-2)
        b.step(3)
        b.synchronize()
        t0 = time.perf_counter()
        b.step(40)
        b.synchronize()
        rates[use] = big.sites * 40 / (time.perf_counter() - t0) / 1e6
        b.close()
    print(f"learned closure: served {served:.3f} of node updates, rel-L2 u {eu:.2e} "
          f"tau_p {et:.2e}, MLUPS {rates[True]:.0f} vs analytic {rates[False]:.0f}")
    s.close()
