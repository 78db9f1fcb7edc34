"""fvlb_reduce_noalloc: the diagnostics reduction for callers that cannot
allocate device memory (a framework allocator that has reserved the GPU's
memory, or an asynchronous pipeline that must not call cudaMalloc/cudaFree
because they can synchronise the device).  Its partial sums live in a static
device array inside the library; the caller passes the state and an output
buffer it already owns.

The test takes a handle's state (through its checkpoint image), gives it to
the allocation-free entry point as caller-owned device buffers, and checks
that two calls in a row reproduce fvlb_reduce of the same handle."""
import ctypes

import numpy as np
import pytest

from paper_2506_13072_gb300 import workloads as W

from gpu_common import fvlb, gpu_sim

pytestmark = pytest.mark.gpu

HEADER = 64


def _state_on_device(sim, pr, precision):
    import torch

    F = fvlb()
    blob = sim.save_state()
    pitch = int(np.frombuffer(blob[40:48].tobytes(), dtype=np.int64)[0])
    Q = 9 if pr.lattice == W.D2Q9 else 19
    C = 3 if pr.lattice == W.D2Q9 else 6
    D = 2 if pr.lattice == W.D2Q9 else 3
    sb = {F.FVLB_FP64: 8, F.FVLB_FP32: 4}.get(precision, 2)
    nf, nh = Q * pitch * sb, C * Q * pitch * sb
    if sb == 2:   # 16-bit forms: FP32 U[D][pitch] and h0[C][pitch] follow
        nf += 4 * D * pitch
        nh += 4 * C * pitch
    f = torch.from_numpy(blob[HEADER:HEADER + nf].copy()).cuda()
    h = torch.from_numpy(blob[HEADER + nf:HEADER + nf + nh].copy()).cuda()
    return f, h, pitch


@pytest.mark.parametrize("case", ["d3q19_fp32", "d2q9_fp16_walls", "d3q19_fp64"])
def test_reduce_noalloc_matches_reduce(case):
    import torch

    F = fvlb()
    if case == "d3q19_fp32":
        pr = W.taylor_green_3d(n=24, U0=0.02, Re=100, Wi=1.0, beta=0.5)
        prec = F.FVLB_FP32
    elif case == "d3q19_fp64":
        pr = W.taylor_green_3d(n=20, U0=0.02, Re=100, Wi=1.0, beta=0.5)
        prec = F.FVLB_FP64
    else:
        pr = W.poiseuille(L=33, nx=40, Wi=1.0, beta=0.1)
        prec = F.FVLB_FP16_DEV
    sim = gpu_sim(pr, prec)
    sim.step(7)
    ref = sim.reduce()
    f, h, pitch = _state_on_device(sim, pr, prec)
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    Fv = (ctypes.c_double * 3)(*[float(v) for v in pr.F0])
    if pr.force_kind not in (W.FORCE_CONST,):
        Fv = None
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        r = F.lib.fvlb_reduce_noalloc(pr.lattice, prec, pr.nx, pr.ny, pr.nz, f.data_ptr(),
                                      h.data_ptr(), pitch, pr.eta_p, pr.lam, Fv,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert r == F.FVLB_OK, F.last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = np.array([ref["mass"], *ref["momentum"], ref["KE"], ref["PE"],
                         ref["nonfinite"], ref["umax"]])
        # same kernels, same launch shape, same summation order: equal within
        # the FP64 parity tolerance
        assert np.allclose(got, want, rtol=1e-12, atol=1e-300), (call, got, want)
        out.fill_(float("nan"))
    sim.close()


def test_reduce_noalloc_rejects_bad_arguments():
    """Every rejected call returns FVLB_EINVAL with a message and leaves the
    caller's output buffer as it was."""
    import torch

    F = fvlb()
    # room for h'[6][19][64] (the largest array the valid call below reads)
    buf = torch.zeros(6 * 19 * 64, dtype=torch.float32, device="cuda")
    out = torch.full((8,), 7.0, dtype=torch.float64, device="cuda")
    f, h, o = buf.data_ptr(), buf.data_ptr(), out.data_ptr()

    def call(lattice=19, storage=None, nx=4, ny=4, nz=4, pitch=64, eta_p=0.1, lam=10.0,
             fp=f, hp=h, op=o):
        st = F.FVLB_FP32 if storage is None else storage
        return F.lib.fvlb_reduce_noalloc(lattice, st, nx, ny, nz, fp, hp, pitch, eta_p, lam, None,
                                         ctypes.c_void_p(op), None)

    bad = [dict(nx=0), dict(pitch=32),                      # pitch < N
           dict(nx=4096, ny=4096, nz=4096, pitch=4096 ** 3),  # beyond the limit
           dict(lattice=7), dict(storage=6), dict(storage=-1),
           dict(fp=None), dict(hp=None), dict(op=None),
           dict(lam=0.0), dict(lam=-1.0), dict(lam=float("inf")), dict(eta_p=-0.1),
           dict(eta_p=float("nan"))]
    for kw in bad:
        assert call(**kw) == F.FVLB_EINVAL, kw
        assert "fvlb_reduce_noalloc" in F.last_error()
        torch.cuda.synchronize()
        assert (out.cpu().numpy() == 7.0).all(), kw
    # a valid call on the same buffers goes through
    assert call() == F.FVLB_OK
    torch.cuda.synchronize()
