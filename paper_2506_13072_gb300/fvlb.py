"""Python binding of the fvlb C ABI (include/fvlb.h).

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libfvlb.so``.  There is no CPU fallback; if the library is missing
the import of this module fails.  PyTorch supplies device memory (through the
library's allocator hooks, backed by torch's caching allocator) and the CUDA
stream.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libfvlb.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "fvlb.h")

FVLB_D2Q9 = 9
FVLB_D3Q19 = 19

FVLB_OK = 0
FVLB_EINVAL = -1
FVLB_ENOMEM = -2
FVLB_ECUDA = -3
FVLB_EUNSTABLE = -4
FVLB_ETIMEOUT = -5
FVLB_ESTATE = -6

FVLB_FORCE_NONE = 0
FVLB_FORCE_CONST = 1
FVLB_FORCE_FOUR_ROLL = 2
FVLB_FORCE_COSINE = 3

FVLB_FP64 = 0
FVLB_FP32 = 1
FVLB_FP16_DEV = 2
FVLB_BF16_DEV = 3
FVLB_FP16_DEV_SR = 4
FVLB_BF16_DEV_SR = 5

FVLB_KERNEL_FUSED = 0
FVLB_KERNEL_SPLIT = 1

FVLB_SCHEME_PRESENT = 0
FVLB_SCHEME_ORIGINAL = 1
FVLB_MODEL_OLDROYD_B = 0
FVLB_MODEL_GIESEKUS = 1
FVLB_MODEL_PTT_LINEAR = 2
FVLB_MODEL_PTT_EXP = 3

FVLB_FIELD_U = 0
FVLB_FIELD_P = 1
FVLB_FIELD_A = 2
FVLB_FIELD_TAU_P = 3

PRECISIONS = {"fp64": FVLB_FP64, "fp32": FVLB_FP32, "fp16_dev": FVLB_FP16_DEV,
              "bf16_dev": FVLB_BF16_DEV, "fp16_dev_sr": FVLB_FP16_DEV_SR,
              "bf16_dev_sr": FVLB_BF16_DEV_SR}


class FvlbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fvlb error {code}: {msg}")
        self.code = code


class fvlb_force(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("F0", ctypes.c_double * 3),
                ("k", ctypes.c_double), ("omega", ctypes.c_double)]


class fvlb_instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("tau_s", ctypes.c_double),
                ("eta_p", ctypes.c_double), ("lam", ctypes.c_double), ("force", fvlb_force),
                ("walls", ctypes.c_uint)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

if not os.path.exists(LIB_PATH):
    raise ImportError(f"the CUDA library {LIB_PATH} is not built; run "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")

lib = ctypes.CDLL(LIB_PATH)

_H = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_SIGS = {
    "fvlb_set_allocator": ([ALLOC_FN, FREE_FN, ctypes.c_void_p], ctypes.c_int),
    "fvlb_create": ([ctypes.POINTER(_H), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                     ctypes.POINTER(fvlb_force)], ctypes.c_int),
    "fvlb_set_walls": ([_H, ctypes.c_uint], ctypes.c_int),
    "fvlb_set_precision": ([_H, ctypes.c_int], ctypes.c_int),
    "fvlb_set_kernel": ([_H, ctypes.c_int], ctypes.c_int),
    "fvlb_set_scheme": ([_H, ctypes.c_int], ctypes.c_int),
    "fvlb_set_model": ([_H, ctypes.c_int, ctypes.c_double], ctypes.c_int),
    "fvlb_conformation": ([_H, _dp], ctypes.c_int),
    "fvlb_repair_conformation": ([_H, ctypes.c_double, ctypes.POINTER(ctypes.c_longlong)],
                                 ctypes.c_int),
    "fvlb_set_check_interval": ([_H, ctypes.c_long], ctypes.c_int),
    "fvlb_status": ([_H, ctypes.c_int], ctypes.c_int),
    "fvlb_set_stream": ([_H, ctypes.c_void_p], ctypes.c_int),
    "fvlb_init_fields": ([_H, _dp, _dp, _dp], ctypes.c_int),
    "fvlb_step": ([_H, ctypes.c_long], ctypes.c_int),
    "fvlb_fields": ([_H, ctypes.c_int, _dp, ctypes.c_size_t], ctypes.c_int),
    "fvlb_reduce": ([_H, _dp], ctypes.c_int),
    "fvlb_synchronize": ([_H], ctypes.c_int),
    "fvlb_get_time": ([_H, ctypes.POINTER(ctypes.c_long)], ctypes.c_int),
    "fvlb_state_size": ([_H, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "fvlb_save_state": ([_H, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "fvlb_load_state": ([_H, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "fvlb_bytes_per_update": ([_H, _dp], ctypes.c_int),
    "fvlb_last_error": ([_H], ctypes.c_char_p),
    "fvlb_reduce_noalloc": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double,
                             ctypes.c_double, _dp, ctypes.c_void_p, ctypes.c_void_p],
                            ctypes.c_int),
    "fvlb_destroy": ([_H], ctypes.c_int),
    "fvlb_batch_create": ([ctypes.POINTER(_H), ctypes.c_int, ctypes.c_int,
                           ctypes.POINTER(fvlb_instance), ctypes.c_int], ctypes.c_int),
    "fvlb_batch_set_stream": ([_H, ctypes.c_void_p], ctypes.c_int),
    "fvlb_batch_init_fields": ([_H, ctypes.c_int, _dp, _dp, _dp], ctypes.c_int),
    "fvlb_batch_step": ([_H, ctypes.c_long], ctypes.c_int),
    "fvlb_batch_fields": ([_H, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_size_t], ctypes.c_int),
    "fvlb_batch_info": ([_H, ctypes.POINTER(ctypes.c_longlong), _dp, ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_int), _dp], ctypes.c_int),
    "fvlb_batch_synchronize": ([_H], ctypes.c_int),
    "fvlb_batch_get_time": ([_H, ctypes.POINTER(ctypes.c_long)], ctypes.c_int),
    "fvlb_batch_last_error": ([_H], ctypes.c_char_p),
    "fvlb_batch_destroy": ([_H], ctypes.c_int),
    "fvlb_mlp_create": ([ctypes.POINTER(_H), ctypes.c_int, ctypes.c_long, ctypes.c_uint], ctypes.c_int),
    "fvlb_mlp_collect": ([_H, _H, ctypes.c_long], ctypes.c_int),
    "fvlb_mlp_count": ([_H, ctypes.POINTER(ctypes.c_long)], ctypes.c_int),
    "fvlb_mlp_set_loss": ([_H, ctypes.c_double], ctypes.c_int),
    "fvlb_mlp_get_pairs": ([_H, _fp, _fp, ctypes.c_long], ctypes.c_int),
    "fvlb_mlp_train": ([_H, ctypes.c_long, ctypes.c_int, ctypes.c_double, _dp], ctypes.c_int),
    "fvlb_mlp_num_params": ([_H, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "fvlb_mlp_get_params": ([_H, _fp, ctypes.c_size_t], ctypes.c_int),
    "fvlb_mlp_set_params": ([_H, _fp, ctypes.c_size_t], ctypes.c_int),
    "fvlb_mlp_grad": ([_H, _fp, _fp, ctypes.c_long, _fp, _dp], ctypes.c_int),
    "fvlb_mlp_infer": ([_H, _fp, ctypes.c_long, _fp], ctypes.c_int),
    "fvlb_mlp_last_error": ([_H], ctypes.c_char_p),
    "fvlb_mlp_destroy": ([_H], ctypes.c_int),
    "fvlb_set_closure": ([_H, _H, ctypes.c_double], ctypes.c_int),
    "fvlb_closure_stats": ([_H, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)],
                           ctypes.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


def header_symbols(path: str = HEADER_PATH):
    """Names of the entry points declared in include/fvlb.h."""
    with open(path) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fvlb_[a-z0-9_]+)\s*\(", text)))


def last_error(h=None) -> str:
    msg = lib.fvlb_last_error(h)
    return msg.decode() if msg else ""


def check(code, h=None):
    if code != FVLB_OK:
        raise FvlbError(code, last_error(h))
    return code


# ---------------------------------------------------------------------------
# Device memory from torch's caching allocator
# ---------------------------------------------------------------------------
_alloc_refs = None


def use_torch_allocator():
    """Route the library's device allocations through torch's caching
    allocator (on the current device and stream)."""
    global _alloc_refs
    import torch

    if _alloc_refs is not None:
        return

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except Exception:  # out of memory -> the library reports FVLB_ENOMEM
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    check(lib.fvlb_set_allocator(a, f, None))
    _alloc_refs = (a, f)


def use_cuda_allocator():
    global _alloc_refs
    check(lib.fvlb_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _alloc_refs = None


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


class Simulation:
    """One fvlb handle.

    ``lattice`` is FVLB_D2Q9 or FVLB_D3Q19; field arrays use the grid shape
    (ny, nx) or (nz, ny, nx) with components last: u [..., D], p [...],
    A and tau_p [..., C] in compact symmetric order (2D xx, xy, yy; 3D xx,
    yy, zz, xy, xz, yz).
    """

    def __init__(self, lattice, nx, ny, nz=1, tau_s=0.8, eta_p=0.0, lam=1.0,
                 force_kind=FVLB_FORCE_NONE, F0=(0.0, 0.0, 0.0), k=0.0, omega=0.0,
                 walls=0, precision=FVLB_FP64, kernel=FVLB_KERNEL_FUSED, stream=None,
                 scheme=FVLB_SCHEME_PRESENT, model=FVLB_MODEL_OLDROYD_B, mpar=0.0):
        self.lattice = lattice
        self.D = 2 if lattice == FVLB_D2Q9 else 3
        self.C = 3 if self.D == 2 else 6
        self.nx, self.ny, self.nz = nx, ny, (1 if self.D == 2 else nz)
        self.N = self.nx * self.ny * self.nz
        frc = fvlb_force()
        frc.kind = int(force_kind)
        for a in range(3):
            frc.F0[a] = float(F0[a]) if a < len(F0) else 0.0
        frc.k, frc.omega = float(k), float(omega)
        h = _H()
        check(lib.fvlb_create(ctypes.byref(h), int(lattice), int(nx), int(ny), int(self.nz),
                              float(tau_s), float(eta_p), float(lam), ctypes.byref(frc)))
        self.h = h
        try:
            check(lib.fvlb_set_scheme(h, int(scheme)), h)
            check(lib.fvlb_set_model(h, int(model), float(mpar)), h)
            check(lib.fvlb_set_walls(h, int(walls)), h)
            if isinstance(precision, str):
                precision = PRECISIONS[precision]
            check(lib.fvlb_set_precision(h, int(precision)), h)
            check(lib.fvlb_set_kernel(h, int(kernel)), h)
            if stream is not None:
                self.set_stream(stream)
        except Exception:
            lib.fvlb_destroy(h)
            self.h = None
            raise

    @classmethod
    def from_problem(cls, pr, **kw):
        kw.setdefault("model", getattr(pr, "model", FVLB_MODEL_OLDROYD_B))
        kw.setdefault("mpar", getattr(pr, "mpar", 0.0))
        s = cls(pr.lattice, pr.nx, pr.ny, pr.nz, pr.tau_s, pr.eta_p, pr.lam, pr.force_kind,
                pr.F0, pr.k, pr.omega, pr.walls, **kw)
        return s

    # -- life cycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            lib.fvlb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration -------------------------------------------------------
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        ptr = getattr(stream, "cuda_stream", stream)
        check(lib.fvlb_set_stream(self.h, ctypes.c_void_p(ptr or 0)), self.h)

    def set_kernel(self, variant):
        check(lib.fvlb_set_kernel(self.h, int(variant)), self.h)

    def set_scheme(self, scheme):
        check(lib.fvlb_set_scheme(self.h, int(scheme)), self.h)

    def set_check_interval(self, every):
        """Check the state for non-finite values every `every` steps (0: off);
        a failed check makes later steps raise FvlbError(FVLB_EUNSTABLE)."""
        check(lib.fvlb_set_check_interval(self.h, int(every)), self.h)

    def status(self, wait=False):
        """FVLB_OK, or FVLB_EUNSTABLE once a periodic check found a non-finite
        value (no exception)."""
        return lib.fvlb_status(self.h, 1 if wait else 0)

    def set_model(self, model, mpar=0.0):
        check(lib.fvlb_set_model(self.h, int(model), float(mpar)), self.h)

    @property
    def shape(self):
        return (self.ny, self.nx) if self.D == 2 else (self.nz, self.ny, self.nx)

    # -- state ---------------------------------------------------------------
    def init_fields(self, u=None, p=None, A=None):
        """u [..., D], p [...], A [..., C] (compact) or [..., D, D] (full)."""
        N, D, C = self.N, self.D, self.C
        uu = None if u is None else np.ascontiguousarray(np.asarray(u, np.float64).reshape(N * D))
        pp = None if p is None else np.ascontiguousarray(np.asarray(p, np.float64).reshape(N))
        AA = None
        if A is not None:
            A = np.asarray(A, np.float64)
            if A.shape[-2:] == (D, D):
                A = full_to_compact(A)
            AA = np.ascontiguousarray(A.reshape(N * C))
        check(lib.fvlb_init_fields(self.h, _ptr(uu), _ptr(pp), _ptr(AA)), self.h)

    def step(self, n=1):
        check(lib.fvlb_step(self.h, int(n)), self.h)

    def synchronize(self):
        check(lib.fvlb_synchronize(self.h), self.h)

    @property
    def t(self):
        t = ctypes.c_long()
        check(lib.fvlb_get_time(self.h, ctypes.byref(t)), self.h)
        return t.value

    def fields(self, which, out=None):
        nc = {FVLB_FIELD_U: self.D, FVLB_FIELD_P: 1, FVLB_FIELD_A: self.C,
              FVLB_FIELD_TAU_P: self.C}[which]
        if out is None:
            out = np.empty(self.N * nc, np.float64)
        check(lib.fvlb_fields(self.h, int(which), _ptr(out), out.size), self.h)
        shp = self.shape if nc == 1 else self.shape + (nc,)
        return out.reshape(shp)

    def u(self):
        return self.fields(FVLB_FIELD_U)

    def p(self):
        return self.fields(FVLB_FIELD_P)

    def A(self):
        return self.fields(FVLB_FIELD_A)

    def tau_p(self):
        return self.fields(FVLB_FIELD_TAU_P)

    def reduce(self, check_finite=True):
        out = np.zeros(8)
        r = lib.fvlb_reduce(self.h, _ptr(out))
        if r != FVLB_OK and not (r == FVLB_EUNSTABLE and not check_finite):
            raise FvlbError(r, last_error(self.h))
        return dict(mass=out[0], momentum=out[1:4].copy(), KE=out[4], PE=out[5],
                    nonfinite=int(out[6]), umax=out[7])

    def conformation(self):
        """Positive-definiteness check of A: nodes whose smallest eigenvalue
        is not > 0, the smallest eigenvalue, the largest tr A."""
        out = np.zeros(3)
        check(lib.fvlb_conformation(self.h, _ptr(out)), self.h)
        return dict(not_spd=int(out[0]), min_eig=out[1], max_trA=out[2])

    def repair_conformation(self, eps):
        """Clip the eigenvalues of A below eps at every node (eigenvectors
        kept); returns the number of nodes changed."""
        n = ctypes.c_longlong()
        check(lib.fvlb_repair_conformation(self.h, float(eps), ctypes.byref(n)), self.h)
        return n.value

    def state_size(self):
        n = ctypes.c_size_t()
        check(lib.fvlb_state_size(self.h, ctypes.byref(n)), self.h)
        return n.value

    def save_state(self):
        buf = np.empty(self.state_size(), np.uint8)
        check(lib.fvlb_save_state(self.h, buf.ctypes.data_as(ctypes.c_void_p), buf.size), self.h)
        return buf

    def load_state(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        check(lib.fvlb_load_state(self.h, buf.ctypes.data_as(ctypes.c_void_p), buf.size), self.h)

    def bytes_per_update(self):
        b = ctypes.c_double()
        check(lib.fvlb_bytes_per_update(self.h, ctypes.byref(b)), self.h)
        return b.value

    def set_closure(self, mlp, tol=1e-2):
        """Use a trained Mlp for the stress source (None: analytic)."""
        self._mlp = mlp
        check(lib.fvlb_set_closure(self.h, mlp.h if mlp is not None else None, float(tol)), self.h)

    def closure_stats(self):
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        check(lib.fvlb_closure_stats(self.h, ctypes.byref(a), ctypes.byref(b)), self.h)
        return dict(network=a.value, fallback=b.value)


def full_to_compact(A):
    """[..., D, D] -> [..., C] in the library's compact order."""
    D = A.shape[-1]
    if D == 2:
        return np.stack([A[..., 0, 0], A[..., 0, 1], A[..., 1, 1]], -1)
    return np.stack([A[..., 0, 0], A[..., 1, 1], A[..., 2, 2], A[..., 0, 1], A[..., 0, 2],
                     A[..., 1, 2]], -1)


def compact_to_full(A):
    C = A.shape[-1]
    if C == 3:
        out = np.empty(A.shape[:-1] + (2, 2))
        out[..., 0, 0], out[..., 0, 1], out[..., 1, 0], out[..., 1, 1] = \
            A[..., 0], A[..., 1], A[..., 1], A[..., 2]
        return out
    out = np.empty(A.shape[:-1] + (3, 3))
    idx = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (0, 2): 4, (1, 2): 5}
    for (a, b), k in idx.items():
        out[..., a, b] = A[..., k]
        out[..., b, a] = A[..., k]
    return out


class Batch:
    """fvlb_batch_* handle: many D2Q9 problems advanced by one launch per step.

    ``problems`` are workloads.Problem objects (lattice D2Q9)."""

    def __init__(self, problems, precision=FVLB_FP32, stream=None):
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        arr = (fvlb_instance * len(problems))()
        for i, pr in enumerate(problems):
            a = arr[i]
            a.nx, a.ny = pr.nx, pr.ny
            a.tau_s, a.eta_p, a.lam = pr.tau_s, pr.eta_p, pr.lam
            a.force.kind = int(pr.force_kind)
            for q in range(3):
                a.force.F0[q] = float(pr.F0[q]) if q < len(pr.F0) else 0.0
            a.force.k, a.force.omega = float(pr.k), float(pr.omega)
            a.walls = int(pr.walls)
        h = _H()
        check(lib.fvlb_batch_create(ctypes.byref(h), FVLB_D2Q9, len(problems), arr, int(precision)))
        self.h = h
        self.problems = list(problems)
        if stream is not None:
            ptr = getattr(stream, "cuda_stream", stream)
            self._check(lib.fvlb_batch_set_stream(h, ctypes.c_void_p(ptr)))

    def _check(self, code):
        if code != FVLB_OK:
            raise FvlbError(code, (lib.fvlb_batch_last_error(self.h) or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            lib.fvlb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, index, u=None, p=None, A=None):
        pr = self.problems[index]
        N = pr.nx * pr.ny
        uu = None if u is None else np.ascontiguousarray(np.asarray(u, np.float64).reshape(N * 2))
        pp = None if p is None else np.ascontiguousarray(np.asarray(p, np.float64).reshape(N))
        AA = None
        if A is not None:
            A = np.asarray(A, np.float64)
            if A.shape[-2:] == (2, 2):
                A = full_to_compact(A)
            AA = np.ascontiguousarray(A.reshape(N * 3))
        self._check(lib.fvlb_batch_init_fields(self.h, int(index), _ptr(uu), _ptr(pp), _ptr(AA)))

    def step(self, n=1):
        self._check(lib.fvlb_batch_step(self.h, int(n)))

    def synchronize(self):
        self._check(lib.fvlb_batch_synchronize(self.h))

    @property
    def t(self):
        t = ctypes.c_long()
        self._check(lib.fvlb_batch_get_time(self.h, ctypes.byref(t)))
        return t.value

    def fields(self, index, which):
        pr = self.problems[index]
        nc = {FVLB_FIELD_U: 2, FVLB_FIELD_P: 1, FVLB_FIELD_A: 3, FVLB_FIELD_TAU_P: 3}[which]
        out = np.empty(pr.nx * pr.ny * nc, np.float64)
        self._check(lib.fvlb_batch_fields(self.h, int(index), int(which), _ptr(out), out.size))
        return out.reshape((pr.ny, pr.nx) if nc == 1 else (pr.ny, pr.nx, nc))

    def info(self):
        sites = ctypes.c_longlong()
        bpu = ctypes.c_double()
        gx, rows = ctypes.c_int(), ctypes.c_int()
        ms = ctypes.c_double()
        self._check(lib.fvlb_batch_info(self.h, ctypes.byref(sites), ctypes.byref(bpu),
                                        ctypes.byref(gx), ctypes.byref(rows), ctypes.byref(ms)))
        return dict(sites=sites.value, bytes_per_update=bpu.value, gx=gx.value, rows=rows.value,
                    tuned_ms_per_step=ms.value)


def _f32p(a):
    return a.ctypes.data_as(_fp)


class Mlp:
    """fvlb_mlp_* handle: the learned stress closure's network."""

    def __init__(self, lattice, capacity=1 << 20, seed=0):
        h = _H()
        check(lib.fvlb_mlp_create(ctypes.byref(h), int(lattice), int(capacity), int(seed)))
        self.h = h
        self.lattice = lattice
        self.IN, self.OUT = (8, 3) if lattice == FVLB_D2Q9 else (15, 6)

    def _check(self, code):
        if code != FVLB_OK:
            raise FvlbError(code, (lib.fvlb_mlp_last_error(self.h) or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            lib.fvlb_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def collect(self, sim, stride=1):
        self._check(lib.fvlb_mlp_collect(self.h, sim.h, int(stride)))

    @property
    def count(self):
        n = ctypes.c_long()
        self._check(lib.fvlb_mlp_count(self.h, ctypes.byref(n)))
        return n.value

    def pairs(self, n=None):
        n = self.count if n is None else n
        x = np.empty((n, self.IN), np.float32)
        y = np.empty((n, self.OUT), np.float32)
        self._check(lib.fvlb_mlp_get_pairs(self.h, _f32p(x), _f32p(y), n))
        return x, y

    def set_loss(self, delta=0.0):
        """delta > 0: relative loss, each pair weighted 1/(mean t^2 + delta^2)."""
        self._check(lib.fvlb_mlp_set_loss(self.h, float(delta)))

    def train(self, steps, batch=1024, lr=1e-3):
        loss = ctypes.c_double()
        self._check(lib.fvlb_mlp_train(self.h, int(steps), int(batch), float(lr), ctypes.byref(loss)))
        return loss.value

    def params(self):
        n = ctypes.c_size_t()
        self._check(lib.fvlb_mlp_num_params(self.h, ctypes.byref(n)))
        out = np.empty(n.value, np.float32)
        self._check(lib.fvlb_mlp_get_params(self.h, _f32p(out), out.size))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        self._check(lib.fvlb_mlp_set_params(self.h, _f32p(flat), flat.size))

    def grad(self, x, y):
        x = np.ascontiguousarray(x, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        n = ctypes.c_size_t()
        self._check(lib.fvlb_mlp_num_params(self.h, ctypes.byref(n)))
        g = np.empty(n.value, np.float32)
        loss = ctypes.c_double()
        self._check(lib.fvlb_mlp_grad(self.h, _f32p(x), _f32p(y), x.shape[0], _f32p(g),
                                      ctypes.byref(loss)))
        return loss.value, g

    def infer(self, x):
        x = np.ascontiguousarray(x, np.float32)
        y = np.empty((x.shape[0], self.OUT), np.float32)
        self._check(lib.fvlb_mlp_infer(self.h, _f32p(x), x.shape[0], _f32p(y)))
        return y


def mlp_flatten(p):
    """oracle-style parameter dict -> the library's flat FP32 order."""
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(),
                           p["b3"]]).astype(np.float32)


def mlp_unflatten(flat, nin, nout, H=64):
    sizes = [("W1", (H, nin)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (nout, H)),
             ("b3", (nout,))]
    out, o = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], np.float64).reshape(shp)
        o += n
    return out
