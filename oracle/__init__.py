"""FP64 CPU oracle for the fluctuating lattice Boltzmann method (arXiv 2506.13072).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or calls it.

The arithmetic lives in ``fvlb_oracle.c`` (plain C, FP64, one loop per step of
the paper's algorithm); this module only compiles it with gcc and marshals
arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

D2Q9 = 9
D3Q19 = 19

FORCE_NONE = 0
FORCE_CONST = 1
FORCE_FOUR_ROLL = 2
FORCE_COSINE = 3

FIELD_U = 0
FIELD_P = 1
FIELD_A = 2
FIELD_TAU_P = 3

# scheme: the present method (f^B) or the original one it is compared with
# (div tau_p as a body force, reading R8 of fvlb_oracle.c)
SCHEME_PRESENT = 0
SCHEME_ORIGINAL = 1

# constitutive model (reading R9 of fvlb_oracle.c); its parameter is alpha
# (Giesekus) or eps (PTT)
MODEL_OLDROYD_B = 0
MODEL_GIESEKUS = 1
MODEL_PTT_LINEAR = 2
MODEL_PTT_EXP = 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fvlb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no FMA contraction) and return
    the path of the shared library."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, dp, ctypes.c_double, ctypes.c_double]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_set_walls.argtypes = [ctypes.c_void_p, ctypes.c_uint]
            L.orc_set_walls.restype = ctypes.c_int
            L.orc_set_tau_h.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.orc_set_scheme.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_set_scheme.restype = ctypes.c_int
            L.orc_set_model.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
            L.orc_set_model.restype = ctypes.c_int
            L.orc_time.argtypes = [ctypes.c_void_p]
            L.orc_time.restype = ctypes.c_long
            L.orc_init.argtypes = [ctypes.c_void_p, dp, dp, dp]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            L.orc_fields.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
            L.orc_fields.restype = ctypes.c_int
            L.orc_get_state.argtypes = [ctypes.c_void_p, dp, dp, dp, ip]
            L.orc_set_state.argtypes = [ctypes.c_void_p, dp, dp, dp, ctypes.c_int, ctypes.c_long]
            L.orc_lattice.argtypes = [ctypes.c_int, ip, ip, ip, dp, ip]
            L.orc_lattice.restype = ctypes.c_int
            L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
            L.orc_forcing.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp]
            L.orc_fB.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
            L.orc_fB_matrix.argtypes = [ctypes.c_int, dp]
            L.orc_pressure.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp,
                                       ctypes.c_double, ctypes.c_double]
            L.orc_pressure.restype = ctypes.c_double
            L.orc_force_at.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_long, dp]
            L.orc_repair.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.orc_repair.restype = ctypes.c_long
            _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


# ----------------------------------------------------------------------------
# Per-site building blocks
# ----------------------------------------------------------------------------

def lattice(lat: int):
    """Return (c [Q,3] int, w [Q], opp [Q]) of the lattice."""
    Q = ctypes.c_int()
    D = ctypes.c_int()
    c = (ctypes.c_int * (19 * 3))()
    w = (ctypes.c_double * 19)()
    opp = (ctypes.c_int * 19)()
    if lib().orc_lattice(lat, ctypes.byref(Q), ctypes.byref(D), c, w, opp) != 0:
        raise ValueError("unknown lattice")
    q = Q.value
    return (np.array(c[: 3 * q], dtype=np.int64).reshape(q, 3),
            np.array(w[:q]), np.array(opp[:q], dtype=np.int64))


def qsize(lat: int) -> int:
    return 9 if lat == D2Q9 else 19


def feq(lat: int, p: float, u) -> np.ndarray:
    u3 = np.zeros(3)
    u3[: len(u)] = u
    out = np.zeros(qsize(lat))
    lib().orc_feq(lat, float(p), _dp(u3), _dp(out))
    return out


def forcing(lat: int, tau_f: float, F, u) -> np.ndarray:
    F3 = np.zeros(3)
    F3[: len(F)] = F
    u3 = np.zeros(3)
    u3[: len(u)] = u
    out = np.zeros(qsize(lat))
    lib().orc_forcing(lat, float(tau_f), _dp(F3), _dp(u3), _dp(out))
    return out


def fB(lat: int, tau_f: float, tau_p) -> np.ndarray:
    """f^B from a full D x D polymer-stress tensor."""
    t = _f64(tau_p).ravel()
    out = np.zeros(qsize(lat))
    lib().orc_fB(lat, float(tau_f), _dp(np.ascontiguousarray(t)), _dp(out))
    return out


def fB_matrix(lat: int) -> np.ndarray:
    if lat == D2Q9:
        out = np.zeros((9, 4))
    else:
        out = np.zeros((19, 13))
    lib().orc_fB_matrix(lat, _dp(out))
    return out


def pressure(lat: int, tau_f: float, f, u, F0: float, fB0: float) -> float:
    f = _f64(f)
    u3 = np.zeros(3)
    u3[: len(u)] = u
    return lib().orc_pressure(lat, float(tau_f), _dp(f), _dp(u3), float(F0), float(fB0))


# ----------------------------------------------------------------------------
# The simulation object
# ----------------------------------------------------------------------------

class Oracle:
    """One lattice, one set of parameters, FP64 state on the host.

    Shapes follow the grid ``(nz, ny, nx)`` (x fastest); in 2D ``nz = 1``.
    Tensors are full ``D x D`` (row-major) on the last axis.
    """

    def __init__(self, lat, nx, ny, nz=1, tau_s=0.8, eta_p=0.0, lam=1.0,
                 force_kind=FORCE_NONE, F0=(0.0, 0.0, 0.0), k=0.0, omega=0.0,
                 walls=0, tau_h=None, scheme=SCHEME_PRESENT, model=MODEL_OLDROYD_B,
                 mpar=0.0):
        self.lat = lat
        self.D = 2 if lat == D2Q9 else 3
        self.Q = qsize(lat)
        self.nx, self.ny, self.nz = nx, ny, (1 if self.D == 2 else nz)
        self.N = self.nx * self.ny * self.nz
        F = np.zeros(3)
        F[: len(F0)] = F0
        self._F0 = F
        self._h = lib().orc_create(lat, nx, ny, self.nz, float(tau_s), float(eta_p),
                                   float(lam), int(force_kind), _dp(F), float(k),
                                   float(omega))
        if not self._h:
            raise ValueError("invalid oracle parameters")
        if lib().orc_set_scheme(self._h, int(scheme)) != 0:
            lib().orc_destroy(self._h)
            self._h = None
            raise ValueError("invalid scheme")
        if lib().orc_set_model(self._h, int(model), float(mpar)) != 0:
            lib().orc_destroy(self._h)
            self._h = None
            raise ValueError("invalid constitutive model")
        if lib().orc_set_walls(self._h, int(walls)) != 0:
            lib().orc_destroy(self._h)
            self._h = None
            raise ValueError("invalid wall mask")
        if tau_h is not None:
            lib().orc_set_tau_h(self._h, float(tau_h))
        self.init()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.D == 3 else (self.ny, self.nx)

    @property
    def t(self) -> int:
        return lib().orc_time(self._h)

    def init(self, u=None, p=None, A=None):
        """u: [..., D]; p: [...]; A: [..., D, D] (full) on the grid shape."""
        D, N = self.D, self.N
        u = _f64(u, (N * D,)) if u is not None else None
        p = _f64(p, (N,)) if p is not None else None
        A = _f64(A, (N * D * D,)) if A is not None else None
        lib().orc_init(self._h, _dp(u), _dp(p), _dp(A))

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def fields(self, which: int) -> np.ndarray:
        D, N = self.D, self.N
        if which == FIELD_U:
            out = np.zeros((N, D))
        elif which == FIELD_P:
            out = np.zeros(N)
        elif which in (FIELD_A, FIELD_TAU_P):
            out = np.zeros((N, D, D))
        else:
            raise ValueError(which)
        if lib().orc_fields(self._h, int(which), _dp(out)) != 0:
            raise ValueError(which)
        return out.reshape(self.shape + out.shape[1:])

    def u(self):
        return self.fields(FIELD_U)

    def p(self):
        return self.fields(FIELD_P)

    def A(self):
        return self.fields(FIELD_A)

    def tau_p(self):
        return self.fields(FIELD_TAU_P)

    def get_state(self):
        D, N, Q = self.D, self.N, self.Q
        f = np.zeros((N, Q))
        h = np.zeros((N, D * D, Q))
        chi = np.zeros((N, D * D))
        first = ctypes.c_int()
        lib().orc_get_state(self._h, _dp(f), _dp(h), _dp(chi), ctypes.byref(first))
        return f, h, chi, bool(first.value)

    def set_state(self, f, h, chi, first, t):
        D, N, Q = self.D, self.N, self.Q
        lib().orc_set_state(self._h, _dp(_f64(f, (N * Q,))), _dp(_f64(h, (N * D * D * Q,))),
                            _dp(_f64(chi, (N * D * D,))), int(bool(first)), int(t))

    def repair(self, eps: float) -> int:
        """High-Wi repair (reading R11 of fvlb_oracle.c): clip the
        eigenvalues of A below eps at every node; returns the number of
        nodes changed."""
        return int(lib().orc_repair(self._h, float(eps)))

    def force_at(self, x, y, z=0, t=None):
        out = np.zeros(3)
        lib().orc_force_at(self._h, int(x), int(y), int(z), int(self.t if t is None else t), _dp(out))
        return out
