"""FP64 CPU oracle for bead-rod Brownian dynamics with HI (arXiv 2208.06559, Sec. 3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library never
imports, links or calls it, and the two share no code.

The arithmetic lives in ``bd_oracle.c`` (plain C loops, FP64); this module
compiles it with gcc and marshals numpy arrays through ctypes.  Every function
cites the passage of the paper it follows in ``bd_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bd_oracle.c")
_HDR = os.path.join(_HERE, "bd_oracle.h")
_LIB = os.path.join(_HERE, "libbd_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_NOT_PD = -4
ERR_CONSTRAINT = -5
FLOW_NONE, FLOW_SHEAR, FLOW_UNIAXIAL = 0, 1, 2
RIGID, FRAENKEL = 0, 1
SCHEME_MIDPOINT, SCHEME_EULER = 0, 1
OBS_STRIDE = 12


class Params(ctypes.Structure):
    _fields_ = [
        ("hstar", ctypes.c_double),
        ("a", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("flow", ctypes.c_int),
        ("Wi", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("max_newton", ctypes.c_int),
        ("constraint", ctypes.c_int),
        ("kspring", ctypes.c_double),
        ("scheme", ctypes.c_int),
    ]


def make_params(hstar=0.25, a=0.0, dt=1e-4, flow=FLOW_NONE, Wi=0.0, lam=1.0,
                tol=1e-13, max_newton=50, constraint=RIGID, kspring=0.0,
                scheme=SCHEME_MIDPOINT) -> Params:
    return Params(float(hstar), float(a), float(dt), int(flow), float(Wi),
                  float(lam), float(tol), int(max_newton), int(constraint), float(kspring),
                  int(scheme))


def build(force: bool = False) -> str:
    """Compile bd_oracle.c into libbd_oracle.so (gcc, -O2, OpenMP)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_rpy_block.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp]
        L.or_assemble.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
        L.or_cholesky.argtypes = [ctypes.c_int, dp, dp]
        L.or_cholesky.restype = ctypes.c_int
        L.or_trmv_lower.argtypes = [ctypes.c_int, dp, dp, dp]
        L.or_gemv.argtypes = [ctypes.c_int, dp, dp, dp]
        L.or_trsv_lower_t.argtypes = [ctypes.c_int, dp, dp, dp]
        L.or_tangent_project.argtypes = [ctypes.c_int, dp, dp, dp]
        L.or_kappa.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        L.or_factor_residual.argtypes = [ctypes.c_int, dp, dp]
        L.or_factor_residual.restype = ctypes.c_double
        L.or_tension_solve.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, dp, dp, ip]
        L.or_tension_solve.restype = ctypes.c_int
        L.or_step.argtypes = [ctypes.POINTER(Params), ctypes.c_int, dp, dp, dp, ip, dp]
        L.or_step.restype = ctypes.c_int
        L.or_run.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ip, dp, ctypes.c_int,
                             dp, dp, ip, ip, dp]
        L.or_observables.argtypes = [ctypes.c_int, dp, dp, dp]
        L.or_fraenkel_update.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                         dp, dp, dp, dp]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def num_threads() -> int:
    return lib().or_num_threads()


def rpy_block(R, hstar, a):
    R = np.ascontiguousarray(R, dtype=np.float64)
    out = np.zeros(9)
    lib().or_rpy_block(_d(R), hstar, a, _d(out))
    return out.reshape(3, 3)


def assemble(r, hstar, a=0.0):
    """Dense 3N x 3N diffusion tensor, Sec. 3 Eqs. (7)-(9)."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    N = r.shape[0]
    D = np.zeros((3 * N, 3 * N))
    lib().or_assemble(N, _d(r), hstar, a, _d(D))
    return D


def cholesky(D):
    """Unblocked Cholesky, Sec. 3 Eq. (10).  Returns (L, status)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    L = np.zeros_like(D)
    st = lib().or_cholesky(D.shape[0], _d(D), _d(L))
    return L, st


def trmv_lower(L, x):
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.zeros_like(x)
    lib().or_trmv_lower(L.shape[0], _d(L), _d(x), _d(y))
    return y


def trsv_lower_t(L, x):
    """z = L^{-T} x (back substitution with the transpose of lower-triangular L)."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    z = np.zeros_like(x)
    lib().or_trsv_lower_t(L.shape[0], _d(L), _d(x), _d(z))
    return z


def tangent_project(r, y):
    """Orthogonal projection of a bead displacement y onto the tangent space of
    the rod constraints |Q_k| = 1 at positions r."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1, 3)
    out = np.zeros_like(y)
    lib().or_tangent_project(r.shape[0], _d(r), _d(y), _d(out))
    return out


def gemv(A, x):
    A = np.ascontiguousarray(A, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.zeros_like(x)
    lib().or_gemv(A.shape[0], _d(A), _d(x), _d(y))
    return y


def kappa(flow, rate):
    k = np.zeros(9)
    lib().or_kappa(flow, rate, _d(k))
    return k.reshape(3, 3)


def factor_residual(D, L):
    D = np.ascontiguousarray(D, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    return lib().or_factor_residual(D.shape[0], _d(D), _d(L))


def tension_solve(D, rstar, u, dt, tol=1e-13, max_newton=50):
    """Newton for the rod tensions (rigid limit of Eqs. (13)-(17)).
    Returns (T, r(T), status, iterations)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    rstar = np.ascontiguousarray(rstar, dtype=np.float64).reshape(-1, 3)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
    N = rstar.shape[0]
    T = np.zeros(max(N - 1, 1))
    rout = np.zeros_like(rstar)
    it = ctypes.c_int(0)
    st = lib().or_tension_solve(N, _d(D), _d(rstar), _d(u), dt, tol, max_newton,
                                _d(T), _d(rout), ctypes.byref(it))
    return T[: N - 1], rout, st, it.value


def step(params: Params, r, xi):
    """One time step of one chain.  Returns (r_new, T, status, iters, maxdev)."""
    r = np.array(r, dtype=np.float64).reshape(-1, 3)
    xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, 3)
    N = r.shape[0]
    T = np.zeros(max(N - 1, 1))
    it = ctypes.c_int(0)
    md = ctypes.c_double(0.0)
    st = lib().or_step(ctypes.byref(params), N, _d(r), _d(xi), _d(T),
                       ctypes.byref(it), ctypes.byref(md))
    return r, T[: N - 1], st, it.value, md.value


def run(params: Params, Nc, r, noise):
    """n_steps steps for a batch.  r: [sum N, 3]; noise: [n_steps, sum N, 3].
    Returns (r_new, T, status, iters, maxdev)."""
    Nc = np.ascontiguousarray(Nc, dtype=np.int32)
    r = np.array(r, dtype=np.float64).reshape(-1, 3)
    noise = np.ascontiguousarray(noise, dtype=np.float64)
    n_steps = noise.shape[0] if noise.ndim == 3 else 0
    nc = Nc.shape[0]
    T = np.zeros(max(int(Nc.sum()) - nc, 1))
    status = np.zeros(nc, dtype=np.int32)
    iters = np.zeros(nc, dtype=np.int32)
    maxdev = np.zeros(nc)
    lib().or_run(ctypes.byref(params), nc, _i(Nc), _d(r), n_steps,
                 _d(noise) if n_steps else None, _d(T), _i(status), _i(iters), _d(maxdev))
    return r, T[: int(Nc.sum()) - nc], status, iters, maxdev


def fraenkel_update(D, kappa_, dt, kspring, r, y):
    """Semi-implicit Fraenkel-spring update (Sec. 3 eqQ2, Eqs. (23)-(25)) of
    one chain from positions r and scaled Brownian displacement y.
    Returns (r_new, T) with T_k = K* (|Q_k| - 1) / |Q_k| at the new links."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    kap = np.ascontiguousarray(kappa_, dtype=np.float64).reshape(9)
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1, 3)
    N = r.shape[0]
    rn = np.zeros_like(r)
    T = np.zeros(max(N - 1, 1))
    lib().or_fraenkel_update(N, _d(D), _d(kap), float(dt), float(kspring), _d(r), _d(y), _d(rn), _d(T))
    return rn, T[: N - 1]


def observables(r, T=None):
    """Per-chain observables of Sec. 5 Eqs. (25)-(29); T: tensions of the rods."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(OBS_STRIDE)
    Tp = None
    if T is not None:
        T = np.ascontiguousarray(T, dtype=np.float64)
        Tp = _d(T)
    lib().or_observables(r.shape[0], _d(r), Tp, _d(out))
    return out
