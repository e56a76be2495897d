"""Thin Python binding of libbd (include/bd.h): argument marshalling only.

Every stage of the time step runs in the library's CUDA kernels.  PyTorch
provides device memory (tensors) and streams; nothing here computes physics.
If libbd.so has not been built, loading raises immediately: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbd.so")

BD_OK = 0
BD_ERR_ARG = -1
BD_ERR_CUDA = -2
BD_ERR_OOM = -3
BD_ERR_NOT_PD = -4
BD_ERR_CONSTRAINT = -5
BD_ERR_TIMEOUT = -6
BD_ERR_STATE = -7

FLOW_NONE, FLOW_SHEAR, FLOW_UNIAXIAL = 0, 1, 2
FP64, MIXED_TF32, MIXED_BF16 = 0, 1, 2
RIGID, FRAENKEL = 0, 1
SCHEME_MIDPOINT, SCHEME_EULER = 0, 1
OBS_STRIDE = 12
# column indices of the observables row (include/bd.h BD_OBS_*)
OBS_REE_X, OBS_R2, OBS_RG2, OBS_STRETCH, OBS_MAXDEV, OBS_NEWTON = 0, 3, 4, 5, 6, 7
OBS_TAU_XX, OBS_TAU_YY, OBS_TAU_ZZ, OBS_TAU_XY = 8, 9, 10, 11

_lib = None


class Params(ctypes.Structure):
    _fields_ = [
        ("n_chains", ctypes.c_int),
        ("n_beads", ctypes.POINTER(ctypes.c_int)),
        ("h_star", ctypes.c_double),
        ("a", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("flow", ctypes.c_int),
        ("Wi", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("constraint", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("max_newton", ctypes.c_int),
        ("refine", ctypes.c_int),
        ("k_spring", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("lanes", ctypes.c_int),
    ]


EXPORTS = {
    "bd_params_default": (None, [ctypes.POINTER(Params)]),
    "bd_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]),
    "bd_destroy": (None, [ctypes.c_void_p]),
    "bd_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bd_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bd_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "bd_observables": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "bd_chain_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "bd_factor_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_double)]),
    "bd_assemble": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "bd_factor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "bd_brownian": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "bd_mobility_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "bd_get_tensions": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bd_midpoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "bd_read_matrix": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_void_p]),
    "bd_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "bd_kernel_launches": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ulonglong),
                                          ctypes.c_void_p]),
    "bd_lanes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "bd_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "bd_profile_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double)]),
    "bd_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                  ctypes.c_void_p]),
    "bd_tune_factor": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_void_p]),
    "bd_set_factor_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "bd_mobility_apply_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
}
STATIC_MAX_BEADS = 1024


def lib():
    """Load libbd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class BDError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {lib().bd_strerror(code).decode()} ({code})")
        self.code = code


def _check(code: int, what: str) -> int:
    if code != BD_OK:
        raise BDError(code, what)
    return code


def _stream(stream) -> ctypes.c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _f64(t, what: str, numel: int, device: Optional[int] = None, host_ok: bool = False):
    """Check a tensor before its pointer goes to the library: float64,
    contiguous, at least `numel` elements, and on the context's CUDA device
    (or in host memory where the call accepts it).  The library sees only a
    pointer, so a wrong element type or a short buffer would be read past its
    end; this raises instead."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: expected a torch.Tensor, got {type(t).__name__}")
    if t.dtype != torch.float64:
        raise ValueError(f"{what}: expected float64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: the tensor must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{what}: {t.numel()} elements, {numel} needed")
    if t.is_cuda:
        if device is not None and t.device.index != device:
            raise ValueError(f"{what}: tensor on cuda:{t.device.index}, context on cuda:{device}")
    elif not host_ok:
        raise ValueError(f"{what}: expected a CUDA tensor")
    return t


def mobility_apply_static(r, f, h_star: float = 0.25, a: float = 0.0, out=None, stream=None):
    """u = D(r) f for one chain through the allocation-free entry point
    (positions r and forces f: CUDA float64 [N, 3], N <= STATIC_MAX_BEADS)."""
    import torch
    n = 3 * int(r.shape[0])
    _f64(r, "mobility_apply_static: r", n)
    _f64(f, "mobility_apply_static: f", n, device=r.device.index)
    if out is None:
        out = torch.empty_like(f)
    _f64(out, "mobility_apply_static: out", n, device=r.device.index)
    # the library works on the current device and its scratch array there
    with torch.cuda.device(r.device):
        st = stream if stream is not None else torch.cuda.current_stream(r.device)
        _check(lib().bd_mobility_apply_static(_ptr(r), int(r.shape[0]), float(h_star), float(a),
                                              _ptr(f), _ptr(out), _stream(st)),
               "bd_mobility_apply_static")
    return out


class Context:
    """A batch of bead-rod chains held by one libbd context on one GPU.

    Positions, noise and forces are torch float64 tensors shaped [sum N, 3]
    (noise [n_steps, sum N, 3]) on the CUDA device, or on the CPU for
    ``step`` (host noise is copied by the library)."""

    def __init__(self, n_beads: Sequence[int], h_star: float = 0.25, dt: float = 1e-4,
                 flow: int = FLOW_NONE, Wi: float = 0.0, lam: float = 1.0, a: float = 0.0,
                 precision: int = FP64, tol: float = 1e-13, max_newton: int = 50,
                 refine: int = 1, constraint: int = RIGID, k_spring: float = 1e4,
                 scheme: int = SCHEME_MIDPOINT, lanes: int = 0):
        import torch
        L = lib()
        # the library's current device at creation (without CUDA, bd_create reports the error)
        self.device = torch.cuda.current_device() if torch.cuda.is_available() else None
        self.n_beads = np.ascontiguousarray(np.asarray(n_beads, dtype=np.int32))
        self.n_chains = int(self.n_beads.shape[0])
        self.total_beads = int(self.n_beads.sum())
        self.total_rods = self.total_beads - self.n_chains
        p = Params()
        L.bd_params_default(ctypes.byref(p))
        p.n_chains = self.n_chains
        p.n_beads = self.n_beads.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        p.h_star, p.a, p.dt = float(h_star), float(a), float(dt)
        p.flow, p.Wi, p.lambda_ = int(flow), float(Wi), float(lam)
        p.precision, p.tol, p.max_newton, p.refine = int(precision), float(tol), int(max_newton), int(refine)
        p.constraint, p.k_spring, p.scheme = int(constraint), float(k_spring), int(scheme)
        p.lanes = int(lanes)
        h = ctypes.c_void_p()
        _check(L.bd_create(ctypes.byref(p), ctypes.byref(h)), "bd_create")
        self._h = h
        self.precision = int(precision)
        self.constraint = int(constraint)
        self.scheme = int(scheme)

    def close(self):
        if getattr(self, "_h", None):
            lib().bd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state ---------------------------------------------------------
    def set_state(self, r, stream=None):
        _f64(r, "set_state", 3 * self.total_beads, self.device)
        _check(lib().bd_set_state(self._h, _ptr(r), _stream(stream)), "bd_set_state")

    def get_state(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.total_beads, 3), dtype=torch.float64, device=f"cuda:{self.device}")
        _f64(out, "get_state", 3 * self.total_beads, self.device)
        _check(lib().bd_get_state(self._h, _ptr(out), _stream(stream)), "bd_get_state")
        return out

    # -- the step ------------------------------------------------------
    def step(self, noise, n_steps: Optional[int] = None, stream=None):
        """Advance n_steps time steps with noise [n_steps, sum N, 3] (device or host)."""
        if n_steps is None:
            n_steps = int(noise.shape[0])
        _f64(noise, "step: noise", int(n_steps) * self.total_beads * 3, self.device, host_ok=True)
        _check(lib().bd_step(self._h, int(n_steps), _ptr(noise), _stream(stream)), "bd_step")

    def observables(self, out=None, stream=None, with_status: bool = True):
        import torch
        if out is None:
            out = torch.empty((self.n_chains, OBS_STRIDE), dtype=torch.float64, device=f"cuda:{self.device}")
        _f64(out, "observables", self.n_chains * OBS_STRIDE, self.device, host_ok=True)
        st = np.zeros(self.n_chains, dtype=np.int32) if with_status else None
        rc = lib().bd_observables(self._h, _ptr(out),
                                  st.ctypes.data_as(ctypes.c_void_p) if st is not None else None,
                                  _stream(stream))
        if rc not in (BD_OK, BD_ERR_NOT_PD, BD_ERR_CONSTRAINT):
            _check(rc, "bd_observables")
        return out, st

    def chain_status(self, stream=None):
        st = np.zeros(self.n_chains, dtype=np.int32)
        it = np.zeros(self.n_chains, dtype=np.int32)
        lib().bd_chain_status(self._h, st.ctypes.data_as(ctypes.c_void_p),
                              it.ctypes.data_as(ctypes.c_void_p), _stream(stream))
        return st, it

    def kernel_launches(self, stream=None) -> int:
        v = ctypes.c_ulonglong()
        _check(lib().bd_kernel_launches(self._h, ctypes.byref(v), _stream(stream)),
               "bd_kernel_launches")
        return int(v.value)

    def lanes(self) -> int:
        """Concurrent sub-batches the library steps this context's chains in."""
        v = ctypes.c_int()
        _check(lib().bd_lanes(self._h, ctypes.byref(v)), "bd_lanes")
        return int(v.value)

    PROFILE_STAGES = ("assemble", "factor", "brownian", "k_wait_predictor", "tension",
                      "commit", "step", "k_chain_end")

    def profile_step(self, noise, newton_iters: int = 0) -> dict:
        """One step launched kernel by kernel with stage-boundary events:
        {stage: ms}, keys PROFILE_STAGES (k_chain_end from the step start)."""
        import torch
        _f64(noise, "profile_step: noise", 3 * self.total_beads, self.device)
        torch.cuda.synchronize()  # earlier work on other streams (e.g. set_state) is finished
        out = (ctypes.c_double * 8)()
        _check(lib().bd_profile_step(self._h, _ptr(noise), int(newton_iters), out), "bd_profile_step")
        return dict(zip(self.PROFILE_STAGES, list(out)))

    def adjoint(self, r0, noise, dJdr_final, ckpt_every: int = 20, stream=None):
        """(dJ/dWi, dJ/dh*) at fixed noise for J with gradient dJdr_final at the
        final positions; the context ends at the final state."""
        n = 3 * self.total_beads
        _f64(r0, "adjoint: r0", n, self.device)
        _f64(noise, "adjoint: noise", int(noise.shape[0]) * n, self.device)
        _f64(dJdr_final, "adjoint: dJdr_final", n, self.device)
        g = (ctypes.c_double * 2)()
        rc = lib().bd_adjoint(self._h, _ptr(r0), int(noise.shape[0]), _ptr(noise), int(ckpt_every),
                              _ptr(dJdr_final), g, _stream(stream))
        if rc not in (BD_OK,):
            _check(rc, "bd_adjoint")
        return float(g[0]), float(g[1])

    def tune_factor(self, cache_path: Optional[str] = None, stream=None):
        """Pick the mixed factorisation's super-panel width and chain-group
        count by timing (bd_tune_factor), or reuse the entry of a JSON cache
        keyed by the padded order, chain count and precision.  Returns
        (panel, groups, ms) (ms is None for a cached entry)."""
        import json
        n_pad = int(-(-3 * int(self.n_beads.max()) // 128) * 128)
        key = f"prec{self.precision}:np{n_pad}:chains{self.n_chains}"
        cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        if key in cache:
            p, g = cache[key]["panel"], cache[key]["groups"]
            _check(lib().bd_set_factor_config(self._h, int(p), int(g)), "bd_set_factor_config")
            return p, g, None
        p, g, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().bd_tune_factor(self._h, ctypes.byref(p), ctypes.byref(g), ctypes.byref(ms),
                                    _stream(stream)), "bd_tune_factor")
        if cache_path:
            cache[key] = {"panel": p.value, "groups": g.value, "ms": ms.value}
            tmp = cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
            os.replace(tmp, cache_path)
        return p.value, g.value, ms.value

    def factor_residual(self, chain: int) -> float:
        v = ctypes.c_double()
        _check(lib().bd_factor_residual(self._h, int(chain), ctypes.byref(v)), "bd_factor_residual")
        return v.value

    # -- stages ----------------------------------------------------------
    def assemble(self, stream=None):
        _check(lib().bd_assemble(self._h, _stream(stream)), "bd_assemble")

    def factor(self, stream=None):
        _check(lib().bd_factor(self._h, _stream(stream)), "bd_factor")

    def brownian(self, xi, stream=None):
        import torch
        _f64(xi, "brownian: xi", 3 * self.total_beads, self.device)
        y = torch.empty_like(xi)
        _check(lib().bd_brownian(self._h, _ptr(xi), _ptr(y), _stream(stream)), "bd_brownian")
        return y

    def mobility_apply(self, f, stream=None):
        import torch
        _f64(f, "mobility_apply: f", 3 * self.total_beads, self.device)
        u = torch.empty_like(f)
        _check(lib().bd_mobility_apply(self._h, _ptr(f), _ptr(u), _stream(stream)),
               "bd_mobility_apply")
        return u

    def midpoint(self, xi, stream=None):
        """Midpoint stage of the corrected rigid-rod step (after assemble and
        factor): (r_m, y) with r_m = r + P y_B / 2 and y the step's Brownian
        displacement sqrt(2 dt) D(r_m) B^{-T} xi."""
        import torch
        _f64(xi, "midpoint: xi", 3 * self.total_beads, self.device)
        rm = torch.empty_like(xi)
        y = torch.empty_like(xi)
        _check(lib().bd_midpoint(self._h, _ptr(xi), _ptr(rm), _ptr(y), _stream(stream)), "bd_midpoint")
        return rm, y

    def tensions(self, stream=None):
        import torch
        T = torch.zeros(max(self.total_rods, 1), dtype=torch.float64, device=f"cuda:{self.device}")
        _check(lib().bd_get_tensions(self._h, _ptr(T), _stream(stream)), "bd_get_tensions")
        return T[: self.total_rods]

    def read_matrix(self, chain: int, which: int) -> np.ndarray:
        import torch
        torch.cuda.synchronize()
        n = 3 * int(self.n_beads[chain])
        out = np.zeros((n, n), dtype=np.float64)
        _check(lib().bd_read_matrix(self._h, int(chain), int(which),
                                    out.ctypes.data_as(ctypes.c_void_p)), "bd_read_matrix")
        return out


def simulate(Wi, h_star, n_beads, r0, noise, dt: float = 1e-4, flow: int = FLOW_UNIAXIAL,
             lam: float = 1.0, tol: float = 1e-13, max_newton: int = 50, ckpt_every: int = 20,
             scheme: int = SCHEME_MIDPOINT):
    """Final positions after noise.shape[0] FP64 steps from r0, differentiable
    with respect to the 0-dim float64 tensors Wi and h_star (a = h_star).

    The backward pass calls bd_adjoint with the incoming gradient at the final
    positions; the noise is held fixed (pathwise derivative)."""
    import torch

    class _Run(torch.autograd.Function):
        @staticmethod
        def forward(ctx_, wi, hs):
            c = Context(n_beads, h_star=float(hs), dt=dt, flow=flow, Wi=float(wi), lam=lam, tol=tol,
                        max_newton=max_newton, scheme=scheme)
            c.set_state(r0)
            c.step(noise)
            out = c.get_state()
            torch.cuda.synchronize()
            st, _ = c.chain_status()
            c.close()
            if (st != BD_OK).any():
                raise BDError(int(st.min()), "simulate")
            ctx_.save_for_backward(wi, hs)
            return out

        @staticmethod
        def backward(ctx_, grad_out):
            wi, hs = ctx_.saved_tensors
            c = Context(n_beads, h_star=float(hs), dt=dt, flow=flow, Wi=float(wi), lam=lam, tol=tol,
                        max_newton=max_newton, scheme=scheme)
            gw, gh = c.adjoint(r0, noise, grad_out.contiguous(), ckpt_every)
            c.close()
            return (torch.tensor(gw, dtype=wi.dtype, device=wi.device),
                    torch.tensor(gh, dtype=hs.dtype, device=hs.device))

    return _Run.apply(Wi, h_star)
