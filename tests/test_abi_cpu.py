"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/bd.h declares; argument validation and error
strings work without touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_06559_gb300 import build as b
    b.build()
    from paper_2208_06559_gb300 import binding
    return binding.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "bd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(bd_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("bd_create", "bd_destroy", "bd_set_state", "bd_get_state", "bd_step",
                 "bd_observables", "bd_factor_residual", "bd_strerror"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2208_06559_gb300 import binding
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in binding.EXPORTS, f"binding misses {name}"


def test_strerror_and_defaults(lib):
    from paper_2208_06559_gb300 import binding
    assert lib.bd_strerror(0) == b"ok"
    assert b"positive definite" in lib.bd_strerror(-4)
    p = binding.Params()
    lib.bd_params_default(ctypes.byref(p))
    assert p.n_chains == 1 and p.h_star == 0.25 and p.dt == 1e-4 and p.tol == 1e-13
    assert p.max_newton == 50 and p.precision == 0
    assert p.constraint == 0 and p.k_spring == 1e4 and p.scheme == 0 and p.lanes == 0


@pytest.mark.parametrize("mutate", [
    lambda p, nb: setattr(p, "n_chains", 0),
    lambda p, nb: setattr(p, "dt", 0.0),
    lambda p, nb: setattr(p, "h_star", -1.0),
    lambda p, nb: (setattr(p, "h_star", 0.5), setattr(p, "a", 0.25)),  # a < h*: not PD
    lambda p, nb: setattr(p, "flow", 7),
    lambda p, nb: setattr(p, "precision", 9),
    lambda p, nb: setattr(p, "precision", 2),   # BF16 operands: no such factorisation is built
    lambda p, nb: setattr(p, "scheme", 2),
    lambda p, nb: nb.__setitem__(0, 1),   # a chain needs >= 2 beads
    lambda p, nb: nb.__setitem__(1, 4097),  # past the FP64 path's per-chain limit of 4096 beads
    lambda p, nb: (setattr(p, "precision", 1), nb.__setitem__(1, 8193)),  # past the mixed path's 8192
    lambda p, nb: setattr(p, "dt", float("nan")),
    lambda p, nb: setattr(p, "h_star", float("nan")),
    lambda p, nb: setattr(p, "dt", float("inf")),
    lambda p, nb: setattr(p, "Wi", float("nan")),
    lambda p, nb: setattr(p, "lambda_", float("inf")),
    lambda p, nb: setattr(p, "tol", float("nan")),
    lambda p, nb: setattr(p, "constraint", 2),
    lambda p, nb: (setattr(p, "constraint", 1), setattr(p, "k_spring", 0.0)),  # Fraenkel needs K* > 0
    lambda p, nb: setattr(p, "lanes", -1),
    lambda p, nb: setattr(p, "lanes", 9),   # at most 8 concurrent sub-batches
])
def test_create_rejects_bad_arguments_before_any_device_call(lib, mutate):
    from paper_2208_06559_gb300 import binding
    nb = np.array([16, 20], np.int32)
    p = binding.Params()
    lib.bd_params_default(ctypes.byref(p))
    p.n_chains = 2
    mutate(p, nb)
    p.n_beads = nb.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    h = ctypes.c_void_p()
    assert lib.bd_create(ctypes.byref(p), ctypes.byref(h)) == binding.BD_ERR_ARG
    assert not h.value
    assert lib.bd_create(None, ctypes.byref(h)) == binding.BD_ERR_ARG
    assert lib.bd_step(None, 1, None, None) == binding.BD_ERR_ARG
    assert lib.bd_profile_step(None, None, 0, None) == binding.BD_ERR_ARG
    assert lib.bd_selftest_bounded_wait(0, None) == binding.BD_ERR_ARG
    lib.bd_destroy(None)


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2208_06559_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "bd_oracle" not in txt, f


def test_binding_checks_tensors_before_the_library_sees_them():
    """The binding hands the library bare pointers, so it checks element type,
    layout, size and placement first (no GPU needed: these all raise on the host)."""
    import torch
    from paper_2208_06559_gb300.binding import _f64
    ok = torch.zeros((4, 3), dtype=torch.float64)
    assert _f64(ok, "x", 12, host_ok=True) is ok
    with pytest.raises(TypeError):
        _f64(ok.numpy(), "x", 12, host_ok=True)
    with pytest.raises(ValueError, match="float64"):
        _f64(ok.float(), "x", 12, host_ok=True)
    with pytest.raises(ValueError, match="contiguous"):
        _f64(torch.zeros((3, 4), dtype=torch.float64).t(), "x", 12, host_ok=True)
    with pytest.raises(ValueError, match="needed"):
        _f64(ok, "x", 13, host_ok=True)
    with pytest.raises(ValueError, match="CUDA"):
        _f64(ok, "x", 12)


def test_binding_host_buffers_where_the_library_copies(monkeypatch):
    """bd_step and bd_observables take host memory (the library stages the
    copy), so the binding lets host noise and a host observables buffer
    through; positions must be on the device.  Run against a stub library:
    only the binding's own checks are exercised."""
    import torch
    from paper_2208_06559_gb300 import binding

    class _Stub:
        def __getattr__(self, name):
            return lambda *a, **k: b"stub" if name == "bd_strerror" else 0

    monkeypatch.setattr(binding, "_lib", _Stub())
    monkeypatch.setattr(binding, "_stream", lambda stream=None: ctypes.c_void_p(0))
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    ctx = binding.Context([5, 7])
    noise = torch.zeros((2, 12, 3), dtype=torch.float64)
    ctx.step(noise[0:1])
    ctx.observables(out=torch.empty((2, binding.OBS_STRIDE), dtype=torch.float64), with_status=False)
    with pytest.raises(ValueError, match="CUDA"):
        ctx.set_state(torch.zeros((12, 3), dtype=torch.float64))
    with pytest.raises(ValueError, match="float64"):
        ctx.step(noise.float()[0:1])
    with pytest.raises(ValueError, match="needed"):
        ctx.step(noise[0:1], n_steps=2 + 1)
    ctx._h = None
