"""The allocation-free mobility product (bd_mobility_apply_static).

It serves callers that cannot allocate device memory and so cannot create a
context; its scratch is a fixed device array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle as orc
from paper_2208_06559_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bd():
    from paper_2208_06559_gb300 import build as b
    b.build()
    import paper_2208_06559_gb300 as pkg
    pkg.lib()
    return pkg


@pytest.mark.parametrize("N,hs,a", [(700, 0.25, 0.0), (37, 0.5, 0.6), (1024, 0.25, 0.25), (2, 0.25, 0.0)])
def test_static_matches_context_product_two_calls(bd, N, hs, a):
    r = torch.from_numpy(inputs.random_walk([N], 100 + N)).cuda()
    ctx = bd.Context([N], h_star=hs, a=a)
    ctx.set_state(r)
    ctx.assemble()
    for call in range(2):   # two calls in a row share the scratch array
        f = torch.from_numpy(inputs.gaussian_noise(1, N, 200 + call)[0]).cuda()
        u_ref = ctx.mobility_apply(f)
        u = bd.binding.mobility_apply_static(r, f, h_star=hs, a=a)
        torch.cuda.synchronize()
        err = (u - u_ref).abs().max().item() / max(u_ref.abs().max().item(), 1.0)
        assert err < 1e-13, (call, err)
        # and against the FP64 oracle's assembled D times f
        u_orc = orc.gemv(orc.assemble(r.cpu().numpy(), hs, a), f.cpu().numpy().ravel())
        np.testing.assert_allclose(u.cpu().numpy().ravel(), u_orc, rtol=0,
                                   atol=1e-13 * max(np.abs(u_orc).max(), 1.0))
    ctx.close()


def test_static_rejects_oversize_and_bad_args(bd):
    L = bd.lib()
    N = bd.binding.STATIC_MAX_BEADS + 1
    r = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros_like(r)
    u = torch.zeros_like(r)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert L.bd_mobility_apply_static(p(r), N, 0.25, 0.0, p(f), p(u), None) == bd.binding.BD_ERR_ARG
    assert L.bd_mobility_apply_static(p(r), 0, 0.25, 0.0, p(f), p(u), None) == bd.binding.BD_ERR_ARG
    assert L.bd_mobility_apply_static(p(r), 10, 0.5, 0.25, p(f), p(u), None) == bd.binding.BD_ERR_ARG
    assert L.bd_mobility_apply_static(None, 10, 0.25, 0.0, p(f), p(u), None) == bd.binding.BD_ERR_ARG
    assert L.bd_mobility_apply_static(p(r), 10, float("inf"), 0.0, p(f), p(u), None) == bd.binding.BD_ERR_ARG
    assert L.bd_mobility_apply_static(p(r), 10, 0.25, float("inf"), p(f), p(u), None) == bd.binding.BD_ERR_ARG
    assert L.bd_mobility_apply_static(p(r), 10, float("nan"), 0.0, p(f), p(u), None) == bd.binding.BD_ERR_ARG
    host = torch.zeros((10, 3), dtype=torch.float64)   # host memory is not the current device's
    assert L.bd_mobility_apply_static(p(host), 10, 0.25, 0.0, p(f), p(u), None) == bd.binding.BD_ERR_ARG
