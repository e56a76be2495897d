"""Pathwise gradients of the mean chain stretch with respect to Wi and h*
(bd_adjoint, forward-mode tangents of the FP64 step) against central finite
differences (step 1e-5) of the GPU path and of the FP64 CPU oracle."""
import numpy as np
import pytest

import oracle as orc
from paper_2208_06559_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NC = np.array([12, 20, 7], np.int32)
STEPS, DT, WI, HS, FD = 15, 1e-3, 5.0, 0.25, 1e-5
SCHEME = 1  # the Euler rigid-rod step (the tangents follow that step map)


@pytest.fixture(scope="module")
def bd():
    from paper_2208_06559_gb300 import build as b
    b.build()
    import paper_2208_06559_gb300 as pkg
    pkg.lib()
    return pkg


def stretch_and_grad(r, Nc):
    """J = mean_c |r_{N-1} - r_0| / (N - 1) and dJ/dr."""
    off = np.concatenate([[0], np.cumsum(Nc)])
    g = np.zeros_like(r)
    J = 0.0
    for c, N in enumerate(Nc):
        R = r[off[c + 1] - 1] - r[off[c]]
        nr = np.linalg.norm(R)
        J += nr / (N - 1)
        g[off[c + 1] - 1] += R / nr / (N - 1)
        g[off[c]] -= R / nr / (N - 1)
    return J / len(Nc), g / len(Nc)


def gpu_run(bd, r0, noise, Wi, hs):
    ctx = bd.Context(NC, h_star=hs, dt=DT, flow=bd.FLOW_UNIAXIAL, Wi=Wi, scheme=SCHEME)
    ctx.set_state(torch.from_numpy(r0).cuda())
    ctx.step(torch.from_numpy(noise).cuda())
    r = ctx.get_state().cpu().numpy()
    st, _ = ctx.chain_status()
    ctx.close()
    assert (st == 0).all()
    return r


def oracle_run(r0, noise, Wi, hs):
    p = orc.make_params(hstar=hs, dt=DT, flow=orc.FLOW_UNIAXIAL, Wi=Wi, scheme=SCHEME)
    r, _, st, _, _ = orc.run(p, NC, r0, noise)
    assert (st == 0).all()
    return r


def test_adjoint_matches_finite_differences(bd):
    r0 = inputs.random_walk(NC, 501)
    noise = inputs.gaussian_noise(STEPS, int(NC.sum()), 502)
    ctx = bd.Context(NC, h_star=HS, dt=DT, flow=bd.FLOW_UNIAXIAL, Wi=WI, scheme=SCHEME)
    r_fin = gpu_run(bd, r0, noise, WI, HS)
    J0, dJdr = stretch_and_grad(r_fin, NC)
    gw, gh = ctx.adjoint(torch.from_numpy(r0).cuda(), torch.from_numpy(noise).cuda(),
                         torch.from_numpy(dJdr).cuda())
    # the context ends at the final state of the same path
    np.testing.assert_allclose(ctx.get_state().cpu().numpy(), r_fin, rtol=0, atol=1e-12)
    ctx.close()
    Jg = lambda w, h: stretch_and_grad(gpu_run(bd, r0, noise, w, h), NC)[0]
    Jo = lambda w, h: stretch_and_grad(oracle_run(r0, noise, w, h), NC)[0]
    fd_gpu = ((Jg(WI + FD, HS) - Jg(WI - FD, HS)) / (2 * FD), (Jg(WI, HS + FD) - Jg(WI, HS - FD)) / (2 * FD))
    fd_orc = ((Jo(WI + FD, HS) - Jo(WI - FD, HS)) / (2 * FD), (Jo(WI, HS + FD) - Jo(WI, HS - FD)) / (2 * FD))
    for got, a, b in zip((gw, gh), fd_gpu, fd_orc):
        assert abs(got - a) <= 1e-6 * abs(a), (got, a)
        assert abs(got - b) <= 1e-6 * abs(b), (got, b)


def test_autograd_function(bd):
    r0 = torch.from_numpy(inputs.random_walk(NC, 503)).cuda()
    noise = torch.from_numpy(inputs.gaussian_noise(8, int(NC.sum()), 504)).cuda()
    Wi = torch.tensor(WI, dtype=torch.float64, requires_grad=True)
    hs = torch.tensor(HS, dtype=torch.float64, requires_grad=True)
    r = bd.binding.simulate(Wi, hs, NC, r0, noise, dt=DT, scheme=SCHEME)
    off = np.concatenate([[0], np.cumsum(NC)])
    J = sum((r[off[c + 1] - 1] - r[off[c]]).norm() / (N - 1) for c, N in enumerate(NC)) / len(NC)
    J.backward()
    ctx = bd.Context(NC, h_star=HS, dt=DT, flow=bd.FLOW_UNIAXIAL, Wi=WI, scheme=SCHEME)
    _, dJdr = stretch_and_grad(r.detach().cpu().numpy(), NC)
    gw, gh = ctx.adjoint(r0, noise, torch.from_numpy(dJdr).cuda())
    ctx.close()
    np.testing.assert_allclose([Wi.grad.item(), hs.grad.item()], [gw, gh], rtol=1e-12)


def test_adjoint_rejects_mixed_precision(bd):
    ctx = bd.Context(NC, precision=bd.MIXED_TF32)
    r0 = torch.from_numpy(inputs.random_walk(NC, 505)).cuda()
    noise = torch.zeros((2, int(NC.sum()), 3), dtype=torch.float64, device="cuda")
    with pytest.raises(bd.BDError):
        ctx.adjoint(r0, noise, torch.zeros_like(r0))
    ctx.close()
