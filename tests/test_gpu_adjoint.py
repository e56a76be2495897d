"""Pathwise gradients of the mean chain stretch with respect to Wi and h*
(bd_adjoint, forward-mode tangents of the FP64 step, midpoint and Euler
rigid-rod steps) against central finite differences (step 1e-5) of the GPU
path and of the FP64 CPU oracle."""
import numpy as np
import pytest

import oracle as orc
from paper_2208_06559_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NC = np.array([12, 20, 7], np.int32)
STEPS, DT, WI, HS, FD = 15, 1e-3, 5.0, 0.25, 1e-5
SCHEMES = [0, 1]  # midpoint and Euler rigid-rod steps


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


def gpu_run(bd, r0, noise, Wi, hs, scheme, Nc=NC, dt=DT):
    ctx = bd.Context(Nc, h_star=hs, dt=dt, flow=bd.FLOW_UNIAXIAL, Wi=Wi, scheme=scheme)
    ctx.set_state(torch.from_numpy(r0).cuda())
    ctx.step(torch.from_numpy(noise).cuda())
    r = ctx.get_state().cpu().numpy()
    st, _ = ctx.chain_status()
    ctx.close()
    assert (st == 0).all()
    return r


def oracle_run(r0, noise, Wi, hs, scheme, Nc=NC, dt=DT):
    p = orc.make_params(hstar=hs, dt=dt, flow=orc.FLOW_UNIAXIAL, Wi=Wi, scheme=scheme)
    r, _, st, _, _ = orc.run(p, Nc, r0, noise)
    assert (st == 0).all()
    return r


@pytest.mark.parametrize("scheme", SCHEMES)
def test_adjoint_matches_finite_differences(bd, scheme):
    r0 = inputs.random_walk(NC, 501)
    noise = inputs.gaussian_noise(STEPS, int(NC.sum()), 502)
    ctx = bd.Context(NC, h_star=HS, dt=DT, flow=bd.FLOW_UNIAXIAL, Wi=WI, scheme=scheme)
    r_fin = gpu_run(bd, r0, noise, WI, HS, scheme)
    J0, dJdr = stretch_and_grad(r_fin, NC)
    gw, gh = ctx.adjoint(torch.from_numpy(r0).cuda(), torch.from_numpy(noise).cuda(),
                         torch.from_numpy(dJdr).cuda())
    # the context ends at the final state of the same path
    np.testing.assert_allclose(ctx.get_state().cpu().numpy(), r_fin, rtol=0, atol=1e-12)
    ctx.close()
    Jg = lambda w, h: stretch_and_grad(gpu_run(bd, r0, noise, w, h, scheme), NC)[0]
    Jo = lambda w, h: stretch_and_grad(oracle_run(r0, noise, w, h, scheme), NC)[0]
    fd_gpu = ((Jg(WI + FD, HS) - Jg(WI - FD, HS)) / (2 * FD), (Jg(WI, HS + FD) - Jg(WI, HS - FD)) / (2 * FD))
    fd_orc = ((Jo(WI + FD, HS) - Jo(WI - FD, HS)) / (2 * FD), (Jo(WI, HS + FD) - Jo(WI, HS - FD)) / (2 * FD))
    for got, a, b in zip((gw, gh), fd_gpu, fd_orc):
        assert abs(got - a) <= 1e-6 * abs(a), (got, a)
        assert abs(got - b) <= 1e-6 * abs(b), (got, b)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_autograd_function(bd, scheme):
    r0 = torch.from_numpy(inputs.random_walk(NC, 503)).cuda()
    noise = torch.from_numpy(inputs.gaussian_noise(8, int(NC.sum()), 504)).cuda()
    Wi = torch.tensor(WI, dtype=torch.float64, requires_grad=True)
    hs = torch.tensor(HS, dtype=torch.float64, requires_grad=True)
    r = bd.binding.simulate(Wi, hs, NC, r0, noise, dt=DT, scheme=scheme)
    off = np.concatenate([[0], np.cumsum(NC)])
    J = sum((r[off[c + 1] - 1] - r[off[c]]).norm() / (N - 1) for c, N in enumerate(NC)) / len(NC)
    J.backward()
    ctx = bd.Context(NC, h_star=HS, dt=DT, flow=bd.FLOW_UNIAXIAL, Wi=WI, scheme=scheme)
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


def test_adjoint_uneven_batch_workload(bd):
    """The uneven-batch workload: 128 chains with N drawn from U{50..500},
    uniaxial extension Wi = 5, dt = 1e-4, 50 midpoint steps.  The adjoint
    gradient of the mean stretch matches central finite differences of the
    GPU path to 1e-6 relative; on the four shortest chains it also matches
    central finite differences of the oracle."""
    Nc = inputs.uneven_lengths(128, 50, 500, 1239)
    steps, dt, wi = 50, 1e-4, 5.0
    r0 = inputs.random_walk(Nc, 1240)
    noise = inputs.gaussian_noise(steps, int(Nc.sum()), 1241)
    r_fin = gpu_run(bd, r0, noise, wi, HS, 0, Nc, dt)
    J0, dJdr = stretch_and_grad(r_fin, Nc)
    ctx = bd.Context(Nc, h_star=HS, dt=dt, flow=bd.FLOW_UNIAXIAL, Wi=wi)
    gw, gh = ctx.adjoint(torch.from_numpy(r0).cuda(), torch.from_numpy(noise).cuda(),
                         torch.from_numpy(dJdr).cuda())
    ctx.close()
    Jg = lambda w, h: stretch_and_grad(gpu_run(bd, r0, noise, w, h, 0, Nc, dt), Nc)[0]
    fd = ((Jg(wi + FD, HS) - Jg(wi - FD, HS)) / (2 * FD), (Jg(wi, HS + FD) - Jg(wi, HS - FD)) / (2 * FD))
    for got, want in zip((gw, gh), fd):
        assert abs(got - want) <= 1e-6 * abs(want), (got, want)
    # oracle on the four shortest chains (their own adjoint on the GPU)
    pick = np.argsort(Nc, kind="stable")[:4]
    off = np.concatenate([[0], np.cumsum(Nc)])
    sel = np.concatenate([np.arange(off[c], off[c + 1]) for c in pick])
    Ns = Nc[pick]
    r0s, nzs = r0[sel], np.ascontiguousarray(noise[:, sel])
    _, dJs = stretch_and_grad(gpu_run(bd, r0s, nzs, wi, HS, 0, Ns, dt), Ns)
    cs = bd.Context(Ns, h_star=HS, dt=dt, flow=bd.FLOW_UNIAXIAL, Wi=wi)
    gws, ghs = cs.adjoint(torch.from_numpy(r0s).cuda(), torch.from_numpy(nzs).cuda(), torch.from_numpy(dJs).cuda())
    cs.close()
    Jo = lambda w, h: stretch_and_grad(oracle_run(r0s, nzs, w, h, 0, Ns, dt), Ns)[0]
    fdo = ((Jo(wi + FD, HS) - Jo(wi - FD, HS)) / (2 * FD), (Jo(wi, HS + FD) - Jo(wi, HS - FD)) / (2 * FD))
    for got, want in zip((gws, ghs), fdo):
        assert abs(got - want) <= 1e-6 * abs(want), (got, want)


def test_adjoint_with_lanes_equals_one_batch(bd):
    """An FP64 context split into 2 or 3 lanes (concurrent sub-batches)
    returns the gradient of the single batch: every lane contributes its
    chains' part, reading its beads of the caller's noise; the final states
    agree as well."""
    Nc = np.array([12, 20, 7, 16, 9, 25], np.int32)
    r0 = inputs.random_walk(Nc, 511)
    noise = inputs.gaussian_noise(10, int(Nc.sum()), 512)
    r_fin = gpu_run(bd, r0, noise, WI, HS, 0, Nc)
    _, dJdr = stretch_and_grad(r_fin, Nc)
    res = {}
    for lanes in (1, 2, 3):
        ctx = bd.Context(Nc, h_star=HS, dt=DT, flow=bd.FLOW_UNIAXIAL, Wi=WI, lanes=lanes)
        assert ctx.lanes() == lanes
        g = ctx.adjoint(torch.from_numpy(r0).cuda(), torch.from_numpy(noise).cuda(), torch.from_numpy(dJdr).cuda())
        res[lanes] = (np.array(g), ctx.get_state().cpu().numpy())
        ctx.close()
    for lanes in (2, 3):
        np.testing.assert_allclose(res[lanes][0], res[1][0], rtol=1e-10)
        np.testing.assert_allclose(res[lanes][1], res[1][1], rtol=0, atol=1e-12)
