"""The paper's own constraint mode on the GPU: Fraenkel springs with the
semi-implicit link update of Sec. 3 (Eq. (3), eqQ2, Eqs. (23)-(25)), against
the FP64 oracle on the same seeded inputs."""
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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def run_both(bd, Nc, steps, seed, precision=0, **phys):
    Nc = np.asarray(Nc, np.int32)
    r0 = inputs.random_walk(Nc, seed)
    noise = inputs.gaussian_noise(steps, int(Nc.sum()), seed + 1)
    kw = dict(h_star=phys.get("hstar", 0.25), dt=phys.get("dt", 1e-4), flow=phys.get("flow", 0),
              Wi=phys.get("Wi", 0.0), k_spring=phys.get("K", 1e4))
    ctx = bd.Context(Nc, precision=precision, constraint=bd.FRAENKEL, **kw)
    ctx.set_state(cuda(r0))
    ctx.step(cuda(noise))
    r_gpu = ctx.get_state().cpu().numpy()
    obs, st = ctx.observables()
    T_gpu = ctx.tensions().cpu().numpy()
    nl = ctx.kernel_launches()
    ctx.close()
    p = orc.make_params(hstar=kw["h_star"], dt=kw["dt"], flow=kw["flow"], Wi=kw["Wi"],
                        constraint=orc.FRAENKEL, kspring=kw["k_spring"])
    r_ref, T_ref, st_ref, it_ref, md_ref = orc.run(p, Nc, r0, noise)
    return r0, r_gpu, r_ref, st, st_ref, obs.cpu().numpy(), T_gpu, T_ref, nl


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1.0)


def test_fraenkel_parity_uneven_shear_100_steps(bd):
    """Ragged batch (tile tails, a dumbbell), K* = 1e4, dt = 1e-4, shear
    Wi = 100, 100 steps: positions to 1e-10, spring coefficients and the
    Kramers stress against the oracle."""
    Nc = [2, 17, 65, 100, 33]
    r0, rg, rr, st, str_, obs, Tg, Tr, nl = run_both(bd, Nc, 100, 501, flow=1, Wi=100.0)
    assert (st == 0).all() and (str_ == 0).all()
    assert rel(rg, rr) < 1e-10
    np.testing.assert_allclose(Tg, Tr, rtol=1e-7, atol=1e-7 * np.abs(Tr).max())
    off = np.concatenate([[0], np.cumsum(Nc)])
    toff = np.concatenate([[0], np.cumsum(np.array(Nc) - 1)])
    for c in range(len(Nc)):
        ref = orc.observables(rr[off[c]:off[c + 1]], Tr[toff[c]:toff[c + 1]])
        np.testing.assert_allclose(obs[c, :6], ref[:6], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(obs[c, 8:12], ref[8:12], rtol=1e-6, atol=1e-6 * np.abs(ref[8:12]).max())
    assert nl > 0


def test_fraenkel_parity_equilibrium_paper_settings(bd):
    """The paper's equilibrium settings (dt = 1e-3, K* = 1000, h* = 0.25), 50 steps."""
    r0, rg, rr, st, str_, obs, Tg, Tr, nl = run_both(bd, [40, 41], 50, 503, dt=1e-3, K=1000.0)
    assert (st == 0).all()
    assert rel(rg, rr) < 1e-10


def test_fraenkel_mixed_close_to_fp64(bd):
    """Mixed precision (TF32 factor with refinement, FP32 storage) against
    the FP64 Fraenkel path on the same noise: one step stays within the
    factor's error (relative displacement error < 1e-3)."""
    Nc = np.array([300, 257], np.int32)
    r0 = inputs.random_walk(Nc, 505)
    noise = cuda(inputs.gaussian_noise(1, int(Nc.sum()), 506))
    out = []
    for prec in (bd.FP64, bd.MIXED_TF32):
        ctx = bd.Context(Nc, precision=prec, constraint=bd.FRAENKEL, k_spring=1e4, flow=2, Wi=10.0)
        ctx.set_state(cuda(r0))
        ctx.step(noise)
        st, _ = ctx.chain_status()
        assert (st == 0).all()
        out.append(ctx.get_state().cpu().numpy() - r0)
        ctx.close()
    assert np.abs(out[1] - out[0]).max() / np.abs(out[0]).max() < 1e-3


def test_fraenkel_not_pd_chain_frozen(bd):
    good = inputs.random_walk([10], 3)
    bad = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 0, 0]], float)
    r0 = np.concatenate([good, bad])
    ctx = bd.Context([10, 4], constraint=bd.FRAENKEL)
    ctx.set_state(cuda(r0))
    ctx.step(cuda(inputs.gaussian_noise(2, 14, 4)))
    r1 = ctx.get_state().cpu().numpy()
    obs, st = ctx.observables()
    assert st[0] == 0 and st[1] == bd.binding.BD_ERR_NOT_PD
    np.testing.assert_array_equal(r1[10:], bad)
    assert np.abs(r1[:10] - good).max() > 0
    ctx.close()


def test_fraenkel_profiled_step_equals_graph_step(bd):
    Nc = np.array([120, 64], np.int32)
    r0 = inputs.random_walk(Nc, 507)
    noise = cuda(inputs.gaussian_noise(1, int(Nc.sum()), 508))
    out = []
    for prof in (False, True):
        ctx = bd.Context(Nc, precision=bd.MIXED_TF32, constraint=bd.FRAENKEL, flow=1, Wi=50.0)
        ctx.set_state(cuda(r0))
        if prof:
            tl = ctx.profile_step(noise[0])
            assert tl["step"] > 0 and tl["factor"] > 0
        else:
            ctx.step(noise)
        out.append(ctx.get_state().cpu().numpy())
        ctx.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_fraenkel_adjoint_rejected(bd):
    ctx = bd.Context([10], constraint=bd.FRAENKEL)
    r0 = cuda(inputs.random_walk([10], 1))
    with pytest.raises(bd.BDError):
        ctx.adjoint(r0, cuda(inputs.gaussian_noise(2, 10, 2)), torch.zeros_like(r0))
    ctx.close()
