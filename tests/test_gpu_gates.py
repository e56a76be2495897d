"""Accuracy gates of the mixed-precision path at the headline shape.

64 chains of N = 1000 beads under simple shear Wi = 100, with the
factorisation shape the benchmark's tuner picks on that workload (super-panel
of 16 tiles, 4 chain groups; two super-panels over the 24 tile columns).

Tolerances (derived, not fitted):
  * TF32 operands carry a unit round-off of 2^-11 = 4.9e-4; the raw factor's
    backward error ||Lt Lt^T - D||_F / ||D||_F is of that order (1e-3 bound).
  * The refined factor B_eff = (Lt + D Lt^{-T}) / 2 satisfies
    B_eff B_eff^T - D = E D'^{-1} E / 4, E = D - Lt Lt^T: second order, so
    with ||E|| / ||D|| ~ 2e-4 and ||D'^{-1}|| ||D|| of order 10 the error is
    ~1e-7, inside the 1e-6 target.
  * The Brownian displacement differs from the FP64 one (L xi) by the first
    order of E: 1e-3 of the largest displacement bounds it elementwise.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2208_06559_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_BEADS, N_CHAINS, PANEL, GROUPS = 1000, 64, 16, 4
DT, WI = 1e-4, 100.0


@pytest.fixture(scope="module")
def bd():
    from paper_2208_06559_gb300 import build as b
    b.build()
    import paper_2208_06559_gb300 as pkg
    pkg.lib()
    return pkg


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def headline_context(bd, r0, precision):
    ctx = bd.Context(np.full(N_CHAINS, N_BEADS, np.int32), h_star=0.25, dt=DT, flow=bd.FLOW_SHEAR, Wi=WI,
                     precision=precision)
    if precision != bd.FP64:
        assert bd.lib().bd_set_factor_config(ctx._h, PANEL, GROUPS) == 0
    ctx.set_state(cuda(r0))
    return ctx


def test_refined_factor_against_the_oracle_d(bd):
    """(i) ||B_eff B_eff^T - D||_F / ||D||_F <= 1e-6 with B_eff formed in FP64
    from the library's tensor-core factor and the oracle's D; the raw factor
    is TF32-level and the library's own residual agrees with the host one."""
    Nc = np.full(N_CHAINS, N_BEADS, np.int32)
    r0 = inputs.random_walk(Nc, 1237)
    ctx = headline_context(bd, r0, bd.MIXED_TF32)
    ctx.assemble()
    ctx.factor()
    st, _ = ctx.chain_status()
    assert (st == 0).all(), st
    for c in (0, 37, 63):
        D = orc.assemble(r0[N_BEADS * c:N_BEADS * (c + 1)], 0.25, 0.25)
        Lt = ctx.read_matrix(c, 1)
        nD = np.linalg.norm(D)
        raw = np.linalg.norm(Lt @ Lt.T - D) / nD
        Linv_t = np.linalg.inv(Lt).T
        Beff = 0.5 * (Lt + D @ Linv_t)
        refined = np.linalg.norm(Beff @ Beff.T - D) / nD
        assert raw < 1e-3, (c, raw)
        assert refined <= 1e-6, (c, refined)
        lib_res = ctx.factor_residual(c)
        assert abs(lib_res - raw) <= 1e-2 * raw, (c, lib_res, raw)
    ctx.close()


def test_one_step_displacement_against_the_oracle(bd):
    """(ii) One step of all 64 chains at the headline shape; for three chains
    the displacement matches the FP64 oracle's step elementwise to 1e-3 of the
    largest displacement, and rods hold to 1e-10."""
    Nc = np.full(N_CHAINS, N_BEADS, np.int32)
    r0 = inputs.random_walk(Nc, 1237)
    noise = inputs.gaussian_noise(1, int(Nc.sum()), 1238)
    ctx = headline_context(bd, r0, bd.MIXED_TF32)
    ctx.step(cuda(noise))
    r1 = ctx.get_state().cpu().numpy()
    obs, st = ctx.observables()
    assert (st == 0).all(), st
    assert obs[:, bd.OBS_MAXDEV].max().item() < 1e-10
    ctx.close()
    pick = [0, 31, 63]
    sl = np.concatenate([np.arange(N_BEADS * c, N_BEADS * (c + 1)) for c in pick])
    nz = noise[:, sl]
    p = orc.make_params(hstar=0.25, dt=DT, flow=orc.FLOW_SHEAR, Wi=WI)
    rr, _, st_ref, _, _ = orc.run(p, np.full(len(pick), N_BEADS, np.int32), r0[sl], nz)
    assert (st_ref == 0).all()
    d_gpu, d_ref = r1[sl] - r0[sl], rr - r0[sl]
    err = np.abs(d_gpu - d_ref).max() / np.abs(d_ref).max()
    assert err < 1e-3, err


def test_ensemble_stretch_against_fp64(bd):
    """(iii) 8 chains x 200 steps of shear from the same state and noise:
    the ensemble <R^2> and mean stretch of the mixed path are within 3
    standard errors (over chains) of the FP64 path's, which matches the oracle
    to 1e-10 (test_gpu_parity); per chain the two differ only pathwise by the
    factor's first-order error."""
    Nc = np.full(8, N_BEADS, np.int32)
    r0 = inputs.random_walk(Nc, 1239)
    noise = cuda(inputs.gaussian_noise(200, int(Nc.sum()), 1240))
    res = {}
    for prec in (bd.FP64, bd.MIXED_TF32):
        ctx = bd.Context(Nc, h_star=0.25, dt=DT, flow=bd.FLOW_SHEAR, Wi=WI, precision=prec)
        ctx.set_state(cuda(r0))
        ctx.step(noise)
        obs, st = ctx.observables()
        assert (st == 0).all(), (prec, st)
        res[prec] = obs.cpu().numpy()
        ctx.close()
    for col in (bd.OBS_R2, bd.OBS_STRETCH):
        a, b = res[bd.MIXED_TF32][:, col], res[bd.FP64][:, col]
        se = b.std(ddof=1) / np.sqrt(len(b))
        assert abs(a.mean() - b.mean()) < 3 * se, (col, a.mean(), b.mean(), se)
        assert np.abs(a - b).max() < 1e-3 * np.abs(b).max(), col


@pytest.mark.parametrize("N", [4000, 4096])
def test_long_chain_one_step_mixed_against_fp64(bd, N):
    """(iv) One chain of N = 4000 beads (3N = 12000, 94 tiles of 128) and of
    the per-chain limit N = 4096 (3N = 12288 fills 96 tiles exactly, 4095 rods
    fill the tension solve) under uniaxial extension Wi = 50, dt = 5e-5: one
    mixed step against one FP64 step on the GPU (oracle-pinned path),
    elementwise to 1e-3 of the largest displacement; rods hold to 1e-10."""
    Nc = np.array([N], np.int32)
    r0 = inputs.random_walk(Nc, 1241)
    noise = cuda(inputs.gaussian_noise(1, N, 1242))
    out = {}
    for prec in (bd.FP64, bd.MIXED_TF32):
        ctx = bd.Context(Nc, h_star=0.25, dt=5e-5, flow=bd.FLOW_UNIAXIAL, Wi=50.0, precision=prec)
        ctx.set_state(cuda(r0))
        ctx.step(noise)
        obs, st = ctx.observables()
        assert (st == 0).all(), (prec, st)
        assert obs[:, bd.OBS_MAXDEV].max().item() < 1e-10
        out[prec] = ctx.get_state().cpu().numpy()
        ctx.close()
    d64 = out[bd.FP64] - r0
    err = np.abs(out[bd.MIXED_TF32] - out[bd.FP64]).max() / np.abs(d64).max()
    assert err < 1e-3, err


@pytest.mark.parametrize("N", [6000, 8192])
def test_chains_beyond_4096_beads(bd, N):
    """The mixed path takes chains of up to 8192 beads (3N = 24576, 192 tiles;
    the refinement's triangular solve on a cluster of four CTAs, the midpoint
    projection by serial elimination past 4095 rods).  One chain: the
    midpoint r_m matches r + P y / 2 computed here with a banded solve of
    (A A^T) x = A y from s Lt xi of the library's own factor (to the FP32
    summation error of its product, 1e-5 of the largest displacement), and two steps of uniaxial extension hold every rod to
    1e-10.  At N = 6000 the refined Brownian displacement also agrees with
    s L xi of an FP64 LAPACK factor of the oracle's D to the factor's
    first-order error."""
    sp = pytest.importorskip("scipy.linalg")
    Nc = np.array([N], np.int32)
    r0 = inputs.random_walk(Nc, 1243)
    xi = inputs.gaussian_noise(2, N, 1244)
    dt = 5e-5
    s = np.sqrt(2 * dt)
    ctx = bd.Context(Nc, h_star=0.25, dt=dt, flow=bd.FLOW_UNIAXIAL, Wi=50.0, precision=bd.MIXED_TF32)
    ctx.set_state(cuda(r0))
    ctx.assemble()
    ctx.factor()
    st, _ = ctx.chain_status()
    assert (st == 0).all(), st
    assert ctx.factor_residual(0) < 1e-3
    rm, _ = ctx.midpoint(cuda(xi[0]))
    rm = rm.cpu().numpy()
    L = ctx.read_matrix(0, 1)
    yB = (s * (L @ xi[0].ravel())).reshape(N, 3)   # the raw displacement that places r_m
    Q = np.diff(r0, axis=0)
    u = Q / np.linalg.norm(Q, axis=1)[:, None]
    c = (u * (yB[1:] - yB[:-1])).sum(1)
    off = -(u[:-1] * u[1:]).sum(1)
    ab = np.zeros((3, N - 1))
    ab[0, 1:] = off
    ab[1, :] = 2.0
    ab[2, :-1] = off
    x = sp.solve_banded((1, 1), ab, c)
    Py = yB.copy()
    Py[:-1] += x[:, None] * u
    Py[1:] -= x[:, None] * u
    np.testing.assert_allclose(rm, r0 + 0.5 * Py, rtol=0, atol=1e-5 * np.abs(yB).max())
    if N == 6000:
        D = orc.assemble(r0, 0.25, 0.25)
        Lx = np.linalg.cholesky(D)
        del D
        y = ctx.brownian(cuda(xi[0])).cpu().numpy().ravel()
        y64 = s * (Lx @ xi[0].ravel())
        assert np.abs(y - y64).max() / np.abs(y64).max() < 1e-2
    del L
    ctx.set_state(cuda(r0))
    ctx.step(cuda(xi))
    obs, st = ctx.observables()
    assert (st == 0).all(), st
    assert obs[:, bd.OBS_MAXDEV].max().item() < 1e-10
    ctx.close()
