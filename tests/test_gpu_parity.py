"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every input is seeded and synthetic (paper_2208_06559_gb300.inputs).  Sizes
span several tiles and a ragged tail; the FP64 path must match the oracle to
1e-10 relative in bead positions after 100 steps, per stage to round-off.
"""
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


def make(bd, Nc, seed=1, **kw):
    Nc = np.asarray(Nc, np.int32)
    r0 = inputs.random_walk(Nc, seed)
    ctx = bd.Context(Nc, **kw)
    ctx.set_state(cuda(r0))
    return ctx, r0


RAGGED = [2, 3, 16, 17, 37, 64, 65, 100]


# ------------------------------------------------------------- assembly
def test_assembly_matches_oracle(bd):
    ctx, r0 = make(bd, RAGGED, seed=3, h_star=0.25)
    ctx.assemble()
    off = np.concatenate([[0], np.cumsum(RAGGED)])
    for c, N in enumerate(RAGGED):
        D = ctx.read_matrix(c, 0)
        Dref = orc.assemble(r0[off[c]:off[c + 1]], 0.25, 0.25)
        np.testing.assert_allclose(D, Dref, rtol=0, atol=2e-16 * 8)
    ctx.close()


def test_assembly_overlap_branch_and_hstar_zero(bd):
    # beads closer than 2a: a chain folded back on itself
    r = np.array([[0, 0, 0], [1, 0, 0], [0.3, 0.2, 0.1], [0.2, 0.9, 0.1]], float)
    for hs, a in ((0.5, 0.5), (0.25, 0.6), (0.0, 0.0)):
        ctx = bd.Context([4], h_star=hs, a=a)
        ctx.set_state(cuda(r))
        ctx.assemble()
        np.testing.assert_allclose(ctx.read_matrix(0, 0), orc.assemble(r, hs, a), atol=1e-15)
        ctx.close()


# ------------------------------------------------------------- Cholesky
@pytest.mark.parametrize("Nc", [[2, 16, 17], [100, 11], [331]])
def test_factor_matches_oracle(bd, Nc):
    ctx, r0 = make(bd, Nc, seed=5)
    ctx.assemble()
    ctx.factor()
    off = np.concatenate([[0], np.cumsum(Nc)])
    for c, N in enumerate(Nc):
        L = ctx.read_matrix(c, 1)
        Lref, st = orc.cholesky(orc.assemble(r0[off[c]:off[c + 1]], 0.25, 0.25))
        assert st == 0
        np.testing.assert_allclose(L, Lref, rtol=0, atol=1e-13)
        assert ctx.factor_residual(c) < 1e-14
    ctx.close()


# ------------------------------------------------- Brownian and mobility
def test_brownian_and_mobility_match_oracle(bd):
    ctx, r0 = make(bd, RAGGED, seed=9, dt=1e-4)
    ctx.assemble()
    ctx.factor()
    tot = int(np.sum(RAGGED))
    xi = inputs.gaussian_noise(1, tot, 10)[0]
    f = inputs.gaussian_noise(1, tot, 11)[0]
    y = ctx.brownian(cuda(xi)).cpu().numpy()
    u = ctx.mobility_apply(cuda(f)).cpu().numpy()
    off = np.concatenate([[0], np.cumsum(RAGGED)])
    for c in range(len(RAGGED)):
        sl = slice(off[c], off[c + 1])
        D = orc.assemble(r0[sl], 0.25, 0.25)
        L, _ = orc.cholesky(D)
        yref = np.sqrt(2e-4) * orc.trmv_lower(L, xi[sl].ravel())
        uref = orc.gemv(D, f[sl].ravel())
        np.testing.assert_allclose(y[sl].ravel(), yref, rtol=0, atol=1e-14 * (1 + np.abs(yref).max()))
        np.testing.assert_allclose(u[sl].ravel(), uref, rtol=0, atol=1e-13 * (1 + np.abs(uref).max()))
    ctx.close()


# ------------------------------------------------------ midpoint stage
@pytest.mark.parametrize("prec", [0, 1])
def test_midpoint_stage_matches_oracle(bd, prec):
    """r_m = r + P y / 2 and the step's displacement s D(r_m) L^{-T} xi of the
    midpoint scheme, against the oracle's projection, back substitution,
    assembly at r_m and product.  FP64 path to round-off; mixed path: r_m
    within the factor's first-order error of the FP64 value (it projects the
    refined displacement), the displacement within that error too."""
    Nc = RAGGED if prec == 0 else [2, 43, 300, 1000]
    ctx, r0 = make(bd, Nc, seed=19, dt=1e-4, precision=prec)
    ctx.assemble()
    ctx.factor()
    tot = int(np.sum(Nc))
    xi = inputs.gaussian_noise(1, tot, 20)[0]
    rm, y = ctx.midpoint(cuda(xi))
    rm, y = rm.cpu().numpy(), y.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(Nc)])
    s = np.sqrt(2e-4)
    for c in range(len(Nc)):
        sl = slice(off[c], off[c + 1])
        D = orc.assemble(r0[sl], 0.25, 0.25)
        L, _ = orc.cholesky(D)
        yB = s * orc.trmv_lower(L, xi[sl].ravel())
        z = orc.trsv_lower_t(L, xi[sl].ravel())
        rm_ref = r0[sl] + 0.5 * orc.tangent_project(r0[sl], yB)
        y_ref = s * orc.gemv(orc.assemble(rm_ref, 0.25, 0.25), z)
        tol_r, tol_y = (1e-14, 1e-13) if prec == 0 else (1e-3, 1e-3)
        np.testing.assert_allclose(rm[sl], rm_ref, rtol=0, atol=tol_r * np.abs(yB).max() + 1e-15)
        np.testing.assert_allclose(y[sl].ravel(), y_ref, rtol=0, atol=tol_y * np.abs(y_ref).max())
    ctx.close()


# ------------------------------------------------------------- full step
def run_both(bd, Nc, steps, seed, **phys):
    Nc = np.asarray(Nc, np.int32)
    r0 = inputs.random_walk(Nc, seed)
    noise = inputs.gaussian_noise(steps, int(Nc.sum()), seed + 1)
    kw = dict(h_star=phys.get("hstar", 0.25), dt=phys.get("dt", 1e-4), flow=phys.get("flow", 0),
              Wi=phys.get("Wi", 0.0), tol=phys.get("tol", 1e-13), max_newton=phys.get("max_newton", 50),
              scheme=phys.get("scheme", 0))
    ctx = bd.Context(Nc, **kw)
    ctx.set_state(cuda(r0))
    ctx.step(cuda(noise))
    r_gpu = ctx.get_state().cpu().numpy()
    obs, st = ctx.observables()
    T_gpu = ctx.tensions().cpu().numpy()
    launches = ctx.kernel_launches()
    ctx.close()
    p = orc.make_params(hstar=kw["h_star"], dt=kw["dt"], flow=kw["flow"], Wi=kw["Wi"],
                        tol=kw["tol"], max_newton=kw["max_newton"], scheme=kw["scheme"])
    r_ref, T_ref, st_ref, it_ref, md_ref = orc.run(p, Nc, r0, noise)
    return r0, r_gpu, r_ref, st, st_ref, obs.cpu().numpy(), T_gpu, T_ref, launches


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1.0)


@pytest.mark.parametrize("scheme", [0, 1])
def test_step_parity_single_chain_n16_100_steps(bd, scheme):
    """One chain of 16 beads at equilibrium (no flow), dt = 1e-4, 100 steps
    (midpoint and Euler rigid-rod steps)."""
    r0, rg, rr, st, str_, obs, Tg, Tr, nl = run_both(bd, [16], 100, 1235, scheme=scheme)
    assert (st == 0).all() and (str_ == 0).all()
    assert rel(rg, rr) < 1e-10
    assert obs[0, 6] < 1e-10      # rod lengths held
    assert nl > 0


@pytest.mark.parametrize("scheme", [0, 1])
def test_step_parity_batch_n100_uniaxial(bd, scheme):
    """8 chains of 100 beads, uniaxial extension Wi = 10, 100 steps; the
    observables (Eqs. (25)-(29)) against the oracle's on the oracle's state."""
    r0, rg, rr, st, str_, obs, Tg, Tr, nl = run_both(bd, [100] * 8, 100, 1236, flow=2, Wi=10.0,
                                                     scheme=scheme)
    assert (st == 0).all() and (str_ == 0).all()
    assert rel(rg, rr) < 1e-10
    assert obs[:, 6].max() < 1e-10
    np.testing.assert_allclose(Tg, Tr, rtol=1e-6, atol=1e-6)
    for c in range(8):
        ref = orc.observables(rr[100 * c:100 * (c + 1)], Tr[99 * c:99 * (c + 1)])
        np.testing.assert_allclose(obs[c, [0, 1, 2, 3, 4, 5]], ref[[0, 1, 2, 3, 4, 5]], rtol=1e-9)
        np.testing.assert_allclose(obs[c, 8:12], ref[8:12], rtol=1e-5, atol=1e-5 * np.abs(ref[8:12]).max())


def test_step_parity_uneven_shear(bd):
    """Uneven batch (ragged tiles, N = 2 dumbbells), simple shear Wi = 100."""
    r0, rg, rr, st, str_, obs, Tg, Tr, nl = run_both(bd, RAGGED, 30, 77, flow=1, Wi=100.0)
    assert (st == 0).all() and (str_ == 0).all()
    assert rel(rg, rr) < 1e-10


def test_step_parity_free_draining(bd):
    r0, rg, rr, st, str_, obs, Tg, Tr, nl = run_both(bd, [20, 33], 50, 91, hstar=0.0, dt=1e-3)
    assert (st == 0).all()
    assert rel(rg, rr) < 1e-10


def test_host_noise_equals_device_noise(bd):
    Nc = np.array([16, 40], np.int32)
    r0 = inputs.random_walk(Nc, 12)
    noise = inputs.gaussian_noise(7, int(Nc.sum()), 13)
    out = []
    for dev in (True, False):
        ctx = bd.Context(Nc, flow=2, Wi=5.0)
        ctx.set_state(cuda(r0))
        nz = cuda(noise) if dev else torch.from_numpy(noise)
        ctx.step(nz)
        out.append(ctx.get_state().cpu().numpy())
        ctx.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_two_calls_equal_one_call(bd):
    Nc = np.array([30], np.int32)
    r0 = inputs.random_walk(Nc, 14)
    noise = inputs.gaussian_noise(6, 30, 15)
    a = bd.Context(Nc)
    a.set_state(cuda(r0))
    a.step(cuda(noise))
    b = bd.Context(Nc)
    b.set_state(cuda(r0))
    b.step(cuda(noise[:2]))
    b.step(cuda(noise[2:]))
    np.testing.assert_array_equal(a.get_state().cpu().numpy(), b.get_state().cpu().numpy())
    a.close()
    b.close()


@pytest.mark.parametrize("precision,unroll", [(0, None), (0, "0"), (1, None), (1, "0")])
def test_one_graph_launch_runs_every_step(bd, monkeypatch, precision, unroll):
    """bd_step advances every chain of an uneven batch by all n steps in one
    launch of the step graph (an outer WHILE node loops over the steps on the
    device): five steps in one call equal five one-step calls bit for bit,
    also with no tension iteration captured ahead of the inner WHILE node
    (its condition is set anew in every step), and both runs count the same
    kernels.  The five-step run also matches the oracle."""
    if unroll is not None:
        monkeypatch.setenv("BD_GRAPH_UNROLL", unroll)
    Nc = np.array([40, 9, 61], np.int32)
    r0 = inputs.random_walk(Nc, 31)
    noise = inputs.gaussian_noise(5, int(Nc.sum()), 32)
    kw = dict(h_star=0.25, dt=1e-3, flow=bd.FLOW_SHEAR, Wi=5.0, precision=precision)
    a = bd.Context(Nc, **kw)
    a.set_state(cuda(r0))
    a.step(cuda(noise))
    b = bd.Context(Nc, **kw)
    b.set_state(cuda(r0))
    for k in range(5):
        b.step(cuda(noise[k:k + 1]))
    ra, rb = a.get_state().cpu().numpy(), b.get_state().cpu().numpy()
    np.testing.assert_array_equal(ra, rb)
    assert a.kernel_launches() == b.kernel_launches() > 0
    for ctx in (a, b):
        st, _ = ctx.chain_status()
        assert (st == 0).all(), st
        ctx.close()
    p = orc.make_params(hstar=0.25, dt=1e-3, flow=orc.FLOW_SHEAR, Wi=5.0)
    rr, _, st_ref, _, _ = orc.run(p, Nc, r0, noise)
    assert (st_ref == 0).all()
    if precision == 0:
        assert np.abs(ra - rr).max() <= 1e-10 * np.abs(rr).max()
    else:  # displacements, to the factor's first-order error (as in the accuracy gates)
        d, dr = ra - r0, rr - r0
        assert np.abs(d - dr).max() <= 1e-3 * np.abs(dr).max(), np.abs(d - dr).max()


@pytest.mark.parametrize("scheme,hstar", [(0, 0.25), (1, 0.25), (0, 0.6)])
def test_fused_short_chain_step_equals_multi_kernel_step(bd, monkeypatch, scheme, hstar):
    """FP64 batches whose chains have at most 32 beads take the fused step
    (one CTA per chain, every matrix in shared memory, all the steps of a
    call in one launch).  On an uneven batch under shear, 20 steps of it
    match 20 steps of the multi-kernel step (BD_SMALL_STEP=0) to round-off,
    with the same status words and tension iteration counts within one, in
    one kernel launch per call; both match the oracle.  h* = a = 0.6 puts
    bonded beads inside 2a (the overlap branch of the RPY tensor)."""
    Nc = np.array([2, 3, 16, 31, 32], np.int32)
    r0 = inputs.random_walk(Nc, 41)
    noise = inputs.gaussian_noise(20, int(Nc.sum()), 42)
    kw = dict(h_star=hstar, a=hstar, dt=1e-3, flow=bd.FLOW_SHEAR, Wi=5.0, scheme=scheme)
    out = {}
    for fused in (True, False):
        if not fused:
            monkeypatch.setenv("BD_SMALL_STEP", "0")
        ctx = bd.Context(Nc, **kw)
        ctx.set_state(cuda(r0))
        ctx.step(cuda(noise))
        st, its = ctx.chain_status()
        out[fused] = (ctx.get_state().cpu().numpy(), st, its, ctx.kernel_launches())
        ctx.close()
    ra, sa, ia, la = out[True]
    rb, sb, ib, lb = out[False]
    assert (sa == 0).all() and (sb == 0).all(), (sa, sb)
    assert np.abs(ra - rb).max() <= 1e-12 * np.abs(rb).max()
    assert np.abs(ia.astype(int) - ib.astype(int)).max() <= 1, (ia, ib)
    assert la == 1 and lb > 100, (la, lb)
    p = orc.make_params(hstar=hstar, a=hstar, dt=1e-3, flow=orc.FLOW_SHEAR, Wi=5.0, scheme=scheme)
    rr, _, st_ref, _, _ = orc.run(p, Nc, r0, noise)
    assert (st_ref == 0).all()
    assert np.abs(ra - rr).max() <= 1e-10 * np.abs(rr).max()


# ------------------------------------------------------------- failures
def test_not_pd_chain_is_frozen_and_others_advance(bd):
    """Two coincident beads with a = h* make D singular: that chain reports
    BD_ERR_NOT_PD and keeps its positions; the other chain advances."""
    good = inputs.random_walk([10], 3)
    bad = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 0, 0]], float)  # bead 3 on bead 0
    r0 = np.concatenate([good, bad])
    ctx = bd.Context([10, 4])
    ctx.set_state(cuda(r0))
    ctx.step(cuda(inputs.gaussian_noise(2, 14, 4)))
    r1 = ctx.get_state().cpu().numpy()
    obs, st = ctx.observables()
    assert st[0] == 0 and st[1] == bd.binding.BD_ERR_NOT_PD
    np.testing.assert_array_equal(r1[10:], bad)
    assert np.abs(r1[:10] - good).max() > 0
    ctx.close()


def test_newton_cap_reports_constraint_error(bd):
    Nc = np.array([30], np.int32)
    ctx = bd.Context(Nc, dt=1e-3, max_newton=1)
    r0 = inputs.random_walk(Nc, 5)
    ctx.set_state(cuda(r0))
    ctx.step(cuda(inputs.gaussian_noise(1, 30, 6)))
    st, it = ctx.chain_status()
    assert st[0] == bd.binding.BD_ERR_CONSTRAINT
    np.testing.assert_array_equal(ctx.get_state().cpu().numpy(), r0)
    ctx.close()


def test_rod_lengths_over_many_steps_and_launch_count(bd):
    Nc = np.array([50, 51, 52], np.int32)
    ctx, r0 = make(bd, Nc, seed=17, dt=1e-4, flow=2, Wi=50.0)
    ctx.step(cuda(inputs.gaussian_noise(300, int(Nc.sum()), 18)))
    obs, st = ctx.observables()
    assert (st == 0).all()
    assert obs[:, 6].max().item() < 1e-10
    assert ctx.kernel_launches() > 300
    ctx.close()
