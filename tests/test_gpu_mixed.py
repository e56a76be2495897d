"""Mixed-precision path (FP32 storage, TF32 tensor-core Cholesky updates,
FP32 diagonal tiles, FP64-accurate tension solve) against the FP64 oracle.

Parity here is not bit-level: the factor carries TF32 rounding (10-bit
mantissa, unit round-off 2^-11 ~ 4.9e-4).  The bounds below follow from that:
a backward error ||B B^T - D||_F / ||D||_F of order 1e-4..1e-3 for the raw
factor, and after the refinement of the Brownian displacement, an error of
second order in the factor error.
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


MIXED_SIZES = [2, 40, 43, 86, 300, 1000]


def test_mixed_factor_backward_error(bd):
    Nc = np.array(MIXED_SIZES, np.int32)
    r0 = inputs.random_walk(Nc, 21)
    ctx = bd.Context(Nc, precision=bd.MIXED_TF32)
    ctx.set_state(cuda(r0))
    ctx.assemble()
    ctx.factor()
    st, _ = ctx.chain_status()
    assert (st == 0).all(), st
    off = np.concatenate([[0], np.cumsum(Nc)])
    for c, N in enumerate(Nc):
        res = ctx.factor_residual(c)
        assert res < 2e-3, (N, res)
        if N <= 300:
            D = orc.assemble(r0[off[c]:off[c + 1]], 0.25, 0.25)
            Lref, _ = orc.cholesky(D)
            L = ctx.read_matrix(c, 1)
            Dg = ctx.read_matrix(c, 0)
            np.testing.assert_allclose(Dg, D, rtol=0, atol=1e-6)      # FP32 storage of D
            assert np.abs(L - Lref).max() < 2e-2 * np.abs(Lref).max(), N
    ctx.close()


def test_mixed_step_constraints_and_displacement(bd):
    """One step from the same state and noise: rod lengths exact to the
    Newton tolerance (FP64 solve), displacement close to the FP64 oracle."""
    Nc = np.array([40, 300, 1000], np.int32)
    r0 = inputs.random_walk(Nc, 22)
    noise = inputs.gaussian_noise(1, int(Nc.sum()), 23)
    ctx = bd.Context(Nc, precision=bd.MIXED_TF32, flow=1, Wi=100.0)
    ctx.set_state(cuda(r0))
    ctx.step(cuda(noise))
    r1 = ctx.get_state().cpu().numpy()
    obs, st = ctx.observables()
    assert (st == 0).all(), st
    assert obs[:, 6].max().item() < 1e-10
    p = orc.make_params(hstar=0.25, dt=1e-4, flow=orc.FLOW_SHEAR, Wi=100.0)
    rr, *_ = orc.run(p, Nc, r0, noise)
    disp_err = np.abs((r1 - r0) - (rr - r0)).max() / np.abs(rr - r0).max()
    assert disp_err < 2e-2, disp_err
    ctx.close()


def test_refined_brownian_displacement(bd):
    """y = s/2 (Lt xi + D Lt^{-T} xi): matches that formula evaluated in FP64
    from the library's own Lt and D to FP32 level (the solve with Lt^T uses
    FP32 inverses of the 128 x 128 diagonal tiles), and the refined factor
    B_eff = (Lt + D Lt^{-T}) / 2 reproduces D to <= 1e-6 while the raw TF32
    factor only does to ~1e-4.  B_eff is a different square root of D than
    the FP64 Cholesky factor L (B_eff - L is first order in the factor
    error), so the displacement agrees with s L xi only to that order."""
    Nc = np.array([43, 300], np.int32)
    r0 = inputs.random_walk(Nc, 31)
    dt = 1e-4
    ctx = bd.Context(Nc, precision=bd.MIXED_TF32, refine=1, dt=dt)
    ctx.set_state(cuda(r0))
    ctx.assemble()
    ctx.factor()
    xi = inputs.gaussian_noise(1, int(Nc.sum()), 32)[0]
    y = ctx.brownian(cuda(xi)).cpu().numpy()
    off = np.concatenate([[0], np.cumsum(Nc)])
    s = np.sqrt(2 * dt)
    for c in range(len(Nc)):
        sl = slice(off[c], off[c + 1])
        Lt = ctx.read_matrix(c, 1)
        D = ctx.read_matrix(c, 0)
        Beff = 0.5 * (Lt + D @ np.linalg.inv(Lt).T)
        yref = s * Beff @ xi[sl].ravel()
        err = np.abs(y[sl].ravel() - yref).max() / np.abs(yref).max()
        assert err < 1e-6, (c, err)
        raw = np.linalg.norm(Lt @ Lt.T - D) / np.linalg.norm(D)
        refined = np.linalg.norm(Beff @ Beff.T - D) / np.linalg.norm(D)
        assert refined < 1e-6 and refined < raw, (raw, refined)
        Dx = orc.assemble(r0[sl], 0.25, 0.25)
        Lx, _ = orc.cholesky(Dx)
        y64 = s * Lx @ xi[sl].ravel()
        assert np.abs(y[sl].ravel() - y64).max() / np.abs(y64).max() < 1e-2
    ctx.close()


def test_mixed_without_refinement_is_plain_factor(bd):
    """refine = 0: y = s Lt xi.  The product sums groups of four FP32
    products (three roundings of at most u = 2^-24 of the group's absolute
    sum) and adds the group sums exactly (two-sum), so every element is
    within 4 u s sum_j |Lt_ij xi_j| of the FP64 product of the same Lt."""
    Nc = np.array([40, 300], np.int32)
    r0 = inputs.random_walk(Nc, 33)
    ctx = bd.Context(Nc, precision=bd.MIXED_TF32, refine=0)
    ctx.set_state(cuda(r0))
    ctx.assemble()
    ctx.factor()
    xi = inputs.gaussian_noise(1, int(Nc.sum()), 34)[0]
    y = ctx.brownian(cuda(xi)).cpu().numpy()
    s = np.sqrt(2e-4)
    off = np.concatenate([[0], np.cumsum(Nc)])
    for c in range(len(Nc)):
        sl = slice(off[c], off[c + 1])
        Lt = ctx.read_matrix(c, 1)
        x = xi[sl].ravel()
        yref = s * Lt @ x
        bound = 4 * 2.0 ** -24 * s * (np.abs(Lt) @ np.abs(x)) + 1e-300
        assert (np.abs(y[sl].ravel() - yref) <= bound).all(), np.max(np.abs(y[sl].ravel() - yref) / bound)
    ctx.close()


def test_factor_tuning_and_configs(bd, tmp_path):
    """Every (panel, groups) shape gives a valid factor; the tuner picks one of
    them, writes the cache, and a cached entry is reused."""
    Nc = np.array([300] * 6 + [200, 43], np.int32)
    r0 = inputs.random_walk(Nc, 41)
    ctx = bd.Context(Nc, precision=bd.MIXED_TF32)
    ctx.set_state(cuda(r0))
    L = bd.lib()
    for panel in (1, 2, 4, 6, 8, 12, 16, 24):
        for groups in (1, 2, 4, 8):
            assert L.bd_set_factor_config(ctx._h, panel, groups) == 0
            ctx.assemble()
            ctx.factor()
            st, _ = ctx.chain_status()
            assert (st == 0).all()
            assert max(ctx.factor_residual(c) for c in (0, 6, 7)) < 2e-3
    cache = str(tmp_path / "tune.json")
    p, g, ms = ctx.tune_factor(cache)
    assert p in (2, 4, 6, 8, 12, 16, 24) and g in (1, 2, 4, 8) and ms > 0
    p2, g2, ms2 = ctx.tune_factor(cache)
    assert (p2, g2, ms2) == (p, g, None)
    ctx.step(cuda(inputs.gaussian_noise(2, int(Nc.sum()), 42)))
    obs, st = ctx.observables()
    assert (st == 0).all() and obs[:, 6].max().item() < 1e-10
    ctx.close()


def test_profiled_step_equals_graph_step(bd):
    """bd_profile_step launches the step's kernels one by one (no graph) with
    stage events: the state after it equals the state after bd_step bit for
    bit, and the stage times are positive and add up to the step."""
    Nc = np.array([300, 1000, 86], np.int32)
    r0 = inputs.random_walk(Nc, 31)
    noise = cuda(inputs.gaussian_noise(1, int(Nc.sum()), 32))
    out = []
    for prof in (False, True):
        ctx = bd.Context(Nc, precision=bd.MIXED_TF32, flow=1, Wi=100.0)
        ctx.set_state(cuda(r0))
        if prof:
            tl = ctx.profile_step(noise[0])
            assert set(tl) == set(bd.Context.PROFILE_STAGES)
            assert all(v > 0 for v in tl.values())
            parts = sum(tl[k] for k in ("assemble", "factor", "brownian", "k_wait_predictor", "tension",
                                        "commit"))
            assert abs(parts - tl["step"]) <= 1e-3 * tl["step"] + 1e-3
        else:
            ctx.step(noise)
        st, _ = ctx.chain_status()
        assert (st == 0).all()
        out.append(ctx.get_state().cpu().numpy())
        ctx.close()
    np.testing.assert_array_equal(out[0], out[1])


# Rod counts m = N - 1 at the edges of the tension path's blocking: the
# 64-wide tiles of K's factor (m = 64, 65), the 256-wide super-blocks of the
# solve (m = 255, 256, 257, 512) and a ragged multi-super-block chain.
EDGE_SIZES = [2, 65, 66, 256, 257, 258, 513, 1300]


def test_rod_space_iteration_without_hi_matches_fp64(bd):
    """h* = 0 makes D = I exactly, so the mixed and FP64 paths share the
    Brownian displacement and differ only in the tension iteration (rod
    space, FP32 G with FP32-rounded directions, super-block solve) against
    the FP64 bead-space iteration: after 3 steps of shear the positions agree
    to ~1e-8 of the displacement."""
    Nc = np.array(EDGE_SIZES, np.int32)
    r0 = inputs.random_walk(Nc, 51)
    noise = cuda(inputs.gaussian_noise(3, int(Nc.sum()), 52))
    out = {}
    for prec in (bd.FP64, bd.MIXED_TF32):
        ctx = bd.Context(Nc, precision=prec, flow=1, Wi=100.0, h_star=0.0)
        ctx.set_state(cuda(r0))
        ctx.step(noise)
        obs, st = ctx.observables()
        assert (st == 0).all(), (prec, st)
        assert obs[:, bd.OBS_MAXDEV].max().item() < 1e-10
        out[prec] = ctx.get_state().cpu().numpy()
        ctx.close()
    d64 = out[bd.FP64] - r0
    err = np.abs(out[bd.MIXED_TF32] - out[bd.FP64]).max() / np.abs(d64).max()
    assert err < 1e-6, err


def test_sixteen_chain_batch_against_fp64(bd):
    """16 chains select 4-CTA clusters for the refinement's triangular solve
    and the tension solve (2 CTAs for larger batches, 8 for smaller): two
    steps of shear Wi = 100 with HI, mixed against FP64 on the same noise --
    every chain converges within the FP64 iteration count + 2, rods hold to
    1e-10, displacements agree to the factor's first-order error (1e-3)."""
    Nc = np.array([300, 257, 129, 400] * 4, np.int32)
    r0 = inputs.random_walk(Nc, 57)
    noise = cuda(inputs.gaussian_noise(2, int(Nc.sum()), 58))
    out, its = {}, {}
    for prec in (bd.FP64, bd.MIXED_TF32):
        ctx = bd.Context(Nc, precision=prec, flow=1, Wi=100.0)
        ctx.set_state(cuda(r0))
        ctx.step(noise)
        obs, st = ctx.observables()
        assert (st == 0).all(), (prec, st)
        assert obs[:, bd.OBS_MAXDEV].max().item() < 1e-10
        out[prec] = ctx.get_state().cpu().numpy()
        its[prec] = ctx.chain_status()[1]
        ctx.close()
    assert (its[bd.MIXED_TF32] <= its[bd.FP64] + 2).all(), (its[bd.MIXED_TF32], its[bd.FP64])
    d64 = out[bd.FP64] - r0
    err = np.abs(out[bd.MIXED_TF32] - out[bd.FP64]).max() / np.abs(d64).max()
    assert err < 1e-3, err


def test_rod_space_iteration_edge_sizes_with_hi(bd):
    """With hydrodynamic interactions at the same edge sizes: every chain
    converges within the FP64 path's iteration count + 2, rods hold to
    1e-10, and the displacement stays within the TF32 factor's reach of the
    FP64 path."""
    Nc = np.array(EDGE_SIZES, np.int32)
    r0 = inputs.random_walk(Nc, 53)
    noise = cuda(inputs.gaussian_noise(2, int(Nc.sum()), 54))
    out, its = {}, {}
    for prec in (bd.FP64, bd.MIXED_TF32):
        ctx = bd.Context(Nc, precision=prec, flow=1, Wi=100.0)
        ctx.set_state(cuda(r0))
        ctx.step(noise)
        obs, st = ctx.observables()
        assert (st == 0).all(), (prec, st)
        assert obs[:, bd.OBS_MAXDEV].max().item() < 1e-10
        its[prec] = obs[:, bd.OBS_NEWTON].cpu().numpy()
        out[prec] = ctx.get_state().cpu().numpy()
        ctx.close()
    assert (its[bd.MIXED_TF32] <= its[bd.FP64] + 2).all(), its
    d64 = out[bd.FP64] - r0
    err = np.abs(out[bd.MIXED_TF32] - out[bd.FP64]).max() / np.abs(d64).max()
    assert err < 5e-2, err


def test_step_brownian_displacement_matches_stage_api(bd):
    """The Brownian displacement inside a graph-replayed step (several chain
    groups, ragged lengths) is the one the stage API computes.  In
    the Fraenkel mode with dt = 1e-12 the link update leaves the explicit step
    unchanged up to 2 dt K* ~ 2e-8 of the link stretch, and the unit bonds of
    the start carry no spring force, so r1 - r0 must equal the standalone
    displacement of the same factor (bd_assemble, bd_factor, bd_brownian)."""
    Nc = np.array([300, 40, 129, 300, 86, 300, 2, 213] * 5, np.int32)
    r0 = inputs.random_walk(Nc, 61)
    xi = inputs.gaussian_noise(1, int(Nc.sum()), 62)
    ctx = bd.Context(Nc, precision=bd.MIXED_TF32, dt=1e-12, constraint=bd.FRAENKEL, k_spring=1e4)
    ctx.set_state(cuda(r0))
    ctx.assemble()
    ctx.factor()
    y = ctx.brownian(cuda(xi[0])).cpu().numpy()
    ctx.step(cuda(xi))
    _, st = ctx.observables()
    assert (st == 0).all(), st
    dr = ctx.get_state().cpu().numpy() - r0
    err = np.abs(dr - y).max() / np.abs(y).max()
    assert err < 1e-6, err
    ctx.close()


def test_lanes_equal_one_batch(bd):
    """A context of 64 uneven chains stepped as 1, 2 or 3 lanes (concurrent
    sub-batches over contiguous chain ranges, each on its own streams) gives
    every chain the result of the single batch: positions, tensions,
    observables and statuses after five steps in one call (host noise), the
    stage calls (assembly, factorisation, Brownian displacement, mobility
    product) and one profiled step.  Lanes of other sizes may pick other
    cluster sizes for the per-chain solves (a different summation order), so
    the bound is far below any misplaced chain or bead and far above
    round-off: 1e-8 of the step's displacement."""
    g = np.random.default_rng(71)
    Nc = g.integers(20, 61, 64).astype(np.int32)
    total = int(Nc.sum())
    r0 = inputs.random_walk(Nc, 72)
    noise_h = torch.from_numpy(inputs.gaussian_noise(5, total, 73))
    xi = cuda(inputs.gaussian_noise(2, total, 74))
    res = {}
    for lanes in (1, 2, 3):
        ctx = bd.Context(Nc, precision=bd.MIXED_TF32, flow=1, Wi=10.0, lanes=lanes)
        assert ctx.lanes() == lanes
        ctx.set_state(cuda(r0))
        ctx.step(noise_h)
        obs, st = ctx.observables()
        obs_host = torch.empty((len(Nc), bd.OBS_STRIDE), dtype=torch.float64).pin_memory()
        ctx.observables(out=obs_host, with_status=False)   # asynchronous, into host memory
        torch.cuda.synchronize()
        np.testing.assert_array_equal(obs_host.numpy(), obs.cpu().numpy())
        out = dict(r=ctx.get_state().cpu().numpy(), T=ctx.tensions().cpu().numpy(), obs=obs.cpu().numpy(),
                   st=st, it=ctx.chain_status()[1], launches=ctx.kernel_launches())
        ctx.assemble()
        ctx.factor()
        out["y"] = ctx.brownian(xi[0]).cpu().numpy()
        out["u"] = ctx.mobility_apply(xi[1]).cpu().numpy()
        ms = ctx.profile_step(xi[0])
        assert ms["step"] > 0.0
        out["r1"] = ctx.get_state().cpu().numpy()
        assert (ctx.chain_status()[0] == 0).all()
        res[lanes] = out
        ctx.close()
    ref = res[1]
    assert (ref["st"] == 0).all() and ref["launches"] > 0
    disp = np.abs(ref["r"] - r0).max()
    for lanes in (2, 3):
        o = res[lanes]
        assert (o["st"] == ref["st"]).all()
        assert (np.abs(o["it"] - ref["it"]) <= 1).all()
        assert o["launches"] > 0
        assert np.abs(o["r"] - ref["r"]).max() < 1e-8 * disp, lanes
        assert np.abs(o["r1"] - ref["r1"]).max() < 1e-8 * disp, lanes
        assert np.abs(o["T"] - ref["T"]).max() < 1e-8 * np.abs(ref["T"]).max(), lanes
        for k in (bd.OBS_R2, bd.OBS_RG2):
            np.testing.assert_allclose(o["obs"][:, k], ref["obs"][:, k], rtol=1e-9)
        assert np.abs(o["y"] - ref["y"]).max() < 1e-8 * np.abs(ref["y"]).max(), lanes
        assert np.abs(o["u"] - ref["u"]).max() < 1e-10 * np.abs(ref["u"]).max(), lanes


def test_automatic_lane_count(bd):
    """Without an explicit count, mixed contexts of >= 32 chains, or of >= 4
    chains one of which has >= 2000 beads, use two lanes, smaller mixed
    batches one; FP64 contexts use one lane per 16 chains up to 8, and one
    when every chain has <= 32 beads (the fused short-chain step)."""
    cases = [(np.full(64, 30), bd.MIXED_TF32, 2), (np.full(32, 30), bd.MIXED_TF32, 2),
             (np.full(31, 30), bd.MIXED_TF32, 1), (np.array([30, 30, 30, 2000]), bd.MIXED_TF32, 2),
             (np.array([30, 30, 1999]), bd.MIXED_TF32, 1), (np.full(64, 30), bd.FP64, 1),
             (np.full(64, 40), bd.FP64, 4), (np.full(31, 40), bd.FP64, 1), (np.full(256, 33), bd.FP64, 8)]
    for Nc, prec, want in cases:
        with bd.Context(Nc.astype(np.int32), precision=prec) as ctx:
            assert ctx.lanes() == want, (len(Nc), int(Nc.max()), prec)
    with bd.Context(np.full(8, 30, np.int32), precision=bd.MIXED_TF32, lanes=8) as ctx:
        assert ctx.lanes() == 8
    with bd.Context(np.full(3, 30, np.int32), precision=bd.MIXED_TF32, lanes=8) as ctx:
        assert ctx.lanes() == 3   # never more lanes than chains
