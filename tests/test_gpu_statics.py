"""Equilibrium statistics of the GPU rigid-rod step with hydrodynamic
interaction (midpoint step), on both precision paths.

HI leaves the statics of rigid rods unchanged: <R^2> = (N - 1) b^2 and
<u_k . u_k+1> = 0, and a rigid trimer's bond angle carries the metric weight
sqrt(4 - cos^2 theta) of its constraints, <cos^2 theta> = 0.3210.  Each is
checked within 3 standard errors over 2000 independent chains (per-chain
time averages of eight samples after a burn-in from stretched starts), the
same estimators the oracle's pins use.
"""
import numpy as np
import pytest

from paper_2208_06559_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RIGID_TRIMER_COS2 = (np.pi / 3 - np.sqrt(3) / 4) / (np.sqrt(3) / 2 + np.pi / 3)
CHAINS, DT, BURN, GAP, SAMPLES = 2000, 1e-3, 3000, 500, 8


@pytest.fixture(scope="module")
def bd():
    from paper_2208_06559_gb300 import build as b
    b.build()
    import paper_2208_06559_gb300 as pkg
    pkg.lib()
    return pkg


def samples(bd, N, precision, seed):
    Nc = np.full(CHAINS, N, np.int32)
    ctx = bd.Context(Nc, h_star=0.25, a=0.25, dt=DT, tol=1e-12, precision=precision)
    ctx.set_state(torch.from_numpy(inputs.random_walk(Nc, seed, stretched=True)).cuda())
    k = seed + 1

    def advance(steps):
        nonlocal k
        for c0 in range(0, steps, GAP):
            nz = inputs.gaussian_noise(min(GAP, steps - c0), CHAINS * N, k)
            k += 1
            ctx.step(torch.from_numpy(nz).cuda())

    advance(BURN)
    R2, cs, c2 = [], [], []
    for _ in range(SAMPLES):
        advance(GAP)
        rr = ctx.get_state().cpu().numpy().reshape(CHAINS, N, 3)
        R = rr[:, -1] - rr[:, 0]
        R2.append((R * R).sum(1))
        Q = np.diff(rr, axis=1)
        c = (Q[:, :-1] * Q[:, 1:]).sum(2)
        cs.append(c.mean(1))
        c2.append((c * c).mean(1))
    st, _ = ctx.chain_status()
    ctx.close()
    assert (st == 0).all(), st
    return [np.mean(x, axis=0) for x in (R2, cs, c2)]


def se(x):
    return x.std(ddof=1) / np.sqrt(len(x))


@pytest.mark.parametrize("precision", [0, 1])
def test_hi_statics_of_rigid_rods(bd, precision):
    """N = 4, h* = 0.25: <R^2> = 3 and <u_k . u_k+1> = 0 within 3 s.e."""
    R2, cs, _ = samples(bd, 4, precision, 300 + precision)
    assert abs(R2.mean() - 3.0) < 3 * se(R2), (R2.mean(), se(R2))
    assert abs(cs.mean()) < 3 * se(cs), (cs.mean(), se(cs))


def test_rigid_trimer_bond_angle_mixed(bd):
    """N = 3, h* = 0.25, mixed path: <cos^2 theta> = 0.3210 within 3 s.e."""
    _, _, c2 = samples(bd, 3, 1, 310)
    assert abs(c2.mean() - RIGID_TRIMER_COS2) < 3 * se(c2), (c2.mean(), se(c2))
