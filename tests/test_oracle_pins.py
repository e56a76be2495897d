"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form
derived from the paper's equations (arXiv 2208.06559, Sec. 3), an invariant, an
independent library routine (LAPACK through numpy) or brute force on tiny
inputs.  A plausible slip anywhere in the oracle (a dropped term, a wrong sign
or index, a transposed operand) fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle as orc
from paper_2208_06559_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def mu_far(R, hs, a):
    """Eigenvalues of the two-bead coupling block for R >= 2a (parallel, perp),
    derived from Sec. 3 Eq. (8): along R the bracket is 2 - 4a^2/(3R^2)."""
    return (hs / a) * (1.5 * a / R - a ** 3 / R ** 3), (hs / a) * (0.75 * a / R + 0.5 * a ** 3 / R ** 3)


def mu_near(R, hs, a):
    """Same for R < 2a, derived from Sec. 3 Eq. (9)."""
    return (hs / a) * (1.0 - 3.0 * R / (16.0 * a)), (hs / a) * (1.0 - 9.0 * R / (32.0 * a))


def unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


# --------------------------------------------------------------------- RPY
@pytest.mark.parametrize("R,hs,a", [(1.0, 0.25, 0.25), (3.7, 0.25, 0.25), (0.7, 0.5, 0.5),
                                    (0.3, 0.25, 0.25), (0.49, 0.25, 0.25), (2.2, 0.1, 0.4)])
def test_two_bead_spectrum(R, hs, a):
    """The 6x6 two-bead D has eigenvalues 1 +- mu_par and 1 +- mu_perp (twice)."""
    d = unit([0.3, -0.8, 0.52])
    r = np.stack([np.zeros(3), R * d])
    D = orc.assemble(r, hs, a)
    mp, mq = (mu_far if R >= 2 * a else mu_near)(R, hs, a)
    want = np.sort([1 + mp, 1 - mp, 1 + mq, 1 + mq, 1 - mq, 1 - mq])
    got = np.sort(np.linalg.eigvalsh(D))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)
    # the coupling block is mu_perp I + (mu_par - mu_perp) d d^T in the
    # bead-major layout: rows 0..2 are bead 0, columns 3..5 are bead 1
    blk = mq * np.eye(3) + (mp - mq) * np.outer(d, d)
    np.testing.assert_allclose(D[0:3, 3:6], blk, atol=1e-15)
    np.testing.assert_allclose(D[3:6, 0:3], blk, atol=1e-15)
    np.testing.assert_array_equal(D[0:3, 0:3], np.eye(3))


def test_unit_bond_values():
    """h* = a = 0.25, R = 1: mu_perp = 0.1953125, mu_par = 0.359375 exactly."""
    blk = orc.rpy_block(np.array([0.0, 0.0, 1.0]), 0.25, 0.25)
    np.testing.assert_allclose(np.diag(blk), [0.1953125, 0.1953125, 0.359375], atol=1e-16)


def test_branch_continuity():
    """Both RPY branches equal (h*/a)[(7/16) I + (3/16) RR/R^2] at R = 2a."""
    hs, a = 0.3, 0.45
    d = unit([1.0, 2.0, -0.5])
    want = (hs / a) * (7 / 16 * np.eye(3) + 3 / 16 * np.outer(d, d))
    for eps in (-1e-13, 0.0, 1e-13):
        blk = orc.rpy_block(2 * a * (1 + eps) * d, hs, a)
        np.testing.assert_allclose(blk, want, atol=1e-12)


def test_coincident_limit():
    """R = 0 takes the limit of the overlap branch, (h*/a) I."""
    np.testing.assert_allclose(orc.rpy_block(np.zeros(3), 0.2, 0.4), 0.5 * np.eye(3), atol=1e-16)


def test_golden_two_bead_layout():
    """Element (row, col) of the two-bead matrix is D_ijkl as printed in Eq. (20)."""
    names = [ln.split() for ln in open(os.path.join(GOLDEN, "two_bead_layout.txt"))
             if ln.strip() and not ln.startswith("#")]
    r = np.array([[0.1, 0.2, -0.3], [0.9, -0.4, 0.35]])
    D = orc.assemble(r, 0.25, 0.25)
    blocks = {(0, 0): np.eye(3), (1, 1): np.eye(3),
              (0, 1): orc.rpy_block(r[0] - r[1], 0.25, 0.25),
              (1, 0): orc.rpy_block(r[1] - r[0], 0.25, 0.25)}
    assert len(names) == 6
    for row in range(6):
        for col in range(6):
            i, j, k, l = (int(c) for c in names[row][col][1:])
            assert D[row, col] == blocks[(i, j)][k, l]


def test_symmetry_and_hstar_zero():
    r = inputs.random_walk([40], 3)
    D = orc.assemble(r, 0.25, 0.25)
    np.testing.assert_array_equal(D, D.T)
    np.testing.assert_array_equal(orc.assemble(r, 0.0, 0.0), np.eye(120))


def test_a_larger_than_hstar_is_shifted_rpy():
    """With a > h*, D = (1 - h*/a) I + (h*/a) RPY_a (RPY_a: h* = a)."""
    r = inputs.random_walk([12], 4)
    hs, a = 0.2, 0.5
    D = orc.assemble(r, hs, a)
    Da = orc.assemble(r, a, a)
    np.testing.assert_allclose(D, (1 - hs / a) * np.eye(36) + (hs / a) * Da, atol=1e-15)


# ---------------------------------------------------------------- Cholesky
def test_cholesky_two_bead_closed_form():
    """Along z, L = [[I, 0], [A, diag(sqrt(1-mu_perp^2) x2, sqrt(1-mu_par^2))]]."""
    hs = a = 0.25
    R = 1.3
    r = np.array([[0, 0, 0], [0, 0, R]], float)
    L, st = orc.cholesky(orc.assemble(r, hs, a))
    assert st == orc.OK
    mp, mq = mu_far(R, hs, a)
    want = np.zeros((6, 6))
    want[:3, :3] = np.eye(3)
    want[3:, :3] = np.diag([mq, mq, mp])
    want[3:, 3:] = np.diag(np.sqrt([1 - mq * mq, 1 - mq * mq, 1 - mp * mp]))
    np.testing.assert_allclose(L, want, atol=1e-15)


@pytest.mark.parametrize("N,seed", [(16, 1), (100, 2), (301, 3)])
def test_cholesky_vs_lapack_and_backward_error(N, seed):
    r = inputs.random_walk([N], seed)
    D = orc.assemble(r, 0.25, 0.25)
    L, st = orc.cholesky(D)
    assert st == orc.OK
    assert np.all(np.triu(L, 1) == 0) and np.all(np.diag(L) > 0)
    assert orc.factor_residual(D, L) <= 1e-13
    np.testing.assert_allclose(L, np.linalg.cholesky(D), rtol=0, atol=1e-12)


def test_rpy_positive_definite_many_conformations():
    """All pivots > 0 on many random freely-jointed conformations (a = h*)."""
    g = inputs.rng(11)
    for s in range(400):
        N = 16 if s % 4 else 100
        r = inputs.random_walk([N], int(g.integers(1 << 30)))
        _, st = orc.cholesky(orc.assemble(r, 0.25, 0.25))
        assert st == orc.OK


def test_not_pd_for_coincident_beads():
    """Two coincident beads with a = h* make D singular: zero pivot."""
    r = np.array([[0.2, 0.1, 0.0], [0.2, 0.1, 0.0]])
    _, st = orc.cholesky(orc.assemble(r, 0.25, 0.25))
    assert st == orc.ERR_NOT_PD


# -------------------------------------------------------------- noise term
def test_trmv_brute_force():
    g = inputs.rng(5)
    for n in (1, 2, 3, 7, 48):
        M = g.standard_normal((n, n))
        L = np.tril(M)
        x = g.standard_normal(n)
        np.testing.assert_allclose(orc.trmv_lower(np.ascontiguousarray(M), x), L @ x,
                                   rtol=1e-13, atol=1e-13)


def test_brownian_covariance_matches_D():
    """Sample covariance of L xi over many xi is D (statistical)."""
    r = inputs.random_walk([4], 8)
    D = orc.assemble(r, 0.25, 0.25)
    L, _ = orc.cholesky(D)
    xi = inputs.gaussian_noise(1, 40000 * 4, 9)[0].reshape(40000, 12)
    y = np.stack([orc.trmv_lower(L, x) for x in xi[:20000]])
    C = y.T @ y / y.shape[0]
    # each entry's standard error is <= sqrt((D_ii D_jj + D_ij^2)/n) <= 0.01
    assert np.abs(C - D).max() < 0.045


# -------------------------------------------------------------------- flow
def test_flow_velocity_fields():
    """Simple shear: v_x = rate * y only.  Uniaxial: traceless, axisymmetric,
    stretching along x (Sec. 3 flow-force paragraph)."""
    g = inputs.rng(2)
    for _ in range(5):
        rpos = g.standard_normal(3)
        v = orc.kappa(orc.FLOW_SHEAR, 2.5) @ rpos
        np.testing.assert_allclose(v, [2.5 * rpos[1], 0, 0], atol=1e-15)
    K = orc.kappa(orc.FLOW_UNIAXIAL, 3.0)
    assert abs(np.trace(K)) < 1e-15
    assert K[0, 0] == 3.0 and K[1, 1] == K[2, 2]
    assert np.count_nonzero(K - np.diag(np.diag(K))) == 0
    assert np.all(orc.kappa(orc.FLOW_NONE, 7.0) == 0)


@pytest.mark.parametrize("hs", [0.0, 0.25])
def test_dumbbell_in_extension_tension(hs):
    """Rigid dumbbell along x in uniaxial extension, no noise: the predictor
    stretches the rod to 1 + rate dt and the tension that restores unit length
    is T = rate / (2 (1 - mu_par(1)))."""
    rate, dt = 10.0, 1e-3
    p = orc.make_params(hstar=hs, a=0.25, dt=dt, flow=orc.FLOW_UNIAXIAL, Wi=rate, lam=1.0)
    r0 = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    r1, T, st, it, md = orc.step(p, r0, np.zeros((2, 3)))
    assert st == orc.OK
    mp = mu_far(1.0, hs, 0.25)[0] if hs > 0 else 0.0
    np.testing.assert_allclose(T[0], rate / (2 * (1 - mp)), rtol=1e-12)
    assert md < 1e-13
    np.testing.assert_allclose(r1[:, 1:], 0.0, atol=1e-15)
    # the centre of mass follows kappa . r_cm (here r_cm = (0.5, 0, 0))
    np.testing.assert_allclose(r1[:, 0].mean(), 0.5 + dt * rate * 0.5, rtol=1e-13)


# ---------------------------------------------------------- tension solve
def _thomas_newton(rstar, u, dt, tol):
    """Independent Newton for h* = 0 (D = I): tridiagonal Jacobian solved by
    the Thomas algorithm."""
    N = rstar.shape[0]
    m = N - 1
    T = (np.linalg.norm(np.diff(rstar, axis=0), axis=1) - 1) / (2 * dt)
    extra = False
    for _ in range(60):
        F = np.zeros((N, 3))
        F[:-1] += T[:, None] * u
        F[1:] -= T[:, None] * u
        r = rstar + dt * F
        Q = np.diff(r, axis=0)
        g = (Q * Q).sum(1) - 1
        if extra:
            return T, r
        if np.abs(g).max() <= tol:
            extra = True
        # dQ_k/dT_k = -2 dt u_k, dQ_k/dT_{k+-1} = dt u_{k+-1}
        diag = -4 * dt * (Q * u).sum(1)
        lo = 2 * dt * (Q[1:] * u[:-1]).sum(1)    # J[k, k-1]
        up = 2 * dt * (Q[:-1] * u[1:]).sum(1)    # J[k, k+1]
        b = -g.copy()
        c = np.zeros(m)
        d = np.zeros(m)
        for k in range(m):
            den = diag[k] - (lo[k - 1] * c[k - 1] if k else 0.0)
            c[k] = up[k] / den if k < m - 1 else 0.0
            d[k] = (b[k] - (lo[k - 1] * d[k - 1] if k else 0.0)) / den
        x = np.zeros(m)
        for k in range(m - 1, -1, -1):
            x[k] = d[k] - (c[k] * x[k + 1] if k < m - 1 else 0.0)
        T = T + x
    raise AssertionError("no convergence")


def _predict(N, seed, dt, hs):
    r = inputs.random_walk([N], seed)
    D = orc.assemble(r, hs, 0.25)
    L, _ = orc.cholesky(D)
    xi = inputs.gaussian_noise(1, N, seed + 1)[0].ravel()
    rstar = r + np.sqrt(2 * dt) * (L @ xi).reshape(N, 3)
    Q0 = np.diff(r, axis=0)
    return D, rstar, Q0 / np.linalg.norm(Q0, axis=1)[:, None]


@pytest.mark.parametrize("N", [2, 3, 17, 60])
def test_tension_free_draining_vs_thomas(N):
    dt = 1e-3
    D, rstar, u = _predict(N, 21 + N, dt, 0.0)
    T, rT, st, it = orc.tension_solve(D, rstar, u, dt)
    assert st == orc.OK
    T2, r2 = _thomas_newton(rstar, u, dt, 1e-13)
    np.testing.assert_allclose(T, T2, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(rT, r2, atol=1e-13)
    assert np.abs(np.linalg.norm(np.diff(rT, axis=0), axis=1) - 1).max() < 1e-13


def test_tension_dumbbell_closed_form():
    """N = 2 with HI: Q(T) = Q* - 2 dt (1 - mu_par) T u, a scalar quadratic."""
    dt, hs, a = 1e-3, 0.25, 0.25
    D, rstar, u = _predict(2, 7, dt, hs)
    T, rT, st, it = orc.tension_solve(D, rstar, u, dt)
    assert st == orc.OK
    c = 2 * dt * (1 - mu_far(1.0, hs, a)[0])
    Qs = rstar[1] - rstar[0]
    qu = Qs @ u[0]
    Tc = (qu - np.sqrt(qu * qu - Qs @ Qs + 1)) / c
    np.testing.assert_allclose(T[0], Tc, rtol=1e-10)


@pytest.mark.parametrize("N,hs", [(10, 0.25), (50, 0.25), (120, 0.5)])
def test_tension_constraint_and_jacobian_by_differences(N, hs):
    """|Q_k| = 1 after the solve, and the solved T is a root of the residual
    evaluated independently here with numpy."""
    dt = 1e-4
    D, rstar, u = _predict(N, 31 + N, dt, hs)
    T, rT, st, it = orc.tension_solve(D, rstar, u, dt)
    assert st == orc.OK and it <= 8
    F = np.zeros((N, 3))
    F[:-1] += T[:, None] * u
    F[1:] -= T[:, None] * u
    r = rstar + dt * (D @ F.ravel()).reshape(N, 3)
    np.testing.assert_allclose(r, rT, atol=1e-14)
    assert np.abs(np.linalg.norm(np.diff(r, axis=0), axis=1) - 1).max() < 1e-13


def test_newton_cap_reports_failure():
    dt = 1e-3
    D, rstar, u = _predict(30, 5, dt, 0.25)
    _, _, st, it = orc.tension_solve(D, rstar, u, dt, tol=1e-13, max_newton=1)
    assert st == orc.ERR_CONSTRAINT


# --------------------------------------------- midpoint scheme (rigid rods)
def test_trsv_lower_t_brute_force():
    """z = L^{-T} x against numpy's general solve of L^T z = x."""
    g = inputs.rng(6)
    for n in (1, 2, 5, 48):
        L = np.tril(g.standard_normal((n, n))) + 4 * np.eye(n)
        x = g.standard_normal(n)
        np.testing.assert_allclose(orc.trsv_lower_t(L, x), np.linalg.solve(L.T, x),
                                   rtol=1e-13, atol=1e-13)


def _constraint_rows(r):
    """Rows of A: -u_k at bead k, +u_k at bead k+1."""
    N = r.shape[0]
    Q = np.diff(r, axis=0)
    u = Q / np.linalg.norm(Q, axis=1)[:, None]
    A = np.zeros((N - 1, 3 * N))
    for k in range(N - 1):
        A[k, 3 * k:3 * k + 3] = -u[k]
        A[k, 3 * k + 3:3 * k + 6] = u[k]
    return A


def test_tangent_projection_properties():
    """P y keeps every rod's length to first order (A P y = 0), is idempotent,
    and y - P y is normal to the tangent space (spanned by the rows of A);
    for a dumbbell P y removes the relative motion along the rod."""
    g = inputs.rng(7)
    for N in (2, 3, 9):
        r = inputs.random_walk([N], 70 + N)
        y = g.standard_normal((N, 3))
        Py = orc.tangent_project(r, y)
        A = _constraint_rows(r)
        assert np.abs(A @ Py.ravel()).max() < 1e-13
        np.testing.assert_allclose(orc.tangent_project(r, Py), Py, atol=1e-13)
        d = (y - Py).ravel()
        coef = np.linalg.lstsq(A.T, d, rcond=None)[0]
        np.testing.assert_allclose(A.T @ coef, d, atol=1e-13)
    r = np.array([[0.0, 0, 0], [0.0, 0.6, 0.8]])
    u = r[1] - r[0]
    y = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.7]])
    s = u @ (y[1] - y[0]) / 2
    np.testing.assert_allclose(orc.tangent_project(r, y), y + s * np.array([u, -u]), atol=1e-15)


def _step_drift(p, r):
    """Mean of (r_new - r)/dt over xi ~ N(0, I), to O(dt): with noise +xi and
    -xi the odd orders cancel, and the expectation of the remaining quadratic
    form in xi is its value at 0 plus the sum of its unit-vector terms."""
    n = r.size

    def g2(xi):
        a = orc.step(p, r, xi.reshape(-1, 3))
        b = orc.step(p, r, -xi.reshape(-1, 3))
        assert a[2] == 0 and b[2] == 0
        return (a[0] + b[0] - 2 * r).ravel() / (2 * p.dt)

    c = g2(np.zeros(n))
    tot = c.copy()
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        tot += g2(e) - c
    return tot


def _rigid_drift_tangent(r, hs, a, kap):
    """Tangent part of the drift of rigid-rod diffusion with HI on the
    constraint surface (equilibrium weight uniform in the surface measure):
    P (kappa r) + P_S sum_ij (P_S)_ij d_j (D_c)_{. i}, with the constrained
    mobility D_c = P D, P = I - D A^T (A D A^T)^{-1} A (flow velocity with the
    constraint forces that hold the rods) and P_S the orthogonal projector
    onto the tangent space; derivatives by central differences of D_c."""
    N = r.shape[0]
    n = 3 * N

    def Dc(x):
        x = x.reshape(N, 3)
        D = orc.assemble(x, hs, a)
        A = _constraint_rows(x)
        return D - D @ A.T @ np.linalg.solve(A @ D @ A.T, A @ D)

    A = _constraint_rows(r)
    D = orc.assemble(r, hs, a)
    P = np.eye(n) - D @ A.T @ np.linalg.solve(A @ D @ A.T, A)
    PS = np.eye(n) - A.T @ np.linalg.solve(A @ A.T, A)
    h = 1e-5
    div = np.zeros(n)
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        dD = (Dc(r.ravel() + e) - Dc(r.ravel() - e)) / (2 * h)
        div += dD @ PS[:, j]          # sum_i dD[:, i] PS[i, j]
    v = (r @ kap.T).ravel()
    return P @ v + PS @ div


@pytest.mark.parametrize("N,hs,a,flow", [(3, 0.25, 0.25, orc.FLOW_NONE), (5, 0.25, 0.25, orc.FLOW_UNIAXIAL),
                                         (4, 0.25, 0.4, orc.FLOW_SHEAR), (4, 0.5, 0.5, orc.FLOW_NONE),
                                         (4, 0.0, 0.25, orc.FLOW_NONE)])
def test_midpoint_step_has_the_rigid_rod_drift(N, hs, a, flow):
    """The step's mean displacement per unit time, projected on the tangent
    space, equals the drift of rigid-rod diffusion with HI; the Euler
    projection misses its HI part (equal only at h* = 0)."""
    r = inputs.random_walk([N], 200 + N)
    Wi = 2.0 if flow != orc.FLOW_NONE else 0.0
    want = _rigid_drift_tangent(r, hs, a, orc.kappa(flow, Wi))
    A = _constraint_rows(r)
    PS = np.eye(3 * N) - A.T @ np.linalg.solve(A @ A.T, A)
    p = orc.make_params(hstar=hs, a=a, dt=1e-6, flow=flow, Wi=Wi, tol=1e-14)
    got = PS @ _step_drift(p, r)
    np.testing.assert_allclose(got, want, atol=2e-4 * max(1.0, np.abs(want).max()))
    pe = orc.make_params(hstar=hs, a=a, dt=1e-6, flow=flow, Wi=Wi, tol=1e-14, scheme=orc.SCHEME_EULER)
    gap = np.abs(PS @ _step_drift(pe, r) - want).max()
    if hs > 0:
        assert gap > 1e-2
    else:
        assert gap < 2e-4


# -------------------------------------------------------------- dynamics
def test_rod_lengths_held_over_many_steps():
    Nc = np.array([16, 33, 5], np.int32)
    r = inputs.random_walk(Nc, 40)
    noise = inputs.gaussian_noise(200, int(Nc.sum()), 41)
    p = orc.make_params(hstar=0.25, dt=1e-4, flow=orc.FLOW_SHEAR, Wi=100.0)
    r1, T, st, it, md = orc.run(p, Nc, r, noise)
    assert np.all(st == 0)
    assert md.max() < 1e-10


def test_low_hstar_matches_free_draining_pathwise():
    """h* -> 0 reproduces the free-draining path to O(h*) (the paper's own
    check in Sec. 5), with the same noise."""
    Nc = np.array([20], np.int32)
    r = inputs.random_walk(Nc, 50)
    noise = inputs.gaussian_noise(100, 20, 51)
    res = []
    for hs in (0.0, 1e-5, 2e-5):
        p = orc.make_params(hstar=hs, a=0.25, dt=1e-3, flow=orc.FLOW_UNIAXIAL, Wi=3.0)
        res.append(orc.run(p, Nc, r, noise)[0])
    d1 = np.abs(res[1] - res[0]).max()
    d2 = np.abs(res[2] - res[0]).max()
    assert 0 < d1 < 1e-3
    np.testing.assert_allclose(d2 / d1, 2.0, rtol=0.05)   # linear in h*


@pytest.mark.slow
def test_dumbbell_rotational_diffusion():
    """<u(t).u(0)> = exp(-2 D_r t) with D_r = 2 (1 - mu_perp(b)) / b^2:
    at h* = a = 0.25, 2 D_r = 3.21875; at h* = 0, 2 D_r = 4."""
    n = 3000
    dt = 5e-4
    Nc = np.full(n, 2, np.int32)
    for hs, rate in ((0.0, 4.0), (0.25, 3.21875)):
        p = orc.make_params(hstar=hs, a=0.25, dt=dt)
        r = inputs.random_walk(Nc, 60)
        u0 = np.diff(r.reshape(n, 2, 3), axis=1)[:, 0]
        seed = 61
        for t_end in (0.1, 0.25):
            steps = int(round(t_end / dt)) - (0 if t_end == 0.1 else int(round(0.1 / dt)))
            r, *_ = orc.run(p, Nc, r, inputs.gaussian_noise(steps, 2 * n, seed))
            seed += 1
            u = np.diff(r.reshape(n, 2, 3), axis=1)[:, 0]
            c = (u * u0).sum(1)
            se = c.std(ddof=1) / np.sqrt(n)
            assert abs(c.mean() - np.exp(-rate * t_end)) < 3 * se + 0.01, (hs, t_end, c.mean())


def _equilibrium_samples(N, hs, n_chains, dt, t_burn, n_samp, t_gap, seed,
                         scheme=orc.SCHEME_MIDPOINT):
    p = orc.make_params(hstar=hs, a=0.25, dt=dt, tol=1e-12, scheme=scheme)
    Nc = np.full(n_chains, N, np.int32)
    r = inputs.random_walk(Nc, seed, stretched=True)
    k = seed + 1

    def adv(r, steps):
        nonlocal k
        r, T, st, it, md = orc.run(p, Nc, r, inputs.gaussian_noise(steps, n_chains * N, k))
        k += 1
        assert np.all(st == 0)
        return r

    r = adv(r, int(t_burn / dt))
    R2, Rg2, cs = [], [], []
    for _ in range(n_samp):
        r = adv(r, int(t_gap / dt))
        rr = r.reshape(n_chains, N, 3)
        R = rr[:, -1] - rr[:, 0]
        R2.append((R * R).sum(1))
        cm = rr.mean(1, keepdims=True)
        Rg2.append(((rr - cm) ** 2).sum(2).mean(1))
        Q = np.diff(rr, axis=1)
        cs.append((Q[:, :-1] * Q[:, 1:]).sum(2).mean(1))
    # per-chain time averages are independent across chains
    return [np.mean(x, axis=0) for x in (R2, Rg2, cs)]


def _se(x):
    return x.std(ddof=1) / np.sqrt(len(x))


@pytest.mark.slow
def test_equilibrium_statics_free_draining():
    """Freely-jointed statistics from a stretched start: <R^2> = (N-1) b^2,
    <Rg^2> = b^2 (N^2-1)/(6N), <u_k . u_k+1> = 0, each within 3 s.e."""
    N = 4
    R2, Rg2, cs = _equilibrium_samples(N, 0.0, 1500, 1e-3, 3.0, 8, 0.5, 70)
    assert abs(R2.mean() - (N - 1)) < 3 * _se(R2)
    assert abs(Rg2.mean() - (N * N - 1) / (6 * N)) < 3 * _se(Rg2)
    assert abs(cs.mean()) < 3 * _se(cs)


@pytest.mark.slow
def test_equilibrium_statics_euler_scheme_is_biased_with_hi():
    """The Euler projection (mobility and rod directions of the start of the
    step) lacks the HI part of the rigid-rod drift: at N = 4, h* = 0.25 it
    shifts <R^2> by a few percent.  The shift stays below 5 %."""
    N = 4
    R2, Rg2, cs = _equilibrium_samples(N, 0.25, 1500, 1e-3, 3.0, 8, 0.5, 80, orc.SCHEME_EULER)
    assert abs(R2.mean() / (N - 1) - 1) < 0.05
    assert abs(cs.mean()) < 0.05


@pytest.mark.slow
def test_equilibrium_statics_with_hi_strict():
    """Midpoint scheme, h* = 0.25: <R^2> = (N - 1) b^2, <Rg^2> = b^2 (N^2-1)/(6N)
    and <u_k . u_k+1> = 0, each within 3 s.e. (HI leaves the statics unchanged)."""
    N = 4
    R2, Rg2, cs = _equilibrium_samples(N, 0.25, 1500, 1e-3, 3.0, 8, 0.5, 90)
    assert abs(R2.mean() - (N - 1)) < 3 * _se(R2)
    assert abs(Rg2.mean() - (N * N - 1) / (6 * N)) < 3 * _se(Rg2)
    assert abs(cs.mean()) < 3 * _se(cs)


# <cos^2> of the bond angle of a rigid trimer.  Rigid constraints weight a
# conformation by sqrt(det G), G = A A^T the Gram matrix of the constraint
# gradients (2 on the diagonal, -cos(theta) off it), relative to the freely
# jointed measure: sqrt(4 - c^2) for a trimer, c = cos(theta).  Then
# <c^2> = int c^2 sqrt(4-c^2) dc / int sqrt(4-c^2) dc over [-1, 1]
#       = (pi/3 - sqrt(3)/4) / (sqrt(3)/2 + pi/3) = 0.32104...,
# against 1/3 for stiff springs (uniform c).
RIGID_TRIMER_COS2 = (np.pi / 3 - np.sqrt(3) / 4) / (np.sqrt(3) / 2 + np.pi / 3)


@pytest.mark.slow
@pytest.mark.parametrize("hs", [0.0, 0.25])
def test_rigid_trimer_bond_angle(hs):
    """<cos^2 theta> of a rigid trimer is the metric-weighted 0.3210, not the
    1/3 of stiff springs, with and without HI, within 3 s.e."""
    n = 2000
    p = orc.make_params(hstar=hs, a=0.25, dt=1e-3, tol=1e-12)
    Nc = np.full(n, 3, np.int32)
    r = inputs.random_walk(Nc, 93, stretched=True)
    r, *_ = orc.run(p, Nc, r, inputs.gaussian_noise(3000, 3 * n, 94))
    c2 = []
    for k in range(8):
        r, _, st, _, _ = orc.run(p, Nc, r, inputs.gaussian_noise(500, 3 * n, 95 + k))
        assert np.all(st == 0)
        Q = np.diff(r.reshape(n, 3, 3), axis=1)
        c2.append(((Q[:, 0] * Q[:, 1]).sum(1)) ** 2)
    c2 = np.mean(c2, axis=0)
    assert abs(c2.mean() - RIGID_TRIMER_COS2) < 3 * _se(c2), (c2.mean(), _se(c2))


def test_observables_closed_forms():
    """Straight chain along x: R_ee = (N-1, 0, 0), Rg^2 = (N^2-1)/12, stretch 1."""
    N = 9
    r = np.zeros((N, 3))
    r[:, 0] = np.arange(N)
    o = orc.observables(r)
    np.testing.assert_allclose(o[:3], [N - 1, 0, 0])
    np.testing.assert_allclose(o[3], (N - 1) ** 2)
    np.testing.assert_allclose(o[4], (N * N - 1) / 12.0, rtol=1e-14)
    np.testing.assert_allclose(o[5], 1.0)
    assert o[6] < 1e-15


def test_kramers_stress_closed_forms():
    """Rod part of the Kramers stress (Sec. 5 Eq. (28)) with the rod force
    T_k Q_k: a straight chain along x gives tau_xx = sum T and nothing else;
    along (1, 1, 0)/sqrt(2) it gives tau_xx = tau_yy = tau_xy = sum T / 2."""
    N = 5
    T = np.array([1.0, 2.0, -0.5, 3.0])
    r = np.zeros((N, 3))
    r[:, 0] = np.arange(N)
    o = orc.observables(r, T)
    np.testing.assert_allclose(o[8:12], [T.sum(), 0, 0, 0], atol=1e-15)
    d = np.array([1.0, 1.0, 0.0]) / np.sqrt(2)
    r2 = np.arange(N)[:, None] * d[None, :]
    o2 = orc.observables(r2, T)
    np.testing.assert_allclose(o2[8:12], [T.sum() / 2, T.sum() / 2, 0, T.sum() / 2], atol=1e-14)
    np.testing.assert_allclose(orc.observables(r)[8:12], 0.0)


def test_dumbbell_stress_in_extension():
    """Dumbbell along x after one noise-free step of uniaxial extension: the
    stress is the closed-form tension, N1 = tau_xx - tau_yy = rate/(2(1 - mu_par))."""
    rate, dt = 10.0, 1e-3
    p = orc.make_params(hstar=0.25, a=0.25, dt=dt, flow=orc.FLOW_UNIAXIAL, Wi=rate)
    r1, T, st, it, md = orc.step(p, np.array([[0.0, 0, 0], [1.0, 0, 0]]), np.zeros((2, 3)))
    o = orc.observables(r1, T)
    np.testing.assert_allclose(o[8] - o[9], rate / (2 * (1 - mu_far(1.0, 0.25, 0.25)[0])), rtol=1e-12)


# ------------------------------------------------ Fraenkel springs (Sec. 3)
def _fraenkel_params(**kw):
    base = dict(hstar=0.25, a=0.25, dt=1e-3, constraint=orc.FRAENKEL, kspring=1000.0)
    base.update(kw)
    return orc.make_params(**base)


def test_fraenkel_zero_stiffness_is_the_explicit_euler_step():
    """With K* = 0 there is no spring force and the semi-implicit update
    reduces to the explicit step r + dt kappa.r + y of Eq. (6): this checks
    the link update and the reconstruction of positions around the centre of
    mass together."""
    r = inputs.random_walk([9], 41)
    y = 1e-2 * inputs.gaussian_noise(1, 9, 42)[0]
    D = orc.assemble(r, 0.25, 0.25)
    kap = orc.kappa(orc.FLOW_SHEAR, 3.0)
    rn, T = orc.fraenkel_update(D, kap, 1e-3, 0.0, r, y)
    np.testing.assert_allclose(rn, r + 1e-3 * r @ kap.T + y, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(T, 0.0)


def test_fraenkel_free_draining_dumbbell_is_backward_euler():
    """h* = 0, no noise, no flow: the bond length of a dumbbell follows the
    backward-Euler step of dL/dt = -2 K* (L - 1), so after n steps
    L_n - 1 = (L_0 - 1) / (1 + 2 dt K*)^n, and the bond keeps its direction."""
    K, dt, L0, n = 50.0, 1e-3, 1.7, 25
    d = np.array([0.3, -0.4, np.sqrt(1 - 0.25)])
    r = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3]]) + np.vstack([np.zeros(3), L0 * d])
    p = _fraenkel_params(hstar=0.0, a=0.0, dt=dt, kspring=K)
    rr, T, st, it, md = orc.run(p, np.array([2], np.int32), r, np.zeros((n, 2, 3)))
    Q = rr[1] - rr[0]
    L = np.linalg.norm(Q)
    np.testing.assert_allclose(L - 1.0, (L0 - 1.0) / (1.0 + 2 * dt * K) ** n, rtol=1e-12)
    np.testing.assert_allclose(Q / L, d, atol=1e-14)
    np.testing.assert_allclose(rr.mean(0), r.mean(0), atol=1e-14)  # no net force, no drift
    np.testing.assert_allclose(T[0], K * (L - 1) / L, rtol=1e-12)


def test_fraenkel_dumbbell_with_hi_one_step():
    """With HI the coupling D_01 = mu_par along the bond stays explicit:
    |Y| = L_0 + 2 dt mu_par K* (L_0 - 1), and |Q'| = (2 dt K* + |Y|) / (2 dt K* + 1)
    (Eq. (25)), with mu_par the parallel RPY coefficient at R = L_0."""
    K, dt, L0, hs = 100.0, 1e-3, 1.5, 0.25
    r = np.array([[0.0, 0.0, 0.0], [L0, 0.0, 0.0]])
    mu_par = orc.rpy_block(np.array([L0, 0.0, 0.0]), hs, hs)[0, 0]
    # closed form of the far-field RPY parallel coefficient (Eq. (8)) as a cross-check
    np.testing.assert_allclose(mu_par, 0.75 * hs / L0 * (2 - 4 * hs * hs / (3 * L0 * L0)), rtol=1e-14)
    p = _fraenkel_params(hstar=hs, a=hs, dt=dt, kspring=K)
    rr, T, st, it, md = orc.run(p, np.array([2], np.int32), r, np.zeros((1, 2, 3)))
    Y = L0 + 2 * dt * mu_par * K * (L0 - 1)
    np.testing.assert_allclose(np.linalg.norm(rr[1] - rr[0]), (2 * dt * K + Y) / (2 * dt * K + 1), rtol=1e-13)


def test_fraenkel_stiff_limit_holds_unit_links():
    """K* -> infinity: |Q'| = (2 dt K* + |Y|) / (2 dt K* + 1) -> 1 for every link."""
    Nc = np.array([30], np.int32)
    r = inputs.random_walk(Nc, 43)
    p = _fraenkel_params(dt=1e-4, kspring=1e13)
    rr, T, st, it, md = orc.run(p, Nc, r, inputs.gaussian_noise(5, 30, 44))
    Q = np.linalg.norm(np.diff(rr, axis=0), axis=1)
    assert np.abs(Q - 1).max() < 1e-8


def _fraenkel_q2(K):
    """<|Q|^2> for the Fraenkel spring's Boltzmann weight Q^2 exp(-K (Q-1)^2 / 2)."""
    q = np.linspace(max(0.0, 1 - 12 / np.sqrt(K)), 1 + 12 / np.sqrt(K), 20001)
    w = q * q * np.exp(-0.5 * K * (q - 1) ** 2)
    return float((w * q * q).sum() / w.sum())


@pytest.mark.parametrize("hs", [0.0, 0.25])
def test_fraenkel_equilibrium_statics(hs):
    """Stiff springs (K* = 1000, dt = 1e-3, the paper's equilibrium settings):
    <R^2> = (N-1) <Q^2> and <Q_k . Q_k+1> = 0 within 3 s.e., with and without
    HI (RPY is divergence free, so the statics do not depend on h*)."""
    N, n_chains, K = 4, 1500, 1000.0
    p = _fraenkel_params(hstar=hs, a=0.25 if hs > 0 else 0.0, kspring=K)
    Nc = np.full(n_chains, N, np.int32)
    r = inputs.random_walk(Nc, 45 + int(hs * 100))
    key = [46]

    def adv(r, steps):
        r, T, st, it, md = orc.run(p, Nc, r, inputs.gaussian_noise(steps, n_chains * N, key[0]))
        key[0] += 1
        assert np.all(st == 0)
        return r

    r = adv(r, 1000)
    R2, cs = [], []
    for _ in range(8):
        r = adv(r, 500)
        rr = r.reshape(n_chains, N, 3)
        R = rr[:, -1] - rr[:, 0]
        R2.append((R * R).sum(1))
        Q = np.diff(rr, axis=1)
        cs.append((Q[:, :-1] * Q[:, 1:]).sum(2).mean(1))
    R2, cs = np.mean(R2, axis=0), np.mean(cs, axis=0)
    assert abs(R2.mean() - (N - 1) * _fraenkel_q2(K)) < 3 * _se(R2)
    assert abs(cs.mean()) < 3 * _se(cs)
