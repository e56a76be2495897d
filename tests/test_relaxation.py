"""Relaxation time lambda (Sec. 5): autocorrelation of the end-to-end vector
and the exponential fit to its last 70 %.  The rigid dumbbell with HI has a
closed form: <R(t) . R(0)> = exp(-2 D_r t) with 2 D_r = 4 (1 - mu_perp) / b^2,
so lambda = 1 / (2 D_r) (= 0.310680 at h* = a = 0.25, b = 1)."""
import numpy as np
import pytest

import oracle as orc
from paper_2208_06559_gb300 import inputs
from paper_2208_06559_gb300.relaxation import autocorrelation, fit_relaxation_time, truncate

MU_PERP = 0.1953125                  # RPY perpendicular coefficient at R = 1, h* = a = 0.25
LAMBDA_DUMBBELL = 1.0 / (4.0 * (1.0 - MU_PERP))


def test_fit_recovers_an_exponential_tail():
    t = np.linspace(0.0, 3.0, 301)
    C = 0.93 * np.exp(-t / 0.37)
    C[:40] += 0.05 * np.exp(-t[:40] / 0.01)  # short-time part outside the fit window
    lam, A = fit_relaxation_time(t, C)
    assert abs(lam - 0.37) < 1e-9 and abs(A - 0.93) < 1e-9


def test_autocorrelation_definitions():
    rng = np.random.default_rng(1)
    R0 = rng.standard_normal((5, 3))
    R = np.stack([R0 * (-1) ** k for k in range(10)])  # flips every sample
    np.testing.assert_allclose(autocorrelation(R, 4), [1, -1, 1, -1, 1])
    np.testing.assert_allclose(autocorrelation(np.stack([R0] * 6), 5), np.ones(6))


def _dumbbell_series(n_chains, dt, n_samples, every, seed):
    p = orc.make_params(hstar=0.25, a=0.25, dt=dt, tol=1e-13)
    Nc = np.full(n_chains, 2, np.int32)
    r = inputs.random_walk(Nc, seed)
    R = np.empty((n_samples, n_chains, 3))
    key = seed + 1
    for s in range(n_samples):
        if s:
            r, T, st, it, md = orc.run(p, Nc, r, inputs.gaussian_noise(every, 2 * n_chains, key))
            key += 1
            assert np.all(st == 0)
        rr = r.reshape(n_chains, 2, 3)
        R[s] = rr[:, 1] - rr[:, 0]
    return R


def test_dumbbell_relaxation_time_closed_form():
    """1500 rigid dumbbells with HI, lags up to 3.2 lambda, each lag averaged
    over at least 100 time origins: the fitted lambda matches
    1 / (4 (1 - mu_perp)) within 4 %."""
    dt, every = 1e-3, 10
    R = _dumbbell_series(1500, dt, 201, every, 301)
    C = autocorrelation(R, 100)
    t = dt * every * np.arange(len(C))
    lam, A = fit_relaxation_time(t, C)
    assert abs(lam / LAMBDA_DUMBBELL - 1) < 0.04, lam
    assert abs(A - 1) < 0.05


@pytest.mark.gpu
def test_gpu_relaxation_pipeline_matches_oracle():
    """measure() on the GPU (FP64) against the same pipeline fed by the
    oracle's trajectories (same seeds and noise chunks): the trajectories agree
    to round-off, so the two lambdas agree to 1e-6; both match the dumbbell's
    closed form."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_06559_gb300 import build as b
    b.build()
    from paper_2208_06559_gb300.relaxation import measure
    n_chains, dt, every, t_max, seed = 512, 1e-3, 10, 1.0, 303
    t, C, lam, A = measure(2, n_chains, dt, t_max, every, seed, chunk=every)
    R = _dumbbell_series(n_chains, dt, len(t) * 2 - 1, every, seed)
    C_ref = autocorrelation(R, len(t) - 1)
    n_fit = max(truncate(C_ref, 0.05), 4)
    lam_ref, _ = fit_relaxation_time(t[:n_fit], C_ref[:n_fit])
    np.testing.assert_allclose(C, C_ref, rtol=0, atol=1e-9)
    assert abs(lam / lam_ref - 1) < 1e-6
    assert abs(lam / LAMBDA_DUMBBELL - 1) < 0.08
