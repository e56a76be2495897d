"""Relaxation time of the chain (Sec. 5): the time scale of the decay of the
autocorrelation of the end-to-end vector, from an exponential fitted to the
last 70 % of that autocorrelation (taken up to where it first drops below a
cutoff, 0.05 by default, beyond which it is noise).

    python -m paper_2208_06559_gb300.relaxation --beads 2,4,8,16 --chains 512 --dt 1e-3 --t-max 20

``autocorrelation`` and ``fit_relaxation_time`` are plain numpy and take the
sampled end-to-end vectors from any source; ``measure`` runs equilibrium
chains (no flow) through the library on the GPU.  The printed JSON lines give
lambda per chain length and the exponent of lambda against N (the paper's
equilibrium scaling check, Sec. 5).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def autocorrelation(R: np.ndarray, max_lag: int) -> np.ndarray:
    """Normalised autocorrelation <R(t0 + k) . R(t0)> / <R(t0) . R(t0)> of the
    end-to-end vectors R [n_samples][n_chains][3] for lags k = 0 .. max_lag,
    averaged over chains and over every time origin t0."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    max_lag = min(max_lag, n - 1)
    c = np.empty(max_lag + 1)
    for k in range(max_lag + 1):
        c[k] = np.mean(np.sum(R[k:] * R[: n - k], axis=2))
    return c / c[0]


def truncate(C: np.ndarray, cutoff: float = 0.05) -> int:
    """Number of leading points of C before it first drops below `cutoff`
    (the part of the autocorrelation that is still signal, not noise)."""
    below = np.nonzero(np.asarray(C) < cutoff)[0]
    return int(below[0]) if len(below) else len(C)


def fit_relaxation_time(t: np.ndarray, C: np.ndarray, fraction: float = 0.7):
    """Fit C(t) = A exp(-t / lambda) to the last `fraction` of the points
    (the window that excludes the short-time, non-exponential start).
    Least squares in C itself, started from the log-linear fit of the
    positive points and refined by Gauss-Newton (kept only while it stays
    finite and decaying).  Returns (lambda, A)."""
    t = np.asarray(t, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    i0 = int(round((1.0 - fraction) * (len(t) - 1)))
    tt, cc = t[i0:], C[i0:]
    pos = cc > 0
    if pos.sum() < 2:
        raise ValueError("autocorrelation has fewer than two positive points in the fit window")
    slope, icpt = np.polyfit(tt[pos], np.log(cc[pos]), 1)
    if not slope < 0:
        raise ValueError("autocorrelation does not decay in the fit window")
    lam, A = -1.0 / slope, float(np.exp(icpt))
    k = 1.0 / lam
    for _ in range(20):  # Gauss-Newton on (A, 1/lambda)
        e = np.exp(-k * tt)
        r = cc - A * e
        J = np.stack([e, -A * tt * e], axis=1)
        step, *_ = np.linalg.lstsq(J, r, rcond=None)
        A2, k2 = A + step[0], k + step[1]
        if not (np.isfinite(A2) and np.isfinite(k2) and k2 > 0):
            break
        A, k = A2, k2
        if abs(step[1]) < 1e-12 * abs(k):
            break
    return float(1.0 / k), float(A)


def measure(n_beads: int, n_chains: int, dt: float, t_max: float, sample_every: int, seed: int,
            h_star: float = 0.25, precision: int = 0, constraint: int = 0, k_spring: float = 1e4,
            t_burn: float = 0.0, chunk: int = 200, cutoff: float = 0.05):
    """Equilibrium run of n_chains chains of n_beads beads (no flow) on the
    GPU; returns (t, C, lambda, A) with the end-to-end autocorrelation C
    sampled every `sample_every` steps (lags up to half the run).  The fit
    covers the last 70 % of C up to where it first drops below `cutoff`."""
    import torch

    from . import binding as b
    from . import inputs

    Nc = np.full(n_chains, n_beads, np.int32)
    ctx = b.Context(Nc, h_star=h_star, dt=dt, precision=precision, constraint=constraint, k_spring=k_spring)
    ctx.set_state(torch.from_numpy(inputs.random_walk(Nc, seed)).cuda())
    total = int(Nc.sum())
    key = seed + 1

    def advance(steps):
        nonlocal key
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            ctx.step(torch.from_numpy(inputs.gaussian_noise(k, total, key)).cuda())
            key += 1
            done += k

    if t_burn > 0:
        advance(int(round(t_burn / dt)))
    n_samples = int(round(t_max / (dt * sample_every))) + 1
    R = np.empty((n_samples, n_chains, 3))
    for s in range(n_samples):
        if s:
            advance(sample_every)
        obs, st = ctx.observables()
        if not (st == 0).all():
            raise RuntimeError(f"chain status {st[st != 0][:4]} during the equilibrium run")
        R[s] = obs[:, b.OBS_REE_X:b.OBS_REE_X + 3].cpu().numpy()
    ctx.close()
    max_lag = n_samples // 2
    C = autocorrelation(R, max_lag)
    t = dt * sample_every * np.arange(len(C))
    n_fit = max(truncate(C, cutoff), 4)
    lam, A = fit_relaxation_time(t[:n_fit], C[:n_fit])
    return t, C, lam, A


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--beads", default="2,4,8,16")
    ap.add_argument("--chains", type=int, default=512)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--t-max", type=float, default=20.0)
    ap.add_argument("--sample-every", type=int, default=20)
    ap.add_argument("--h-star", type=float, default=0.25)
    ap.add_argument("--seed", type=int, default=2024)
    a = ap.parse_args()
    Ns, lams = [], []
    for N in [int(x) for x in a.beads.split(",")]:
        t, C, lam, A = measure(N, a.chains, a.dt, a.t_max, a.sample_every, a.seed + N, a.h_star)
        Ns.append(N)
        lams.append(lam)
        print(json.dumps({"N": N, "chains": a.chains, "lambda": lam, "amplitude": A, "dt": a.dt,
                          "t_max": a.t_max, "h_star": a.h_star}), flush=True)
    if len(Ns) >= 2:
        x, y = np.log(np.array(Ns, float)), np.log(np.array(lams))
        print(json.dumps({"fit_lambda_exponent": float(np.polyfit(x, y, 1)[0])}))


if __name__ == "__main__":
    main()
