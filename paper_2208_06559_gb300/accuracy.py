"""Accuracy of the mixed-precision path against the FP64 path, per result.

    python -m paper_2208_06559_gb300.accuracy --chains 64 --beads 1000 --steps 100

Reports, as one JSON line:
  * factor_backward_error: ||B B^T - D||_F / ||D||_F against the FP64 D, for
    the raw TF32 factor B = L and for the refined factor
    B_eff = (L + D32 L^{-T}) / 2 (D32: the stored FP32 D that the refinement
    multiplies by), formed densely in FP64 on the host from the library's own
    matrices for a few sampled chains;
  * displacement_error: max |dr_mixed - dr_fp64| / max |dr_fp64| for one step
    from the same state with the same noise;
  * ensemble: <R^2> and mean stretch |R_ee| / (N - 1) after --steps steps of
    both paths from the same states with the same noise, with standard errors
    over chains and the difference in units of the combined standard error.
The FP64 path is the reference here because it matches the FP64 CPU oracle
to 1e-10 (tests/test_gpu_parity.py).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    import torch

    import paper_2208_06559_gb300 as bd
    from paper_2208_06559_gb300 import inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("--chains", type=int, default=64)
    ap.add_argument("--beads", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--flow", type=int, default=1)
    ap.add_argument("--Wi", type=float, default=100.0)
    ap.add_argument("--dt", type=float, default=1e-4)
    ap.add_argument("--seed", type=int, default=1237)
    ap.add_argument("--sample-chains", type=int, default=2)
    a = ap.parse_args()

    Nc = np.full(a.chains, a.beads, np.int32)
    r0 = torch.from_numpy(inputs.random_walk(Nc, a.seed)).cuda()
    noise = torch.from_numpy(inputs.gaussian_noise(a.steps, int(Nc.sum()), a.seed + 1)).cuda()
    kw = dict(h_star=0.25, dt=a.dt, flow=a.flow, Wi=a.Wi)
    out = {"chains": a.chains, "beads": a.beads, "steps": a.steps, "flow": a.flow, "Wi": a.Wi}

    # factor backward error against the FP64 D, raw and refined
    mx = bd.Context(Nc, precision=bd.MIXED_TF32, **kw)
    f64 = bd.Context(Nc, precision=bd.FP64, **kw)
    for c in (mx, f64):
        c.set_state(r0)
        c.assemble()
    mx.factor()
    raw, raw_dev, ref = [], [], []
    for c in range(min(a.sample_chains, a.chains)):
        raw_dev.append(mx.factor_residual(c))
        L = mx.read_matrix(c, 1)
        D32 = mx.read_matrix(c, 0)
        D = f64.read_matrix(c, 0)
        nD = np.linalg.norm(D)
        raw.append(float(np.linalg.norm(L @ L.T - D) / nD))
        Beff = 0.5 * (L + D32 @ np.linalg.inv(L).T)
        ref.append(float(np.linalg.norm(Beff @ Beff.T - D) / nD))
    out["factor_backward_error"] = {"raw_tf32": max(raw), "raw_tf32_device": max(raw_dev),
                                    "refined": max(ref), "chains_sampled": len(raw)}
    mx.close()
    f64.close()

    # one-step displacement error
    res = {}
    for name, prec in (("mixed", bd.MIXED_TF32), ("fp64", bd.FP64)):
        c = bd.Context(Nc, precision=prec, **kw)
        c.set_state(r0)
        c.step(noise[0:1])
        res[name] = (c.get_state() - r0).cpu().numpy()
        c.close()
    out["displacement_error"] = float(np.abs(res["mixed"] - res["fp64"]).max() /
                                      np.abs(res["fp64"]).max())

    # ensemble statistics after `steps` steps
    ens = {}
    for name, prec in (("mixed", bd.MIXED_TF32), ("fp64", bd.FP64)):
        c = bd.Context(Nc, precision=prec, **kw)
        c.set_state(r0)
        c.step(noise)
        obs, st = c.observables()
        o = obs.cpu().numpy()
        c.close()
        R2, s = o[:, bd.binding.OBS_R2], o[:, bd.binding.OBS_STRETCH]
        ens[name] = {"R2_mean": float(R2.mean()), "R2_se": float(R2.std(ddof=1) / np.sqrt(len(R2))),
                     "stretch_mean": float(s.mean()), "stretch_se": float(s.std(ddof=1) / np.sqrt(len(s))),
                     "status_ok": bool((st == 0).all())}
    for q in ("R2", "stretch"):
        d = ens["mixed"][q + "_mean"] - ens["fp64"][q + "_mean"]
        se = np.hypot(ens["mixed"][q + "_se"], ens["fp64"][q + "_se"])
        ens[q + "_difference_in_se"] = float(d / se)
    out["ensemble"] = ens
    print(json.dumps(out))


if __name__ == "__main__":
    main()
