"""Stage timing and profiling driver for libbd.

    python -m paper_2208_06559_gb300.stages --chains 64 --beads 1000 --precision tf32 [--reps 3]

Creates one context on cuda:0 with seeded random-walk chains, then times each
stage of the time step through the C ABI with CUDA events on the launching
stream (assembly, Cholesky factorisation, Brownian displacement, mobility
product, one full step) and prints one JSON line.  ``--timeline`` prints the
stage-boundary times of one step launched kernel by kernel (bd_profile_step).  ``--once`` runs every
stage exactly once without timing (a short, fixed launch sequence for
kernel profilers).
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
    ap.add_argument("--precision", default="tf32", choices=["fp64", "tf32"])
    ap.add_argument("--flow", type=int, default=1)
    ap.add_argument("--Wi", type=float, default=100.0)
    ap.add_argument("--dt", type=float, default=1e-4)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--scheme", default="midpoint", choices=["midpoint", "euler"])
    ap.add_argument("--panel", type=int, default=0, help="factorisation super-panel width (mixed; 0: default)")
    ap.add_argument("--groups", type=int, default=0, help="factorisation chain groups (mixed; 0: default)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--once", action="store_true")
    ap.add_argument("--sweep", default="", help="comma-separated bead counts: time one step per N")
    ap.add_argument("--timeline", action="store_true",
                    help="stage-boundary times of one step launched kernel by kernel")
    ap.add_argument("--lanes", type=int, default=0,
                    help="concurrent sub-batches of a mixed context (0: the library's choice); a "
                         "timeline of several lanes sums the lanes' times, profiled one after another")
    a = ap.parse_args()
    if a.sweep:
        sweep(a)
        return

    prec = bd.FP64 if a.precision == "fp64" else bd.MIXED_TF32
    Nc = np.full(a.chains, a.beads, np.int32)
    r0 = torch.from_numpy(inputs.random_walk(Nc, a.seed)).cuda()
    ctx = bd.Context(Nc, flow=a.flow, Wi=a.Wi, dt=a.dt, precision=prec,
                     scheme=bd.SCHEME_MIDPOINT if a.scheme == "midpoint" else bd.SCHEME_EULER, lanes=a.lanes)
    ctx.set_state(r0)
    if prec != bd.FP64 and a.panel > 0:
        bd.lib().bd_set_factor_config(ctx._h, a.panel, a.groups if a.groups > 0 else 1)
    xi = torch.from_numpy(inputs.gaussian_noise(a.reps + 3, int(Nc.sum()), a.seed + 1)).cuda()
    if a.timeline:
        ctx.step(xi[0:1])
        tl = ctx.profile_step(xi[1])
        tl = ctx.profile_step(xi[2])
        print(json.dumps({"chains": a.chains, "beads": a.beads, "precision": a.precision,
                          **{k: round(v, 4) for k, v in tl.items()}}))
        return
    if a.once:
        ctx.assemble()
        ctx.factor()
        ctx.brownian(xi[0])
        ctx.mobility_apply(xi[1])
        ctx.step(xi[2:3])
        torch.cuda.synchronize()
        st, _ = ctx.chain_status()
        print(json.dumps({"ok": bool((st == 0).all())}))
        return

    def ev():
        return torch.cuda.Event(enable_timing=True)

    res = {}

    def timeit(name, fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(a.reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / a.reps

    timeit("assemble_ms", ctx.assemble)
    ts = []
    for _ in range(a.reps):
        ctx.assemble()
        e0, e1 = ev(), ev()
        e0.record()
        ctx.factor()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    res["factor_ms"] = sum(ts) / len(ts)
    timeit("brownian_ms", lambda: ctx.brownian(xi[0]))
    timeit("mobility_ms", lambda: ctx.mobility_apply(xi[1]))
    ctx.step(xi[0:1])
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    ctx.step(xi[1:1 + a.reps])
    e1.record()
    torch.cuda.synchronize()
    res["step_ms"] = e0.elapsed_time(e1) / a.reps
    st, it = ctx.chain_status()
    n = 3.0 * Nc
    res["factor_tflops"] = float(np.sum(n ** 3) / 3) / (res["factor_ms"] * 1e-3) / 1e12
    res["newton_iterations"] = int(it.max())
    res["status_ok"] = bool((st == 0).all())
    print(json.dumps({"chains": a.chains, "beads": a.beads, "precision": a.precision,
                      **{k: (round(v, 4) if isinstance(v, float) else v) for k, v in res.items()}}))


def sweep(a):
    """Step time against chain length (the paper's N-scaling study, Sec. 5):
    one line per N with the step time, the factorisation time and a power-law
    exponent fitted to the step times."""
    import torch

    import paper_2208_06559_gb300 as bd
    from paper_2208_06559_gb300 import inputs

    prec = bd.FP64 if a.precision == "fp64" else bd.MIXED_TF32
    rows = []
    for N in [int(x) for x in a.sweep.split(",")]:
        Nc = np.full(a.chains, N, np.int32)
        ctx = bd.Context(Nc, flow=a.flow, Wi=a.Wi, dt=a.dt, precision=prec, lanes=a.lanes)
        ctx.set_state(torch.from_numpy(inputs.random_walk(Nc, a.seed)).cuda())
        xi = torch.from_numpy(inputs.gaussian_noise(a.reps + 1, int(Nc.sum()), a.seed + 1)).cuda()
        ctx.step(xi[0:1])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.step(xi[1:])
        e1.record()
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / a.reps
        ctx.assemble()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        ctx.factor()
        f1.record()
        torch.cuda.synchronize()
        st, _ = ctx.chain_status()
        ctx.close()
        rows.append({"N": N, "chains": a.chains, "step_ms": round(step_ms, 4),
                     "factor_ms": round(f0.elapsed_time(f1), 4),
                     "chain_steps_per_s": round(a.chains / (step_ms / 1e3), 1),
                     "status_ok": bool((st == 0).all())})
        print(json.dumps(rows[-1]), flush=True)
    if len(rows) >= 2:
        x = np.log([r["N"] for r in rows])
        y = np.log([r["step_ms"] for r in rows])
        fit = {"fit_step_time_exponent": float(np.polyfit(x, y, 1)[0]), "precision": a.precision}
        big = [r for r in rows if r["N"] >= 2000]
        if len(big) >= 2:   # the large-chain regime the paper fits separately (Sec. 5)
            fit["fit_step_time_exponent_N_ge_2000"] = float(
                np.polyfit(np.log([r["N"] for r in big]), np.log([r["step_ms"] for r in big]), 1)[0])
        print(json.dumps(fit))


if __name__ == "__main__":
    main()
