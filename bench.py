#!/usr/bin/env python3
"""Throughput benchmark of the bead-rod BD time step with HI on GB300.

Default workload: 64 chains of N = 1000 beads (D is 3000 x 3000 per chain),
h* = 0.25, simple shear at Wi = 100 (lambda = 1), dt = 1e-4, seeded random-walk
initial conformations and N(0,1) noise.  The mixed-precision path is the
headline; the FP64 path runs the same chains on the same GPU for the ratio.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line is printed by rank 0.  Under torchrun every rank advances its
own replica batch (independent chains, disjoint seeds, no data exchange: weak
scaling); the timing barrier and the max-over-ranks time are the only
collectives.  ``--impl reference`` times the FP64 CPU oracle on the host cores
instead (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2208_06559_gb300 import inputs, replicas  # noqa: E402

METRIC = "chain-timesteps/s at N=1000 (mixed vs FP64, same GPU); Cholesky % tensor peak"
# DRAM bytes read by one mixed factorisation per chain of N = 1000 (1624.9 MB for 16 chains;
# the written tiles stay in L2 during the captured launches): ncu capture of the factorisation
# of 16 chains with the tuned shape.
FACTOR_TRAFFIC_PER_CHAIN_N1000 = 1624.8e6 / 16
UNIT = "chain-timesteps/s"


def factor_tensor_peak(n, bf16_tflops):
    """Tensor peak (TFLOP/s) of the mixed factorisation of chains of order n.

    The panel solves multiply TF32 operands (0.5 x the bf16 rate, the nominal
    1.1 / 2.25 PF ratio), the trailing updates FP16 ones (the bf16 rate).
    With T = ceil(n / 128) tiles per chain the panel solves are T(T-1)/2 tile
    products and the updates (T-1)T(T+1)/6; the peak is the flop-weighted
    harmonic mean of the two rates.  Returns (peak, tf32 peak, TF32 share);
    chains of a single tile have no tile products and get the TF32 peak.
    """
    tf32 = bf16_tflops * 0.5
    T = np.ceil(np.asarray(n, np.float64) / 128.0)
    trsm_tiles = float(np.sum(T * (T - 1) / 2))
    upd_tiles = float(np.sum((T - 1) * T * (T + 1) / 6))
    if trsm_tiles + upd_tiles == 0:
        return tf32, tf32, 1.0
    f_tf32 = trsm_tiles / (trsm_tiles + upd_tiles)
    return 1.0 / (f_tf32 / tf32 + (1.0 - f_tf32) / bf16_tflops), tf32, f_tf32


def hbm_roofline(algorithmic_bytes, ms, hbm_gbs):
    """Roofline entry of an HBM-bound stage: algorithmic bytes per launch over
    the launch's CUDA-event time, against the measured copy bandwidth."""
    gbs = algorithmic_bytes / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs,
            "algorithmic_bytes_per_launch": algorithmic_bytes, "ms_per_launch": ms}


def cpu_model() -> str:
    """The host CPU's model string (x86 'model name', or the Arm implementer
    and part numbers), for the record beside the oracle's timing."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return "unknown"
    for line in info.splitlines():
        if line.lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    impl = part = None
    for line in info.splitlines():
        key = line.split(":", 1)[0].strip().lower()
        if key == "cpu implementer" and impl is None:
            impl = line.split(":", 1)[1].strip()
        elif key == "cpu part" and part is None:
            part = line.split(":", 1)[1].strip()
    if impl or part:
        return f"arm implementer {impl} part {part}"
    return "unknown"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(s[1]) for s in self.samples) if v is not None]
        mx = [v for v in (num(s[2]) for s in self.samples) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 5 + i and s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2208_06559_gb300 as bd

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = inputs.WORKLOADS[args.workload]
    Nc = w.lengths()
    total = int(Nc.sum())
    seed = replicas.replica_seed(w.seed, rank)      # disjoint replicas per rank
    r0_host = inputs.random_walk(Nc, seed)
    r0 = torch.from_numpy(r0_host).to(dev)
    K, W = args.steps, args.warmup
    noise_host = inputs.gaussian_noise(K + W + 2, total, seed + 1)
    noise = torch.from_numpy(noise_host).to(dev)
    peaks, peak_src = load_peaks()
    stream = torch.cuda.current_stream()
    prec = {"fp64": bd.FP64, "tf32": bd.MIXED_TF32}[args.precision] if args.precision else \
        (bd.MIXED_TF32 if w.precision != 0 else bd.FP64)
    scheme = {"midpoint": bd.SCHEME_MIDPOINT, "euler": bd.SCHEME_EULER}[args.scheme]
    kw = dict(h_star=w.hstar, dt=w.dt, flow=w.flow, Wi=w.Wi, tol=args.tol, constraint=w.constraint,
              k_spring=w.kspring, scheme=scheme)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    tuned = {}
    lanes_used = {}

    def timed_steps(p, nsteps, nwarm):
        ctx = bd.Context(Nc, precision=p, **kw)
        lanes_used[p] = ctx.lanes()
        ctx.set_state(r0)
        if p != bd.FP64 and not args.no_tune:   # tile shapes of the tensor-core factorisation
            pan, grp, tms = ctx.tune_factor()
            tuned.update(panel=pan, groups=grp, tuned_factor_ms=tms)
        for i in range(nwarm):
            ctx.step(noise[i:i + 1])
        barrier()
        l0 = ctx.kernel_launches()
        e0, e1 = ev(), ev()
        barrier()
        e0.record(stream)
        ctx.step(noise[nwarm:nwarm + nsteps])
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        launches = ctx.kernel_launches() - l0
        obs, st = ctx.observables()
        return ctx, ms, launches, st, obs

    with ClockSampler(local_rank) as clk:
        ctx, ms, launches, st, obs = timed_steps(prec, K, W)
    units, ms_max = replicas.aggregate(ms, len(Nc) * K, world, device=dev)
    value = units / (ms_max / 1e3)

    # Stage times on the same context, CUDA events on the launching stream.
    # The dominant stage is the Cholesky factorisation (assembly re-run
    # before each factorisation, outside the timed interval).
    reps = 3
    fms = 0.0
    for _ in range(reps):
        a, b = ev(), ev()
        ctx.assemble()
        a.record(stream)
        ctx.factor()
        b.record(stream)
        torch.cuda.synchronize()
        fms += a.elapsed_time(b)
    fms /= reps
    stage = {"factor_ms": fms}
    f = noise[0]
    for name, fn in (("assemble_ms", ctx.assemble), ("brownian_ms", lambda: ctx.brownian(f)),
                     ("mobility_symv_ms", lambda: ctx.mobility_apply(f))):
        fn()
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        stage[name] = a.elapsed_time(b) / reps
    newton = ctx.chain_status()[1]
    stage["newton_iterations_last_step_max"] = int(newton.max())
    ctx.close()

    n = 3 * Nc.astype(np.float64)
    chol_flops = float(np.sum(n ** 3) / 3.0)
    achieved_tf = chol_flops / (fms / 1e3) / 1e12
    esize = 8 if prec == bd.FP64 else 4
    symv_bytes = float(np.sum(n * n / 2.0)) * esize   # upper triangle read once
    # algorithmic bytes of the assembly: the lower triangle of D, n^2/2 elements
    # (the kernel writes both triangles, twice that, so that the factor can
    # overwrite the lower one while D stays in the upper one)
    assemble_bytes = float(np.sum(n * n / 2.0)) * esize
    if prec == bd.FP64:
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": 1.252, "unit": "TFLOP/s",
                "peak_source": "measured FP64 FMA throughput of this GPU (1.252 TFLOP/s)",
                "kernel": "cholesky factorisation (FP64, CUDA cores)"}
    else:
        peak, tf32, f_tf32 = factor_tensor_peak(n, peaks["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": achieved_tf, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"flop-weighted: panel solves TF32 = 0.5 x bf16 burst, trailing updates "
                               f"FP16 = bf16 burst ({peak_src}); TF32 share of the tile flops {f_tf32:.3f}",
                "kernel": "cholesky factorisation (tcgen05: TF32 panel solves, FP16-operand trailing "
                          "updates; FP32 diagonal tiles)",
                "frac_of_tf32_peak": achieved_tf / tf32}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM bytes of one factorisation from ncu (dram__bytes_read.sum + dram__bytes_write.sum over
    # its launches) on 16 chains of N = 1000 with the tuned shape, scaled to the chains here;
    # profiles/factorisation_traffic_n1000x16_mixed.md.  Other workloads: not captured.
    roof["traffic"] = (FACTOR_TRAFFIC_PER_CHAIN_N1000 * len(Nc)
                       if prec != bd.FP64 and int(Nc.min()) == 1000 == int(Nc.max()) else None)
    if roof["traffic"] is not None:
        roof["traffic_source"] = "ncu, 16 chains x N=1000 (panel 16, 4 groups), scaled by chains"
        roof["algorithmic_bytes_per_launch"] = float(np.sum((np.ceil(n / 128) * 128) ** 2)) * 4.0  # lower triangle read + written
    roof["algorithmic_flops_per_launch"] = chol_flops
    roof["ms_per_launch"] = fms
    others = {"mobility_symv": hbm_roofline(symv_bytes, stage["mobility_symv_ms"], peaks["hbm_gbs"]),
              "rpy_assembly": hbm_roofline(assemble_bytes, stage["assemble_ms"], peaks["hbm_gbs"])}
    others["rpy_assembly"]["bytes_written_per_launch"] = 2.0 * assemble_bytes

    # FP64 path on the same chains (the ratio of the metric)
    fp64 = None
    if prec != bd.FP64 and not args.skip_fp64:
        k64 = max(1, min(args.fp64_steps, K))
        ctx64, ms64, _, st64, _ = timed_steps(bd.FP64, k64, 1)
        ctx64.close()
        u64, m64 = replicas.aggregate(ms64, len(Nc) * k64, world, device=dev)
        v64 = u64 / (m64 / 1e3)
        fp64 = {"value": v64, "ms_per_step": m64 / k64, "steps": k64,
                "speedup_mixed_over_fp64": value / v64, "chain_status_ok": bool((st64 == 0).all())}

    # End to end through the public API with host buffers: every step the
    # noise goes host (pinned) -> device and the per-chain observables come back.
    e2e = None
    if not args.skip_e2e:
        ctx = bd.Context(Nc, precision=prec, **kw)
        ctx.set_state(r0)
        if tuned.get("panel"):
            bd.lib().bd_set_factor_config(ctx._h, tuned["panel"], tuned["groups"])
        pinned = torch.from_numpy(noise_host).pin_memory()
        obs_host = torch.empty((len(Nc), bd.OBS_STRIDE), dtype=torch.float64).pin_memory()
        ctx.step(pinned[0:1])
        ctx.observables(out=obs_host, with_status=False)
        barrier()
        ke = max(1, min(K, args.e2e_steps))
        t0 = time.perf_counter()
        for i in range(ke):
            ctx.step(pinned[W + i:W + i + 1])
            ctx.observables(out=obs_host, with_status=False)
        torch.cuda.synchronize()
        el = (time.perf_counter() - t0) * 1e3
        ctx.close()
        ue, me = replicas.aggregate(el, len(Nc) * ke, world, device=dev)
        e2e = {"value": ue / (me / 1e3), "unit": UNIT, "h2d_bytes_per_step": total * 3 * 8,
               "d2h_bytes_per_step": len(Nc) * bd.OBS_STRIDE * 8, "steps": ke}

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = cpu_baseline(w, Nc, r0_host, noise_host, args.cpu_chains, args.scheme)

    if rank == 0:
        tile = 32 if prec == bd.FP64 else 128
        mat_gb = float(np.sum((np.ceil(n / tile) * tile) ** 2)) * esize / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if prec == bd.FP64 else "f32",
            "dtype_detail": "f64 throughout" if prec == bd.FP64 else
                            "f32 storage and arithmetic; tf32 (panel solves) and f16 (trailing updates) "
                            "tensor-core operands with f32 accumulation; f32 diagonal tiles; "
                            "double-float (f64-accurate) tension-solve products",
            "data": "synthetic (seeded random-walk chains, N(0,1) noise)",
            "config": {"workload": w.name, "n_chains_per_gpu": len(Nc), "n_beads": int(Nc.max()),
                       "hstar": w.hstar, "a": w.hstar, "dt": w.dt,
                       "flow": ["none", "shear", "uniaxial"][w.flow], "Wi": w.Wi, "lambda": 1.0,
                       "newton_tol": args.tol,
                       "constraint": ["rigid", "fraenkel"][w.constraint],
                       **({"scheme": args.scheme} if w.constraint == 0 else {}),
                       **({"k_spring": w.kspring} if w.constraint == 1 else {}),
                       "precision": "fp64" if prec == bd.FP64 else "mixed_tf32_refined",
                       "l2": f"inputs larger than L2 (per-step matrices {mat_gb:.1f} GB)",
                       "lanes": lanes_used.get(prec, 1),
                       "parallelism": f"independent replicas x{world}"},
            "roofline": roof, "rooflines_other": others, "stages": stage, "factor_shape": tuned,
            "fp64": fp64,
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(),
            "cpu_baseline": cpu, "chain_status_ok": bool((st == 0).all()),
            "max_rod_length_error": float(obs[:, bd.binding.OBS_MAXDEV].max().item()),
        }
        print(json.dumps(line))


def cpu_baseline(w, Nc, r0, noise_host, max_chains, scheme="midpoint"):
    import oracle as orc
    cores = orc.num_threads()
    S = int(min(len(Nc), max(1, min(cores, max_chains))))
    p = orc.make_params(hstar=w.hstar, dt=w.dt, flow=w.flow, Wi=w.Wi, constraint=w.constraint,
                        kspring=w.kspring, scheme=0 if scheme == "midpoint" else 1)
    Ns = Nc[:S]
    rs = r0[: int(Ns.sum())]
    nz = np.ascontiguousarray(noise_host[:1, : int(Ns.sum())])
    t0 = time.perf_counter()
    orc.run(p, Ns, rs, nz)
    el = time.perf_counter() - t0
    return {"value": S / el, "unit": UNIT, "cores": min(cores, S), "kind": "oracle",
            "sample": f"{S} chains x 1 step of the workload (N={int(Nc.max())}), OpenMP over chains",
            "host_cpus": os.cpu_count(), "cpu_model": cpu_model()}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as orc
    w = inputs.WORKLOADS[args.workload]
    Nc = w.lengths()
    cores = orc.num_threads()
    S = int(min(len(Nc), max(1, min(cores, args.cpu_chains))))
    Ns = Nc[:S]
    r = inputs.random_walk(Ns, w.seed)
    noise = inputs.gaussian_noise(args.steps + args.warmup, int(Ns.sum()), w.seed + 1)
    p = orc.make_params(hstar=w.hstar, dt=w.dt, flow=w.flow, Wi=w.Wi, tol=args.tol,
                        constraint=w.constraint, kspring=w.kspring,
                        scheme=0 if args.scheme == "midpoint" else 1)
    for i in range(args.warmup):
        r, *_ = orc.run(p, Ns, r, noise[i:i + 1])
    t0 = time.perf_counter()
    for i in range(args.steps):
        r, *_ = orc.run(p, Ns, r, noise[args.warmup + i:args.warmup + i + 1])
    el = time.perf_counter() - t0
    v = S * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random-walk chains, N(0,1) noise)",
            "config": {"workload": w.name, "n_chains_sampled": S, "n_beads": int(Nc.max()),
                       "hstar": w.hstar, "dt": w.dt, "Wi": w.Wi, "newton_tol": args.tol},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": min(cores, S), "kind": "oracle",
                             "sample": f"{S} of {len(Nc)} chains per step, FP64 CPU oracle",
                             "host_cpus": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n1000x64_mixed_shear", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp64", "tf32"])
    ap.add_argument("--tol", type=float, default=1e-13)
    ap.add_argument("--scheme", default="midpoint", choices=["midpoint", "euler"],
                    help="rigid-rod step: midpoint corrector (default) or the Euler projection")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-chains", type=int, default=16)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local_rank = replicas.rank_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
