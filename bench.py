"""Benchmark: particle-forces/s of the GB300 FMM at rms relative force error ~1e-7.

One step = one whole force evaluation (tree, scale estimate, upward pass, dual
walk, M2L, P2P, downward pass) of a seeded Plummer sphere of N = 1e6 particles
(G = 1, total mass 1, truncated at 30 scale radii), inputs resident in HBM.
Under torchrun every rank evaluates its own sphere (independent systems: weak
scaling, no collective on the data path); value = total particles / max time.

--impl reference times the CPU oracle (the plain serial FP64 FMM of oracle/) on
a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-forces/s at rms rel. force error 1e-7 vs plain FP64 GPU FMM; p99 latency"
UNIT = "particle-forces/s"
L2_FLUSH_BYTES = 256 << 20


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--p", type=int, default=None, help="expansion order (default: per workload, below)")
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--leaf", type=int, default=None)
    ap.add_argument("--c", type=float, default=None)
    ap.add_argument("--cpu-sample", type=int, default=50000)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64-mode and direct-sum comparisons")
    ap.add_argument("--workload", default="plummer", choices=["plummer", "cusp", "ensemble", "serve", "active"],
                    help="plummer: one N=1e6 sphere (default); cusp: gamma=1.5 model with a central point mass; "
                         "ensemble: 256 spheres of 1e3..1e5 in one forest; serve: 64 systems of 1e4..2e6 "
                         "served at 0.8 of capacity (Poisson arrivals); active: forces for the innermost "
                         "N_a of a Plummer sphere of 1e7 (Sec. 7.1), N_a = 1e3..1e7")
    ap.add_argument("--requests", type=int, default=384, help="serve: requests in the open-loop run")
    ap.add_argument("--slots", type=int, default=2, help="serve: concurrent slots of the request loop")
    ap.add_argument("--autotune", action="store_true",
                    help="choose (p, eps, leaf, p2p_c) for rms 1e-7 on the workload first (untimed)")
    ap.add_argument("--no-configs", action="store_true",
                    help="plummer: skip the sub-records of the cusp, ensemble and served-stream workloads")
    a = ap.parse_args(argv)
    if a.workload in ("cusp", "active") and a.n == 1_000_000:
        a.n = 10_000_000
    for k, v in zip(("p", "eps", "leaf", "c"), PARAMS[a.workload]):
        if getattr(a, k) is None:
            setattr(a, k, v)
    return a


# (p, eps, leaf, p2p_c) per workload from the autotuner at rms 1e-7 (eps with a margin; the
# Plummer sphere's on 10^5 sampled sinks, the truth sample of the bench, whose rms includes
# the few particles near the centre where |a| -> 0): the single large systems take leaf 80;
# ensembles of small systems leaf 48, where large leaves let accepted pairs with theta near 1
# dominate the error
PARAMS = {"plummer": (14, 2.3e-7, 80, 1.0), "cusp": (14, 2.6e-7, 80, 1.0),
          "ensemble": (14, 3.6e-7, 48, 1.0), "serve": (14, 2.0e-7, 48, 1.0),
          "active": (14, 2.3e-7, 80, 1.0)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ALU peaks derived from the unit counts and the maximum SM clock: SMs x 128 FP32 lanes x
# 2 flops (FFMA) x the maximum SM clock (the SM count and clock are read from the device);
# FP64 is the part's nominal 1.25 TFLOP/s
FP64_PEAK_TFLOPS = 1.25


def fp32_peak(dev=None):
    """(TFLOP/s, SM count, max SM MHz) of the FP32 FMA pipes of the device."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        q = subprocess.run(["nvidia-smi", f"--id={torch.cuda.current_device() if dev is None else dev.index}",
                            "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                           capture_output=True, text=True, timeout=20)
        mhz = float(q.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        pass
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz


def max_over_ranks(v, world, device=None):
    """Maximum of a per-rank float over all ranks (the slowest rank sets the job time)."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, world, device=None):
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_value(n_per_rank, world, seconds):
    """Whole-job throughput under weak scaling: every rank's particles over the max time."""
    return n_per_rank * world / seconds


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def m2l_flops(p):
    # complex MACs of eq. (3b) over the outputs n <= p, m >= 0: sum_n (n+1)(p-n+1)^2, 8 flops each
    return 8 * sum((n + 1) * (p - n + 1) ** 2 for n in range(p + 1))


def m2l_rot_flops(p):
    """FP32 flops per pair of the rotation-accelerated M2L (App. A.5), 2 per multiply-add:
    four z rotations (4 multiply-adds per m > 0 of each order), four swaps (one
    multiply-add per entry of the swap matrices' parity pattern: cosine block n+m+l even,
    sine block n+m+l odd; the restricted forward/backward swaps only the rows/columns
    |m| <= min(n, p-n)), the z-axis kernel eq. (A31) over n + k >= 3, and the scaling of
    the kept rotated multipoles and of the results."""
    def swap(n, lim_rows, lim_cols):
        c = sum(1 for m in range(n + 1) for l in range(n + 1) if (n + m + l) % 2 == 0 and m <= lim_rows and l <= lim_cols)
        c += sum(1 for m in range(1, n + 1) for l in range(1, n + 1) if (n + m + l) % 2 and m <= lim_rows and l <= lim_cols)
        return c
    fma = 0
    for n in range(p + 1):
        L = min(n, p - n)
        fma += 4 * 4 * n + 2 * swap(n, n, n) + swap(n, L, n) + swap(n, n, L) + (2 * L + 1) + (2 * n + 1)
        for m in range(L + 1):
            fma += (2 if m else 1) * sum(1 for k in range(max(m, 3 - n), p - n + 1))
    return 2 * fma


def oracle_run(n, p, eps, leaf, c, seed, model="plummer"):
    import oracle
    from paper_1405_2255_gb300 import inputs
    x, mu = (inputs.dehnen if model == "cusp" else inputs.plummer)(n, seed)
    t = time.perf_counter()
    oracle.fmm(x, mu, p=p, eps=eps, leaf_size=leaf, p2p_c=c, keep=False)
    return time.perf_counter() - t


def reference_arm(a, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    from paper_1405_2255_gb300 import inputs
    ns = a.cpu_sample
    seed = inputs.BASE_SEED + 2
    for _ in range(a.warmup):
        oracle_run(ns, a.p, a.eps, a.leaf, a.c, seed)
    ts = [oracle_run(ns, a.p, a.eps, a.leaf, a.c, seed) for _ in range(a.steps)]
    t = float(np.mean(ts))
    v = ns / t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(a),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"oracle FMM (serial C, FP64) on a Plummer sphere of N={ns} from the same "
                                   f"generator and parameters, one evaluation per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# DRAM bytes (read + write) per launch of the dominant kernels, from one ncu capture of
# the same workload and parameters (summaries and commands under profiles/); None for
# any other configuration or once the kernel has changed since the capture
MEASURED_TRAFFIC = {
    ("plummer", 1000000, 14, 2.3e-7, 80, 1.0, "mixed"): {"k_p2p_mixed": 90.4e6, "k_m2l_rot": 72.1e6},
}


def roofline(g, a, prec, phase, full):
    """Achieved vs peak of the dominant kernel: algorithmic flops of the run's own lists
    over that kernel's own launch duration (CUDA events recorded around the launch on its
    stream) averaged over the timed steps; also over its whole phase (list sort, work plan,
    reduction and kernel)."""
    t_m2l = float(np.mean([s["t_m2l"] for s in phase])) * 1e-3
    t_p2p = float(np.mean([s["t_p2p"] for s in phase])) * 1e-3
    k_m2l = float(np.mean([s["t_m2l_kernel"] for s in phase])) * 1e-3
    k_p2p = float(np.mean([s["t_p2p_kernel"] for s in phase])) * 1e-3
    if k_m2l <= 0.0 or k_p2p <= 0.0:  # a path without the marked kernels: the phases
        k_m2l, k_p2p = t_m2l, t_p2p
    loop64, loop32 = g.fmm_alu_peaks()
    mixed = prec == g.FMM_PREC_MIXED
    p32, sms, mhz = fp32_peak()
    pk, loop = (p32, loop32) if mixed else (FP64_PEAK_TFLOPS, loop64)
    src = (f"derived: {sms} SMs x 128 FP32 lanes x 2 flops x {mhz:.0f} MHz" if mixed
           else "nominal FP64 rate of the part (1.25 TFLOP/s)")
    if k_m2l >= k_p2p:
        rot = mixed and 3 <= a.p <= 16
        work = full["n_m2l"] * (m2l_rot_flops(a.p) if rot else m2l_flops(a.p))
        t_k, t_ph = k_m2l, t_m2l
        kern = ("k_m2l_rot (App. A.5 rotations and eq. A31, orders > 2 in FP32)" if rot
                else "k_m2l_rounds (eq. 3b, orders > 2 in FP32)" if mixed else "k_m2l (eq. 3b, FP64)")
    else:
        work = 20.0 * full["p2p_interactions"]
        t_k, t_ph = k_p2p, t_p2p
        kern = "k_p2p_mixed (eq. 1, FP32 two-float)" if mixed else "k_p2p_fp64 (eq. 1)"
    achieved = work / t_k / 1e12
    key = (a.workload, a.n, a.p, a.eps, a.leaf, a.c, a.precision)
    traffic = MEASURED_TRAFFIC.get(key, {}).get(kern.split(" ")[0])
    pair_ceiling = 20.0 * g.fmm_pair_peak(16) / 1e3 if mixed else None  # TFLOP/s, 20 flops per pair
    return {"kernel": kern, "bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
            "frac": achieved / pk, "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read+write)",
            "peak_source": src,
            "kernel_ms": 1e3 * t_k, "timing": "CUDA events around the kernel's launches, mean over the timed steps",
            "phase_ms": 1e3 * t_ph, "achieved_phase": work / t_ph / 1e12, "frac_phase": work / t_ph / 1e12 / pk,
            "peak_loop_measured": loop, "frac_of_loop": achieved / loop,
            "pair_arithmetic_ceiling": pair_ceiling,
            "pair_arithmetic_ceiling_note": "the P2P pair arithmetic alone (fmm_pair_peak, 16 warps per SM as "
                                            "the kernel): 13 FP32 operations and one rsqrt per pair, two sinks "
                                            "per lane, no staging or idle lanes",
            "kernel_share": {"m2l": k_m2l / (float(np.mean([s["t_total"] for s in phase])) * 1e-3),
                             "p2p": k_p2p / (float(np.mean([s["t_total"] for s in phase])) * 1e-3),
                             "note": "each main kernel's own CUDA-event time over the step's (the M2L and the "
                                     "P2P run side by side on two streams)"}}


def sampled_error(ctx, xt, mt, acc, idx, dev, G=1.0):
    """rms and 99.9th percentile of |a - a_direct| / |a_direct| over the sinks idx
    (FP64 direct sums over all sources on the GPU)."""
    import torch
    sinks = torch.from_numpy(np.asarray(idx, dtype=np.int64)).to(dev)
    _, acc_t = ctx.fmm_direct(xt, mt, G, sinks=sinks)
    e = (torch.linalg.norm(acc[sinks] - acc_t, dim=1) / torch.linalg.norm(acc_t, dim=1)).cpu().numpy()
    return e


def cpu_sample_line(a, model="plummer"):
    import oracle
    from paper_1405_2255_gb300 import inputs
    oracle.build()
    tcpu = oracle_run(a.cpu_sample, a.p, a.eps, a.leaf, a.c, inputs.BASE_SEED + 2, model)
    return {"value": a.cpu_sample / tcpu, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle FMM (serial C, FP64) on a {model} system of N={a.cpu_sample} of the same "
                      f"recipe and parameters, one evaluation ({tcpu:.1f} s)"}


def event_ms(fn, stream, warm=3, reps=10, flush=None):
    """Median CUDA-event time (ms, on stream) of fn() over reps runs after warm untimed runs;
    flush (a tensor larger than L2) is overwritten before every timed run."""
    import torch
    for _ in range(warm):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        if flush is not None:
            flush.zero_()
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return float(np.median([e0.elapsed_time(e1) for e0, e1 in ev]))


def ensemble_record(a, g, dev, local, rank, world, prec, steps, warmup, emit_line):
    """256 Plummer spheres of N log-uniform in [1e3, 1e5] with Kroupa-like masses,
    evaluated together as one forest per step (fmm_evaluate_batch)."""
    import torch
    from paper_1405_2255_gb300 import inputs
    p, eps, leaf, c = (a.p, a.eps, a.leaf, a.c) if a.workload == "ensemble" else PARAMS["ensemble"]
    systems = inputs.ensemble(256, inputs.BASE_SEED + 4 + 7919 * rank)
    sizes = np.array([len(m) for _, m in systems])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ntot = int(off[-1])
    xs = np.concatenate([s[0] for s in systems])
    ms = np.concatenate([s[1] for s in systems])
    xt, mt = torch.from_numpy(xs).to(dev), torch.from_numpy(ms).to(dev)
    psi = torch.empty(ntot, dtype=torch.float64, device=dev)
    acc = torch.empty((ntot, 3), dtype=torch.float64, device=dev)
    G = np.ones(len(systems))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = g.Context(p=p, eps=eps, leaf_size=leaf, p2p_c=c, precision=prec, device=local)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(warmup, 3)):
        ctx.fmm_evaluate_batch(off, xt, mt, G, psi=psi, acc=acc)
    torch.cuda.synchronize(dev)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    phase, launches = [], 0
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(steps):
            flush.zero_()
            ev0[k].record(stream)
            ctx.fmm_evaluate_batch(off, xt, mt, G, psi=psi, acc=acc)
            ev1[k].record(stream)
            st = ctx.fmm_last_stats()
            phase.append(st)
            launches += int(st["launches"])
        torch.cuda.synchronize(dev)
    ms_step = max_over_ranks(np.mean([e0.elapsed_time(e1) for e0, e1 in zip(ev0, ev1)]), world, dev)
    value = job_value(ntot, world, ms_step * 1e-3)
    _, _, full = ctx.fmm_evaluate_batch(off, xt, mt, G, psi=psi, acc=acc, stats=True)
    # accuracy: 16 sinks of every system against the FP64 direct sum over that system
    rng = np.random.default_rng(rank)
    errs = []
    for i in range(len(systems)):
        n = int(sizes[i])
        sl = slice(int(off[i]), int(off[i + 1]))
        idx = np.sort(rng.choice(n, min(n, 16), replace=False))
        errs.append(sampled_error(ctx, xt[sl], mt[sl], acc[sl], idx, dev))
    e = np.concatenate(errs)
    rec = {"workload": "ensemble256_plummer_kroupa", "value": value, "unit": UNIT, "ms_per_step": ms_step,
           "steps": steps, "systems": len(systems), "n_total": ntot,
           "n_range": [int(sizes.min()), int(sizes.max())], "p": p, "eps": eps, "leaf_size": leaf, "p2p_c": c,
           "rms_rel_err": float(np.sqrt(np.mean(e ** 2))), "p999_rel_err": float(np.percentile(e, 99.9)),
           "err_sinks": int(len(e)), "launches_per_step": launches / steps,
           "phase_ms": {k: float(np.mean([s_[k] for s_ in phase])) for k in
                        ("t_tree", "t_estimate", "t_up", "t_walk", "t_m2l", "t_p2p", "t_down", "t_total", "t_m2l_kernel", "t_p2p_kernel")}}
    if not emit_line:
        ctx.close()
        return rec
    roof = roofline(g, a, prec, phase, full)
    extras = {}
    if not a.no_extras and rank == 0:
        # the same systems one call each (no forest)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in range(len(systems)):
            sl = slice(int(off[i]), int(off[i + 1]))
            ctx.fmm_evaluate(xt[sl], mt[sl], 1.0, psi=psi[sl], acc=acc[sl])
        torch.cuda.synchronize(dev)
        extras["one_call_per_system_value"] = ntot / (time.perf_counter() - t0)
    # end to end: pinned host inputs in, the forest evaluation, results back to pinned host memory
    xh, mh = torch.from_numpy(xs).pin_memory(), torch.from_numpy(ms).pin_memory()
    ah = torch.empty((ntot, 3), dtype=torch.float64).pin_memory()
    ph = torch.empty(ntot, dtype=torch.float64).pin_memory()
    te = []
    for k in range(steps + 1):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        xt.copy_(xh, non_blocking=True)
        mt.copy_(mh, non_blocking=True)
        ctx.fmm_evaluate_batch(off, xt, mt, G, psi=psi, acc=acc)
        ph.copy_(psi, non_blocking=True)
        ah.copy_(acc, non_blocking=True)
        torch.cuda.synchronize(dev)
        if k:
            te.append(time.perf_counter() - t0)
    t_e2e = max_over_ranks(np.mean(te), world, dev)
    cpu = cpu_sample_line(a) if rank == 0 and world == 1 else None
    if rank == 0:
        cfg = {"workload": "ensemble256_plummer_kroupa", "systems": len(systems), "n_total": ntot,
               "n_range": rec["n_range"],
               "model": "256 truncated Plummer spheres, N log-uniform in [1e3, 1e5], Kroupa-like masses",
               "p": p, "eps": eps, "mac": "18a (low-order a estimate)", "leaf_size": leaf, "p2p_c": c,
               "precision": a.precision, "l2": "flushed between steps (256 MiB write)",
               "parallelism": "one forest per call; replicas across GPUs",
               "rms_rel_err": rec["rms_rel_err"], "p999_rel_err": rec["p999_rel_err"],
               "err_sinks": rec["err_sinks"], "phase_ms": rec["phase_ms"]}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
                "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64" if prec == g.FMM_PREC_MIXED else "f64",
                "data": "synthetic", "config": cfg,
                "e2e": {"value": job_value(ntot, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": 32 * ntot,
                        "d2h_bytes_per_step": 32 * ntot},
                "roofline": roof, "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clk.summary()}
        line.update(extras)
        print(json.dumps(line), flush=True)
    ctx.close()
    return rec


def run_ensemble(a, g, dev, local, rank, world, prec):
    ensemble_record(a, g, dev, local, rank, world, prec, a.steps, a.warmup, True)


def serve_record(a, g, dev, local, rank, world, prec, nreq, warmup, cap_rounds):
    """64 concurrent simulations (half Plummer, half gamma = 1.5 cusps, N log-uniform in
    [1e4, 2e6]) served by the request loop.  Capacity is measured closed-loop (all
    systems submitted at once); then requests arrive as a Poisson process at 0.8 of
    that capacity, each system taking the next request once its previous result is
    back, and latency is counted from arrival to completion.  Returns the record and
    the clock summary."""
    import torch
    from paper_1405_2255_gb300 import inputs
    p, eps, leaf, c = (a.p, a.eps, a.leaf, a.c) if a.workload == "serve" else PARAMS["serve"]
    systems = inputs.served_systems(64, inputs.BASE_SEED + 5 + 7919 * rank)
    sizes = np.array([len(m) for _, m in systems])
    dx = [torch.from_numpy(x).to(dev) for x, _ in systems]
    dm = [torch.from_numpy(m).to(dev) for _, m in systems]
    del systems
    dp = [torch.empty(n, dtype=torch.float64, device=dev) for n in sizes]
    da = [torch.empty((n, 3), dtype=torch.float64, device=dev) for n in sizes]
    ctx = g.Context(p=p, eps=eps, leaf_size=leaf, p2p_c=c, precision=prec, device=local)
    slots = getattr(a, "slots", 2)
    ctx.fmm_serve_config(0, slots)
    ids = [ctx.fmm_system_register(int(n)) for n in sizes]
    torch.cuda.synchronize(dev)

    def closed_loop():
        t0 = time.perf_counter()
        tks = [ctx.fmm_submit(i, dx[k], dm[k], 1.0, dp[k], da[k]) for k, i in enumerate(ids)]
        for t in tks:
            ctx.fmm_poll(t, -1)
        return time.perf_counter() - t0

    for _ in range(max(warmup, 3)):
        closed_loop()
    caps = [closed_loop() for _ in range(max(cap_rounds, 1))]
    t_cap = float(np.median(caps))
    capacity = float(sizes.sum()) / t_cap
    # open loop: aggregate Poisson arrivals at 0.8 capacity, systems in turn
    rate = 0.8 * capacity / float(sizes.mean())
    arrivals = inputs.poisson_arrivals(nreq, rate, inputs.BASE_SEED + 5 + 31 * rank)
    order = np.arange(nreq) % len(sizes)
    backlog = [[] for _ in sizes]
    inflight = {}
    lat, done_n = [], 0
    nxt = 0
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        while nxt < nreq or inflight or any(backlog):
            now = time.perf_counter() - t0
            while nxt < nreq and arrivals[nxt] <= now:
                k = int(order[nxt])
                backlog[k].append(arrivals[nxt])
                nxt += 1
            for k in range(len(sizes)):
                if backlog[k] and k not in inflight:
                    t_arr = backlog[k].pop(0)
                    ts = time.perf_counter() - t0
                    inflight[k] = (ctx.fmm_submit(ids[k], dx[k], dm[k], 1.0, dp[k], da[k]), t_arr, ts)
            for k in list(inflight):
                tk, t_arr, ts = inflight[k]
                l = ctx.fmm_poll(tk, 0)
                if l is not None:
                    lat.append(ts + l - t_arr)
                    done_n += int(sizes[k])
                    del inflight[k]
            time.sleep(2e-4)
        elapsed = time.perf_counter() - t0
    lat_ms = 1e3 * np.array(lat)
    ctx.close()
    # the results of the last requests against each system alone, and their accuracy
    alone = g.Context(p=p, eps=eps, leaf_size=leaf, p2p_c=c, precision=prec, device=local)
    same = 0
    errs = []
    rng = np.random.default_rng(rank)
    for k in range(len(sizes)):
        p1, a1 = alone.fmm_evaluate(dx[k], dm[k], 1.0)
        same += int(torch.equal(a1, da[k]) and torch.equal(p1, dp[k]))
        idx = np.sort(rng.choice(int(sizes[k]), 64, replace=False))
        if k % 2 == 1:
            idx[0] = 0  # the cusps' central point mass
        errs.append(sampled_error(alone, dx[k], dm[k], da[k], np.unique(idx), dev))
    e = np.concatenate(errs)
    alone.close()
    value = sum_over_ranks(done_n, world, dev) / max_over_ranks(elapsed, world, dev)
    rec = {"workload": "serve64_plummer_cusp", "value": value, "unit": UNIT, "systems": len(sizes),
           "n_total": int(sizes.sum()), "n_range": [int(sizes.min()), int(sizes.max())], "p": p, "eps": eps,
           "leaf_size": leaf, "p2p_c": c, "slots": slots, "requests": nreq, "load": 0.8,
           "capacity_pf_s": capacity, "closed_loop_ms": 1e3 * t_cap,
           "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                          "mean": float(lat_ms.mean()), "max": float(lat_ms.max())},
           "results_equal_alone": f"{same}/{len(sizes)}",
           "rms_rel_err": float(np.sqrt(np.mean(e ** 2))), "p999_rel_err": float(np.percentile(e, 99.9)),
           "err_sinks": int(len(e))}
    return rec, clk.summary()


def run_serve(a, g, dev, local, rank, world, prec):
    rec, clocks = serve_record(a, g, dev, local, rank, world, prec, a.requests, a.warmup, a.steps)
    cpu = cpu_sample_line(a) if rank == 0 and world == 1 else None
    if rank == 0:
        cfg = dict(rec)
        cfg.update({"model": "32 truncated Plummer spheres + 32 gamma=1.5 cusps with 1% central point mass, "
                             "N log-uniform in [1e4, 2e6]", "mac": "18a (low-order a estimate)",
                    "precision": a.precision, "l2": "inputs larger than L2 (19M particles resident)",
                    "parallelism": f"{rec['slots']} slots with continuous batching; replicas across GPUs"})
        for k in ("value", "unit"):
            cfg.pop(k)
        line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": a.requests,
                "warmup": a.warmup, "ms_per_step": rec["latency_ms"]["mean"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if prec == g.FMM_PREC_MIXED else "f64", "data": "synthetic", "config": cfg,
                "e2e": None, "roofline": None, "cpu_baseline": cpu, "gpu_launches": None, "clocks": clocks}
        print(json.dumps(line), flush=True)


def run_active(a, g, dev, local, rank, world, prec):
    """Sec. 7.1: forces for the innermost N_a particles of a Plummer sphere of N (the
    paper's Fig. 14 experiment), N_a = N/10^k; all N particles are sources.  The headline
    value is active particle-forces/s at N_a = N/100; the sweep gives ms per step for
    every N_a (tree and upward pass over all N, walk and interactions for the active part)."""
    import torch
    from paper_1405_2255_gb300 import inputs
    x, mu = inputs.plummer(a.n, inputs.BASE_SEED + 2 + 7919 * rank)
    xt, mt = torch.from_numpy(x).to(dev), torch.from_numpy(mu).to(dev)
    order = np.argsort(np.linalg.norm(x, axis=1), kind="stable")
    psi = torch.empty(a.n, dtype=torch.float64, device=dev)
    acc = torch.empty((a.n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = g.Context(p=a.p, eps=a.eps, leaf_size=a.leaf, p2p_c=a.c, precision=prec, device=local)
    stream = torch.cuda.current_stream(dev)
    sweep, head = {}, None
    na_list = sorted({int(a.n // 10 ** k) for k in range(0, 5)} | {1000})
    rng = np.random.default_rng(rank)
    for na in na_list:
        act = np.zeros(a.n, dtype=np.uint8)
        act[order[:na]] = 1
        at = torch.from_numpy(act).to(dev)
        for _ in range(max(a.warmup, 3)):
            ctx.fmm_evaluate_active(xt, mt, at, psi=psi, acc=acc)
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        phase, launches = [], 0
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(local) as clk:
            for e0, e1 in ev:
                flush.zero_()
                e0.record(stream)
                ctx.fmm_evaluate_active(xt, mt, at, psi=psi, acc=acc)
                e1.record(stream)
                st = ctx.fmm_last_stats()
                phase.append(st)
                launches += int(st["launches"])
            torch.cuda.synchronize(dev)
        ms = max_over_ranks(np.mean([e0.elapsed_time(e1) for e0, e1 in ev]), world, dev)
        # the same step on the re-cycled tree of the previous step (Sec. 7.1's other measure;
        # unchanged positions here, so this times the refresh of radii, masses and centres of mass)
        ev_r = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        phase_r = []
        for e0, e1 in ev_r:
            flush.zero_()
            e0.record(stream)
            ctx.fmm_evaluate_active(xt, mt, at, psi=psi, acc=acc, reuse_tree=True)
            e1.record(stream)
            phase_r.append(ctx.fmm_last_stats())
        torch.cuda.synchronize(dev)
        ms_r = max_over_ranks(np.mean([e0.elapsed_time(e1) for e0, e1 in ev_r]), world, dev)
        idx = np.sort(rng.choice(order[:na], min(na, 2048), replace=False))
        e = sampled_error(ctx, xt, mt, acc, idx, dev)
        sweep[na] = {"ms": ms, "rms_rel_err": float(np.sqrt(np.mean(e ** 2))),
                     "phase_ms": {k: float(np.mean([s_[k] for s_ in phase])) for k in
                                  ("t_tree", "t_estimate", "t_up", "t_walk", "t_m2l", "t_p2p", "t_down", "t_total", "t_m2l_kernel", "t_p2p_kernel")},
                     "n_m2l": int(phase[-1]["n_m2l"]), "n_p2p": int(phase[-1]["n_p2p"]),
                     "reused_tree_ms": ms_r, "reused_tree_t_tree": float(np.mean([s_["t_tree"] for s_ in phase_r]))}
        if na == a.n // 100:
            head = (ms, launches / a.steps, clk.summary(), st)
    ms, launches, clocks, st = head
    na = a.n // 100
    value = job_value(na, world, ms * 1e-3)
    if rank == 0:
        cfg = {"workload": f"active_innermost_n{a.n}", "n": a.n, "n_active": na,
               "model": "truncated Plummer sphere R_t=30, equal masses; the innermost N_a particles active",
               "p": a.p, "eps": a.eps, "mac": "18a (low-order a estimate over the active sinks)",
               "leaf_size": a.leaf, "p2p_c": a.c, "precision": a.precision,
               "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas",
               "rms_rel_err": sweep[na]["rms_rel_err"], "err_sinks": min(na, 2048),
               "phase_ms": sweep[na]["phase_ms"], "sweep_by_n_active": {str(k): v for k, v in sweep.items()}}
        line = {"metric": "active particle-forces/s (Sec. 7.1 subset evaluation)", "value": value, "unit": UNIT,
                "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if prec == g.FMM_PREC_MIXED else "f64", "data": "synthetic", "config": cfg,
                "e2e": None, "roofline": None, "cpu_baseline": None, "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    ctx.close()


def config_of(a):
    if a.workload == "cusp":
        return {"workload": f"cusp_n{a.n}", "n": a.n,
                "model": "Dehnen gamma=1.5 truncated at 30 scale radii, equal masses, 1% central point mass",
                "p": a.p, "eps": a.eps, "mac": "18a (low-order a estimate)", "leaf_size": a.leaf, "p2p_c": a.c,
                "precision": a.precision, "l2": "inputs larger than L2 (320 MB of positions)",
                "parallelism": "replicas"}
    return {"workload": f"plummer_n{a.n}", "n": a.n, "model": "truncated Plummer sphere R_t=30, equal masses",
            "p": a.p, "eps": a.eps, "mac": "18a (low-order a estimate)", "leaf_size": a.leaf, "p2p_c": a.c,
            "precision": a.precision, "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas"}


# (p, eps, leaf, p2p_c) of the plain all-FP64 GPU FMM (precision = FP64) at rms 1e-7 on the
# default workload: its own autotuner optimum over p 10..16, leaf 32..128, p2p_c 1..4 (truth on
# 10^5 sampled sinks; eps with a margin)
FP64_PARAMS = (16, 3.3e-7, 96, 1.0)


def cusp_record(a, g, dev, local, rank, prec, steps, warmup):
    """gamma = 1.5 Dehnen cusp of 1e7 particles with a 1 % central point mass."""
    import torch
    from paper_1405_2255_gb300 import inputs
    p, eps, leaf, c = PARAMS["cusp"]
    n = 10_000_000
    x, mu = inputs.dehnen(n, inputs.BASE_SEED + 3 + 7919 * rank)
    xt, mt = torch.from_numpy(x).to(dev), torch.from_numpy(mu).to(dev)
    del x, mu
    psi = torch.empty(n, dtype=torch.float64, device=dev)
    acc = torch.empty((n, 3), dtype=torch.float64, device=dev)
    ctx = g.Context(p=p, eps=eps, leaf_size=leaf, p2p_c=c, precision=prec, device=local)
    stream = torch.cuda.current_stream(dev)
    ms = event_ms(lambda: ctx.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc), stream, max(warmup, 3), steps)
    rng = np.random.default_rng(rank)
    pick = rng.choice(n, 10000, replace=False)
    pick[0] = 0  # the central point mass
    e = sampled_error(ctx, xt, mt, acc, np.unique(pick), dev)
    ctx.close()
    return {"workload": f"cusp_n{n}", "value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "timing": f"median of {steps} after {max(warmup, 3)} warm-up (inputs larger than L2)",
            "p": p, "eps": eps, "leaf_size": leaf, "p2p_c": c,
            "rms_rel_err": float(np.sqrt(np.mean(e ** 2))), "p999_rel_err": float(np.percentile(e, 99.9)),
            "err_sinks": int(len(e))}


def crossover(g, dev, local, prec, flush):
    """Sec. 6.4's comparison with direct summation: the mixed FMM against the GPU FP64 direct
    sum for N = 1e4 .. 1e6 (Plummer spheres of the default generator).  At every N the FMM's
    eps is set by the autotuner's secant steps so that the rms relative error is at most 1e-7
    over all sinks up to N = 1e5 and over 32768 sampled sinks above (p = 14, p2p_c = 1; leaf 48
    below N = 3e5, 80 from there on); the direct sum runs over the same sinks (its time scaled
    to N sinks)."""
    import torch
    from paper_1405_2255_gb300 import autotune, inputs
    stream = torch.cuda.current_stream(dev)
    rows = []
    for n in (10_000, 30_000, 100_000, 300_000, 1_000_000):
        x, mu = inputs.plummer(n, inputs.BASE_SEED + 2)
        xt, mt = torch.from_numpy(x).to(dev), torch.from_numpy(mu).to(dev)
        p, eps, leaf, c = PARAMS["ensemble"] if n < 300_000 else PARAMS["plummer"]
        # the tuner's truth sample (all sinks up to N = 1e5, else 32768 drawn with seed 0) is also
        # the sample the row's rms is checked on
        ntr = n if n <= 100_000 else 32768
        tr = autotune.tune(xt, mt, target_rms=1e-7, ps=(p,), leaves=(leaf,), cs=(c,), nsinks=ntr,
                           precision=prec, eps0=eps, margin=0.95)
        eps = tr.best.eps
        ctx = g.Context(p=p, eps=eps, leaf_size=leaf, p2p_c=c, precision=prec, device=local)
        psi = torch.empty(n, dtype=torch.float64, device=dev)
        acc = torch.empty((n, 3), dtype=torch.float64, device=dev)
        ms = event_ms(lambda: ctx.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc), stream, 3, 5, flush)
        ns = ntr
        sinks = None if ns == n else torch.from_numpy(
            np.sort(np.random.default_rng(0).choice(n, ns, replace=False)).astype(np.int64)).to(dev)
        ms_d = event_ms(lambda: ctx.fmm_direct(xt, mt, 1.0, sinks=sinks), stream, 1, 3)
        _, acc_t = ctx.fmm_direct(xt, mt, 1.0, sinks=sinks)
        idx = torch.arange(n, device=dev) if sinks is None else sinks
        e = (torch.linalg.norm(acc[idx] - acc_t, dim=1) / torch.linalg.norm(acc_t, dim=1)).cpu().numpy()
        fmm_v, dir_v = n / (ms * 1e-3), ns / (ms_d * 1e-3)
        rows.append({"n": n, "fmm_value": fmm_v, "fmm_ms": ms, "direct_value": dir_v,
                     "direct_ms_scaled": ms_d * n / ns, "direct_sinks": ns, "fmm_over_direct": fmm_v / dir_v,
                     "fmm_rms_rel_err": float(np.sqrt(np.mean(e ** 2))), "p": p, "eps": eps, "leaf_size": leaf})
        ctx.close()
        del xt, mt, psi, acc, acc_t
    # the smallest N of the sweep from which on the FMM beats direct summation at every larger N
    cross = None
    for r in reversed(rows):
        if r["fmm_over_direct"] > 1.0:
            cross = r["n"]
        else:
            break
    return {"rows": rows, "fmm_faster_from_n": cross,
            "timing": "CUDA events; FMM median of 5 after 3 warm-ups (L2 flushed), direct median of 3 after 1"}


def main():
    a = parse()
    rank, world, local = dist_env()
    if a.impl == "reference":
        return reference_arm(a, rank, world)
    import torch
    from paper_1405_2255_gb300 import gb3fmm as g
    from paper_1405_2255_gb300 import inputs
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    g.load()
    prec = g.FMM_PREC_MIXED if a.precision == "mixed" else g.FMM_PREC_FP64
    if a.workload == "ensemble":
        return run_ensemble(a, g, dev, local, rank, world, prec)
    if a.workload == "serve":
        return run_serve(a, g, dev, local, rank, world, prec)
    if a.workload == "active":
        return run_active(a, g, dev, local, rank, world, prec)
    if a.workload == "cusp":
        x, mu = inputs.dehnen(a.n, inputs.BASE_SEED + 3 + 7919 * rank)
    else:
        x, mu = inputs.plummer(a.n, inputs.BASE_SEED + 2 + 7919 * rank)
    xt = torch.from_numpy(x).to(dev)
    mt = torch.from_numpy(mu).to(dev)
    tuned = None
    if a.autotune:
        from paper_1405_2255_gb300 import autotune
        r = autotune.tune(xt, mt, target_rms=1e-7, precision=prec)
        a.p, a.eps, a.leaf, a.c = r.best.p, r.best.eps, r.best.leaf_size, r.best.p2p_c
        tuned = {"seconds": r.seconds, "candidates": len(r.tried), "target_rms": r.target_rms,
                 "tuning_rms": r.best.rms, "tuning_ms": r.best.ms}
    psi = torch.empty(a.n, dtype=torch.float64, device=dev)
    acc = torch.empty((a.n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = g.Context(p=a.p, eps=a.eps, leaf_size=a.leaf, p2p_c=a.c, precision=prec, device=local)
    stream = torch.cuda.current_stream(dev)

    for _ in range(max(a.warmup, 3)):
        ctx.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc)
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    phase = []
    launches = 0
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(a.steps):
            flush.zero_()
            ev0[k].record(stream)
            ctx.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc)
            ev1[k].record(stream)
            st = ctx.fmm_last_stats()
            phase.append(st)
            launches += int(st["launches"])
        torch.cuda.synchronize(dev)
    barrier()
    ms = max_over_ranks(np.mean([e0.elapsed_time(e1) for e0, e1 in zip(ev0, ev1)]), world, dev)
    value = job_value(a.n, world, ms * 1e-3)

    # accuracy of the timed configuration: GPU FP64 direct sum over all sources for a seeded
    # sample of 10^5 sinks (fewer when N is smaller)
    rng = np.random.default_rng(rank)
    ns = min(a.n, 100_000)
    pick = rng.choice(a.n, ns, replace=False)
    if a.workload == "cusp":
        pick[0] = 0  # the central point mass is always in the sample
    sinks = torch.from_numpy(np.sort(np.unique(pick)).astype(np.int64)).to(dev)
    ns = int(sinks.numel())
    _, acc_t = ctx.fmm_direct(xt, mt, 1.0, sinks=sinks)

    def errors(acc_):
        return (torch.linalg.norm(acc_[sinks] - acc_t, dim=1) / torch.linalg.norm(acc_t, dim=1)).cpu().numpy()

    e = errors(acc)
    rms, p999 = float(np.sqrt(np.mean(e ** 2))), float(np.percentile(e, 99.9))

    # roofline of the dominant kernel (phase times averaged over the timed steps)
    _, _, full = ctx.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc, stats=True)
    roof = roofline(g, a, prec, phase, full)

    extras = {}
    if not a.no_extras and rank == 0:
        base = {}
        # (i) the plain all-FP64 GPU FMM at its own tuned parameters, and at the mixed mode's
        p64, eps64, leaf64, c64_ = FP64_PARAMS
        c64 = g.Context(p=p64, eps=eps64, leaf_size=leaf64, p2p_c=c64_, precision=g.FMM_PREC_FP64, device=local)
        ms64 = event_ms(lambda: c64.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc), stream, 3, 10, flush)
        e64 = errors(acc)
        c64.set_params(p=a.p, eps=a.eps, leaf_size=a.leaf, p2p_c=a.c)
        ms64m = event_ms(lambda: c64.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc), stream, 1, 3, flush)
        c64.close()
        base["fp64_fmm"] = {"value": a.n / (ms64 * 1e-3), "ms": ms64, "p": p64, "eps": eps64,
                            "leaf_size": leaf64, "p2p_c": c64_, "rms_rel_err": float(np.sqrt(np.mean(e64 ** 2))),
                            "p999_rel_err": float(np.percentile(e64, 99.9)),
                            "params_source": "autotuner with precision = FP64 at rms 1e-7 on this workload",
                            "timing": "CUDA events, median of 10 after 3 warm-ups, L2 flushed",
                            "at_mixed_params_ms": ms64m, "mixed_over_fp64": value / (a.n / (ms64 * 1e-3))}
        # (ii) mixed mode with FP64 expansions (m2l_split = 0: FP32 only in P2P and the estimate),
        # at the FP64 parameters and at the default ones
        lit = g.Context(p=p64, eps=eps64, leaf_size=leaf64, p2p_c=c64_, precision=prec, m2l_split=0,
                        device=local)
        ms_l = event_ms(lambda: lit.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc), stream, 3, 5, flush)
        e_l = errors(acc)
        lit.set_params(p=a.p, eps=a.eps, leaf_size=a.leaf, p2p_c=a.c)
        ms_l2 = event_ms(lambda: lit.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc), stream, 1, 3, flush)
        e_l2 = errors(acc)
        lit.close()
        base["mixed_fp64_expansions"] = {
            "what": "P2P and the scale estimate in FP32, P2M/M2M/M2L/L2L/L2P all in FP64 (m2l_split = 0)",
            "value": a.n / (ms_l * 1e-3), "ms": ms_l, "p": p64, "eps": eps64, "leaf_size": leaf64,
            "p2p_c": c64_, "rms_rel_err": float(np.sqrt(np.mean(e_l ** 2))),
            "at_default_params": {"value": a.n / (ms_l2 * 1e-3), "ms": ms_l2,
                                  "rms_rel_err": float(np.sqrt(np.mean(e_l2 ** 2)))}}
        # (iii) GPU FP64 direct summation: 32768 sampled sinks (enough blocks for every SM), all
        # sources, no f, scaled to N sinks
        nd = min(a.n, 32768)
        dsinks = sinks[torch.randperm(ns, generator=torch.Generator().manual_seed(1))[:nd].to(dev)]
        ms_d = event_ms(lambda: ctx.fmm_direct(xt, mt, 1.0, sinks=dsinks), stream, 1, 3)
        pairs = float(nd) * a.n
        base["fp64_direct"] = {"value": nd / (ms_d * 1e-3), "sinks_timed": nd, "ms_sinks_timed": ms_d,
                               "ms_scaled_to_n": ms_d * a.n / nd, "pairs_per_s": pairs / (ms_d * 1e-3),
                               "fp64_tflops_at_20_per_pair": 20 * pairs / (ms_d * 1e-3) / 1e12,
                               "timing": "CUDA events, median of 3 after 1 warm-up"}
        base["mixed_over_direct"] = value / base["fp64_direct"]["value"]
        if a.workload == "plummer" and a.n == 1_000_000:
            base["crossover"] = crossover(g, dev, local, prec, flush)
        extras["baselines"] = base
        extras["fp64_fmm_value"] = base["fp64_fmm"]["value"]
        extras["fp64_direct_value"] = base["fp64_direct"]["value"]
        # the swap stage of the rotated M2L (App. A.5.1) on the tensor cores against the FMA
        # immediates the M2L kernel uses (a dense small-matrix contraction of the M2L)
        extras["m2l_swap_probe"] = g.fmm_swap_probe(1 << 20, 16)
        # the same step with the tidal tensor (Sec. 7.4) as an extra output
        Tt = torch.empty((a.n, 6), dtype=torch.float64, device=dev)
        extras["with_tidal_ms"] = event_ms(lambda: ctx.fmm_evaluate_active(xt, mt, psi=psi, acc=acc, tidal=Tt),
                                           stream, 1, 3, flush)
        del Tt
        ctx.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc)
    if not a.no_configs and world == 1 and a.workload == "plummer":
        # the other workloads as compact sub-records (each with its own parameters)
        cfgs = {}
        for name, fn in (("cusp", lambda: cusp_record(a, g, dev, local, rank, prec, 5, 3)),
                         ("ensemble", lambda: ensemble_record(a, g, dev, local, rank, world, prec, 10, 3, False)),
                         ("serve", lambda: serve_record(a, g, dev, local, rank, world, prec, 192, 3, 3)[0])):
            try:
                cfgs[name] = fn()
            except Exception as ex:  # a failing sub-record must not hide the headline
                cfgs[name] = {"error": f"{type(ex).__name__}: {ex}"}
            torch.cuda.empty_cache()
        extras["configs"] = cfgs
        if "latency_ms" in cfgs.get("serve", {}):
            extras["p50_latency_ms"] = cfgs["serve"]["latency_ms"]["p50"]
            extras["p99_latency_ms"] = cfgs["serve"]["latency_ms"]["p99"]

    # end to end through the host-buffer entry point (pinned host memory, copies inside)
    xh = torch.from_numpy(x).pin_memory().numpy()
    mh = torch.from_numpy(mu).pin_memory().numpy()
    ph = torch.empty(a.n, dtype=torch.float64).pin_memory().numpy()
    ah = torch.empty((a.n, 3), dtype=torch.float64).pin_memory().numpy()
    ctx.fmm_evaluate_host(xh, mh, 1.0, psi=ph, acc=ah, stream=stream)
    te = []
    for _ in range(a.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.fmm_evaluate_host(xh, mh, 1.0, psi=ph, acc=ah, stream=stream)
        te.append(time.perf_counter() - t0)
    t_e2e = max_over_ranks(np.mean(te), world, dev)

    cpu = cpu_sample_line(a, "cusp" if a.workload == "cusp" else "plummer") if rank == 0 and world == 1 else None

    if rank == 0:
        cfg = config_of(a)
        if tuned:
            cfg["autotune"] = tuned
        cfg.update({"rms_rel_err": rms, "p999_rel_err": p999, "err_sinks": int(ns),
                    "err_truth": "GPU FP64 direct sum over all sources for a seeded sample of sinks",
                    "phase_ms": {k: float(np.mean([s[k] for s in phase])) for k in
                                 ("t_tree", "t_estimate", "t_up", "t_walk", "t_m2l", "t_p2p", "t_down", "t_total", "t_m2l_kernel", "t_p2p_kernel")},
                    "n_m2l": int(full["n_m2l"]), "n_p2p": int(full["n_p2p"]),
                    "p2p_interactions": int(full["p2p_interactions"]), "ncells": int(full["ncells"])})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == g.FMM_PREC_MIXED else "f64", "data": "synthetic",
            "config": cfg,
            "e2e": {"value": job_value(a.n, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": 32 * a.n,
                    "d2h_bytes_per_step": 32 * a.n},
            "roofline": roof, "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clk.summary(),
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
