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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--p", type=int, default=12)
    ap.add_argument("--eps", type=float, default=2e-7)
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--c", type=float, default=4.0)
    ap.add_argument("--cpu-sample", type=int, default=50000)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64-mode and direct-sum comparisons")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ALU peaks derived from the unit counts and the maximum SM clock: 152 SMs x 128 FP32
# lanes x 2 flops (FFMA) x 2070 MHz; FP64 is the part's nominal 1.25 TFLOP/s
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = 1.25


def max_over_ranks(v, world, device=None):
    """Maximum of a per-rank float over all ranks (the slowest rank sets the job time)."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
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


def oracle_run(n, p, eps, leaf, c, seed):
    import oracle
    from paper_1405_2255_gb300 import inputs
    x, mu = inputs.plummer(n, seed)
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


def config_of(a):
    return {"workload": f"plummer_n{a.n}", "n": a.n, "model": "truncated Plummer sphere R_t=30, equal masses",
            "p": a.p, "eps": a.eps, "mac": "18a (low-order a estimate)", "leaf_size": a.leaf, "p2p_c": a.c,
            "precision": a.precision, "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas"}


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
    x, mu = inputs.plummer(a.n, inputs.BASE_SEED + 2 + 7919 * rank)
    xt = torch.from_numpy(x).to(dev)
    mt = torch.from_numpy(mu).to(dev)
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

    # accuracy of the timed configuration: GPU FP64 direct sum on sampled sinks
    rng = np.random.default_rng(rank)
    ns = min(a.n, 4096)
    sinks = torch.from_numpy(np.sort(rng.choice(a.n, ns, replace=False)).astype(np.int64)).to(dev)
    torch.cuda.synchronize(dev)
    td0 = time.perf_counter()
    _, acc_t = ctx.fmm_direct(xt, mt, 1.0, sinks=sinks)
    torch.cuda.synchronize(dev)
    t_direct = time.perf_counter() - td0
    e = (torch.linalg.norm(acc[sinks] - acc_t, dim=1) / torch.linalg.norm(acc_t, dim=1)).cpu().numpy()
    rms, p999 = float(np.sqrt(np.mean(e ** 2))), float(np.percentile(e, 99.9))

    # roofline of the dominant kernel (phase times averaged over the timed steps)
    _, _, full = ctx.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc, stats=True)
    t_m2l = float(np.mean([s["t_m2l"] for s in phase])) * 1e-3
    t_p2p = float(np.mean([s["t_p2p"] for s in phase])) * 1e-3
    loop64, loop32 = g.fmm_alu_peaks()
    mixed = prec == g.FMM_PREC_MIXED
    pk, loop = (FP32_PEAK_TFLOPS, loop32) if mixed else (FP64_PEAK_TFLOPS, loop64)
    src = ("derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz" if mixed
           else "nominal FP64 rate of the part (1.25 TFLOP/s)")
    if t_m2l >= t_p2p:
        achieved = full["n_m2l"] * m2l_flops(a.p) / t_m2l / 1e12
        kern = "k_m2l_split (eq. 3b, orders > 2 in FP32)" if mixed else "k_m2l (eq. 3b, FP64)"
    else:
        achieved = 20.0 * full["p2p_interactions"] / t_p2p / 1e12
        kern = "k_p2p_mixed (eq. 1, FP32 two-float)" if mixed else "k_p2p_fp64 (eq. 1)"
    roof = {"kernel": kern, "bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
            "frac": achieved / pk, "traffic": None, "peak_source": src,
            "peak_loop_measured": loop, "frac_of_loop": achieved / loop}

    extras = {}
    if not a.no_extras and rank == 0:
        # the plain all-FP64 GPU FMM on the same input and parameters
        c64 = g.Context(p=a.p, eps=a.eps, leaf_size=a.leaf, p2p_c=a.c, precision=g.FMM_PREC_FP64, device=local)
        c64.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        c64.fmm_evaluate(xt, mt, 1.0, psi=psi, acc=acc)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        extras["fp64_fmm_value"] = a.n / (e0.elapsed_time(e1) * 1e-3)
        c64.close()
        # GPU FP64 direct summation, timed on the sampled sinks and scaled to N sinks
        extras["fp64_direct_value"] = a.n / (t_direct * a.n / ns)
        extras["direct_sample_sinks"] = ns

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

    cpu = None
    if rank == 0 and world == 1:
        import oracle
        oracle.build()
        tcpu = oracle_run(a.cpu_sample, a.p, a.eps, a.leaf, a.c, inputs.BASE_SEED + 2)
        cpu = {"value": a.cpu_sample / tcpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle FMM (serial C, FP64) on a Plummer sphere of N={a.cpu_sample} of the same "
                         f"recipe and parameters, one evaluation ({tcpu:.1f} s)"}

    if rank == 0:
        cfg = config_of(a)
        cfg.update({"rms_rel_err": rms, "p999_rel_err": p999, "err_sinks": int(ns),
                    "phase_ms": {k: float(np.mean([s[k] for s in phase])) for k in
                                 ("t_tree", "t_estimate", "t_up", "t_walk", "t_m2l", "t_p2p", "t_down", "t_total")},
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
