"""Choice of (p, eps, leaf size, P2P threshold) for a target rms relative force error.

For a given input on the device the tuner measures, for every candidate (p, leaf,
p2p_c), the accuracy parameter eps at which the rms relative acceleration error
over a seeded sample of sinks reaches the target (the error grows about linearly
with eps under the criteria of eqs. 18a,b, so a secant step in log eps converges
in a few evaluations), then times the evaluation at that eps and keeps the fastest
candidate.  The truth is the FP64 direct sum over all sources for the sampled
sinks (fmm_direct), computed once.  Everything runs through the library's C ABI;
this module only drives it.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Candidate:
    p: int
    leaf_size: int
    p2p_c: float
    eps: float = float("nan")
    rms: float = float("nan")
    p999: float = float("nan")
    ms: float = float("inf")
    evaluations: int = 0


@dataclass
class TuneResult:
    best: Candidate
    tried: list = field(default_factory=list)
    target_rms: float = 1e-7
    sinks: int = 0
    seconds: float = 0.0

    def params(self) -> dict:
        b = self.best
        return {"p": b.p, "eps": b.eps, "leaf_size": b.leaf_size, "p2p_c": b.p2p_c}


def _errors(acc, acc_true, sinks):
    import torch
    d = torch.linalg.norm(acc[sinks] - acc_true, dim=1) / torch.linalg.norm(acc_true, dim=1)
    return d.cpu().numpy()


def _time_ms(ctx, x, mu, psi, acc, reps=3):
    import torch
    s = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    ctx.fmm_evaluate(x, mu, 1.0, psi=psi, acc=acc)
    for e0, e1 in ev:
        e0.record(s)
        ctx.fmm_evaluate(x, mu, 1.0, psi=psi, acc=acc)
        e1.record(s)
    torch.cuda.synchronize()
    return float(np.median([e0.elapsed_time(e1) for e0, e1 in ev]))


def tune(x, mu, target_rms=1e-7, ps=(8, 10, 12, 14, 16), leaves=(32, 48, 64, 96), cs=(1.0, 2.0, 4.0, 8.0),
         nsinks=4096, seed=0, precision=None, eps0=2e-7, max_steps=4, margin=0.97, log=None,
         fixed=None) -> TuneResult:
    """x [n,3], mu [n]: float64 CUDA tensors.  Returns the fastest candidate whose
    measured rms relative error is at most target_rms.  fixed: further fmm_params fields
    held for every candidate (e.g. {"adaptive_p": 1})."""
    import torch
    from . import gb3fmm as g
    t0 = time.perf_counter()
    n = int(mu.shape[0])
    prec = g.FMM_PREC_MIXED if precision is None else precision
    rng = np.random.default_rng(seed)
    sinks = torch.from_numpy(np.sort(rng.choice(n, min(n, nsinks), replace=False)).astype(np.int64)).to(x.device)
    ref = g.Context(device=x.device.index or 0)
    _, acc_true = ref.fmm_direct(x, mu, 1.0, sinks=sinks)
    ref.close()
    psi = torch.empty(n, dtype=torch.float64, device=x.device)
    acc = torch.empty((n, 3), dtype=torch.float64, device=x.device)
    tried = []
    best = None
    for p in ps:
        for leaf in leaves:
            for c in cs:
                cand = Candidate(p, leaf, c)
                ctx = g.Context(p=p, eps=eps0, leaf_size=leaf, p2p_c=c, precision=prec,
                                device=x.device.index or 0, **(fixed or {}))
                eps, hist = eps0, []
                for _ in range(max_steps):
                    ctx.set_params(eps=eps)
                    ctx.fmm_evaluate(x, mu, 1.0, psi=psi, acc=acc)
                    e = _errors(acc, acc_true, sinks)
                    rms = float(np.sqrt(np.mean(e ** 2)))
                    hist.append((eps, rms, float(np.percentile(e, 99.9))))
                    cand.evaluations += 1
                    ok = [h for h in hist if h[1] <= target_rms]
                    if ok and max(h[1] for h in ok) >= margin * target_rms:
                        break
                    # secant step in log eps towards margin * target (slope from the last two points)
                    if len(hist) >= 2 and hist[-1][1] != hist[-2][1] and hist[-1][1] > 0 and hist[-2][1] > 0:
                        (e1, r1, _), (e2, r2, _) = hist[-2], hist[-1]
                        slope = (math.log(r2) - math.log(r1)) / (math.log(e2) - math.log(e1))
                        slope = min(max(slope, 0.3), 3.0)
                    else:
                        slope = 1.0
                    eps = eps * (margin * target_rms / max(rms, 1e-300)) ** (1.0 / slope)
                ok = [h for h in hist if h[1] <= target_rms]
                if ok:
                    cand.eps, cand.rms, cand.p999 = max(ok, key=lambda h: h[0])
                    ctx.set_params(eps=cand.eps)
                    cand.ms = _time_ms(ctx, x, mu, psi, acc)
                ctx.close()
                tried.append(cand)
                if log:
                    log(cand)
                if cand.ms < (best.ms if best else float("inf")):
                    best = cand
    if best is None:
        raise RuntimeError("no candidate reached the target error")
    return TuneResult(best, tried, target_rms, int(sinks.numel()), time.perf_counter() - t0)
