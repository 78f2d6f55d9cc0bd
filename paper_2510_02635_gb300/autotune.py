"""Autotuner of the cloud tiling, and the batched driver built on it.

The tunable is `ctas`: how many CTAs one streaming pass over a query's particle cloud
uses (rows per CTA = M / ctas).  Wide tilings fill the GPU for one large instance;
narrow ones leave SMs to the other instances of a concurrent batch.  The tuner times a
short probe solve (same d, M and kind, N_probe levels) through a one-instance plan for
each candidate and keeps the narrowest tiling within `slack` of the fastest, per
(log2 d, M) bucket; results are cached as JSON.  All timing is on the GPU with CUDA
events; nothing here computes any part of the method.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import fbsde
from . import workloads as W

CANDIDATES = (76, 152, 304, 608, 1216)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                             "autotune.json")


def kappa_estimate(w: W.Workload) -> float:
    """Condition number of the ridge regression of a cloud of M Gaussian points in d
    dimensions, from the Marchenko-Pastur law of the sample covariance (eigenvalues in
    [(1 - sqrt q)^2, (1 + sqrt q)^2] in units of the mean, q = d / M, and d - M zero
    eigenvalues when M < d), shifted by the ridge ridge_rel * (mean eigenvalue)."""
    q = w.d / w.M
    lam = max(w.ridge_rel, 1e-12)
    hi = (1.0 + math.sqrt(q)) ** 2 + lam
    lo = ((1.0 - math.sqrt(q)) ** 2 if w.d <= w.M else 0.0) + lam
    return hi / lo


# Largest estimated condition number the FP32 stream path is used for.  The products come
# from FP32 rows, so the regression's error grows like kappa times the FP32 rounding.
# Measured against the FP64 path on 32 batch instances: the error in u was 1.3e-4 at
# kappa = 1.8e4 (M/d = 0.09), and every instance with kappa up to 1.2e4 stayed below 1e-4.
# The bound keeps a margin of 1.5 below that.
KAPPA_FP32_MAX = 8000.0


def route_precision(instances: list[W.Workload], kappa_max: float = KAPPA_FP32_MAX) -> list[W.Workload]:
    """The instances, with the FP32 ones whose regression is too ill-conditioned for FP32
    rows (kappa_estimate > kappa_max) moved to the FP64 path, where its dimension limit
    allows (d <= FBSDE_MAX_D_FP64; wider instances stay FP32)."""
    return [w.with_(precision="fp64")
            if w.precision == "fp32" and kappa_estimate(w) > kappa_max
            and w.d <= fbsde.FBSDE_MAX_D_FP64 else w for w in instances]


def bucket(w: W.Workload) -> str:
    return f"{w.kind}|d2^{int(round(math.log2(w.d)))}|M{w.M}|{w.precision}"


def problem_of(w: W.Workload, theta=None, ctas: int = 0, N: int | None = None):
    return fbsde.make_problem(w.kind, w.d, N or w.N, w.M, w.sigma, w.T, w.precision,
                              theta=theta, A=w.A, c0=w.c0, c1=w.c1,
                              c2=w.extra.get("c2", 0.0), c3=w.extra.get("c3", 0.0), h=w.h,
                              ridge_rel=w.ridge_rel, cg_tol=w.cg_tol,
                              cg_max_iter=w.cg_max_iter, newton_max_iter=w.newton_max_iter,
                              newton_tol=w.newton_tol, ctas=ctas)


def _time_plan(plan, torch, repeats: int) -> float:
    plan.launch()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(repeats):
        plan.launch()
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / repeats


def tune(instances: list[W.Workload], cache_path: str | None = DEFAULT_CACHE,
         n_probe: int = 2, repeats: int = 2, slack: float = 1.10) -> dict:
    """ctas per bucket for the given instances (cached)."""
    import torch
    table = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            table = json.load(fh)
    todo = {}
    for w in instances:
        todo.setdefault(bucket(w), w)
    changed = False
    for key, w in todo.items():
        if key in table:
            continue
        x0 = torch.zeros(1, w.d, dtype=torch.float64, device="cuda")
        times = {}
        for c in CANDIDATES:
            if c > max(1, w.M // 8) * 2:   # more CTAs than row blocks: same as the cap
                continue
            p = problem_of(w, ctas=c, N=min(n_probe, w.N))
            plan = fbsde.Plan([{"problem": p, "Q": 1, "x0": x0, "seed": w.seed}])
            times[c] = _time_plan(plan, torch, repeats)
            plan.close()
        best = min(times.values())
        chosen = min(c for c, t in times.items() if t <= slack * best)
        table[key] = {"ctas": chosen, "probe_ms": {str(c): t for c, t in times.items()}}
        changed = True
    if changed and cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        with open(cache_path, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
    return table


class Batch:
    """A batch of independent instances (Q = 1 each) in one plan, optionally autotuned.
    Route the instances through route_precision first to keep FP32 only where it meets
    the accuracy of the FP64 path."""

    def __init__(self, instances: list[W.Workload], x0s: list[np.ndarray], table: dict | None,
                 branches: int = 0):
        import torch
        self.instances = instances
        self.x0 = [torch.tensor(x, device="cuda") for x in x0s]
        specs = []
        for i, (w, x0) in enumerate(zip(instances, self.x0)):
            ctas = table[bucket(w)]["ctas"] if table else 0
            specs.append({"problem": problem_of(w, ctas=ctas), "Q": 1, "x0": x0, "seed": w.seed,
                          "solve_index0": w.extra.get("index", i)})
        self.plan = fbsde.Plan(specs, branches=branches)

    def launch(self) -> None:
        self.plan.launch()

    def results(self) -> tuple[list, list]:
        return ([float(u[0]) for u in self.plan.u0], [g[0].cpu().numpy() for g in self.plan.grad])

    def close(self) -> None:
        self.plan.close()
