#!/usr/bin/env python
"""Throughput of the localized FBSDE hot path on GB300 (one JSON line on stdout).

A step is one whole solve (Algorithm 1: forward sweep + all N backward levels) of
the d = 10^4 Allen-Cahn workload: Q = 16 query points, M = 16384 particles each,
N = 50 steps, FP32 particle stream with FP64 regression solve and Newton.
Metric: particle-dim updates per second = Q M d N / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU (torchrun, one rank per GPU): the query points shard across ranks with no
collective on the data path (weak scaling: every rank solves its own 16 queries);
the step time is the maximum over ranks.  The reference arm (--impl reference) times
the FP64 CPU oracle on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2510_02635_gb300 import workloads as W  # noqa: E402

WORKLOAD = W.C2_AC_D10000
METRIC = "particle-dim updates/sec (K*M*d per step)"
UNIT = "particle-dim updates/s"


def _matvec_traffic(w: W.Workload) -> float | None:
    """DRAM bytes of one product launch of this workload, scaled from the ncu capture in
    profiles/matvec_traffic.txt; None when the kernel source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "matvec_traffic.txt")
    try:
        lines = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    kv = {ln[0]: ln[1:] for ln in lines}
    src = os.path.join(ROOT, kv["kernel_source"][2])
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != kv["kernel_source"][1]:
        return None
    ctas = w.Q * min(max(1, w.M // 8), -(-608 // w.Q))   # CTAs of one product launch
    return (float(kv["read_bytes_per_particle_dim"][0]) * w.Q * w.M * w.d
            + float(kv["write_bytes_per_cta"][0]) * ctas)


def _step_traffic(w: W.Workload) -> float | None:
    """DRAM bytes of the fused step's launches in one solve (N - 1 level steps; the
    terminal launch writes only), scaled from the ncu capture in profiles/step_traffic.txt;
    None when the kernel source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "step_traffic.txt")
    try:
        lines = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    kv = {ln[0]: ln[1:] for ln in lines}
    src = os.path.join(ROOT, kv["kernel_source"][2])
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != kv["kernel_source"][1]:
        return None
    pd = w.Q * w.M * w.d
    rd, wr = float(kv["read_bytes_per_particle_dim"][0]), float(kv["write_bytes_per_particle_dim"][0])
    return (rd + wr) * pd * (w.N - 1) + wr * pd


def _accuracy(w: W.Workload, u: "np.ndarray", grad: "np.ndarray") -> dict:
    """Error of every query's u(0, x0) and grad u(0, x0) against the workload's closed
    form, and of query 0 against the FP64 oracle's solve of the same stream (stored by
    tests/golden/make_closed_form_bounds.py, valid while the oracle source is unchanged),
    with the scheme's own error bound from that oracle sweep."""
    import hashlib

    import numpy as np
    x0 = W.inputs(w)["x0"]
    eu, eg = [], []
    for q in range(u.shape[0]):
        us, gs = W.exact_solution(w, x0[q % x0.shape[0]])
        eu.append(abs(float(u[q]) - us) / abs(us))
        eg.append(float(np.linalg.norm(grad[q] - gs) / np.linalg.norm(gs)))
    out = {"closed_form": {"rel_err_u": eu, "rel_err_grad": eg, "max_rel_err_u": max(eu),
                           "max_rel_err_grad": max(eg)}}
    path = os.path.join(ROOT, "tests", "golden", "closed_form_bounds.json")
    try:
        ref = json.load(open(path))
    except OSError:
        out["vs_oracle"] = {"unavailable": "no stored oracle solve"}
        return out
    src = hashlib.sha256(open(os.path.join(ROOT, "oracle", "fbsde_oracle.c"), "rb").read()).hexdigest()
    entry = ref["workloads"].get(w.name)
    if entry is None or src != ref["oracle_source_sha256"]:
        out["vs_oracle"] = {"unavailable": "stored oracle solve is stale or missing"}
        return out
    o = entry["oracle_query0"]
    og = np.asarray(o["grad"])
    out["vs_oracle"] = {"query": 0, "rel_err_u": abs(float(u[0]) - o["u0"]) / abs(o["u0"]),
                        "rel_err_grad": float(np.linalg.norm(grad[0] - og) /
                                              max(np.linalg.norm(og), abs(o["u0"]))),
                        "tolerance": 1e-4}
    out["scheme_bound"] = {"rel_err_u": entry["u"]["bound"], "rel_err_grad": entry["grad"]["bound"],
                           "streams": entry["streams"], "rule": ref["bound_rule"],
                           "all_queries_within": bool(max(eu) <= entry["u"]["bound"] and
                                                      max(eg) <= entry["grad"]["bound"])}
    return out


def _peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.gpu_id = gpu_id

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _gpu_uuid(torch) -> str | None:
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(w: W.Workload, levels: int = 2) -> dict:
    """The FP64 oracle on one query of the workload: the full forward sweep and `levels`
    backward levels, timed per phase; the whole-solve time is extrapolated as
    t_forward + N t_level, so value = M d N / that time."""
    import oracle
    inp = W.inputs(w)
    p = oracle.Problem(w.kind, w.d, w.sigma, w.T, w.N, w.M, theta=inp["theta"], h=w.h,
                       ridge_rel=w.ridge_rel, cg_tol=1e-12)
    t0 = time.perf_counter()
    r = oracle.solve(p, inp["x0"][0], w.seed, 0, max_levels=levels)
    wall = time.perf_counter() - t0
    t_level = r["backward_s"] / levels
    t_full = r["forward_s"] + w.N * t_level
    return {"value": w.M * w.d * w.N / t_full, "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle", "wall_s": wall, "forward_s": r["forward_s"],
            "level_s": t_level,
            "sample": (f"1 of {w.Q} queries (d={w.d}, M={w.M}), full forward sweep of "
                       f"N={w.N} steps + {levels} backward levels in FP64, whole-solve time "
                       f"extrapolated as t_fwd + N*t_level")}


def cpu_model() -> str:
    """Host CPU model (lscpu), or the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip() + f" ({platform.machine()})"
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def oracle_baseline(w: W.Workload) -> dict:
    """The oracle on the host cores: one warm-up, then the best of 3 samples (forward sweep
    + 1 backward level each, extrapolated as t_fwd + N t_level) with every core."""
    oracle_sample(w, levels=1)
    runs = [oracle_sample(w, levels=1) for _ in range(3)]
    best = max(runs, key=lambda r: r["value"])
    best.pop("wall_s")
    best["sample"] += "; best of 3 after 1 warm-up"
    best["cpu_model"] = cpu_model()
    best["values_of_3"] = [r["value"] for r in runs]
    return best


def start_single_thread_baseline(w: W.Workload):
    """The same oracle sample with one thread, in a background process (its result is read
    by finish_single_thread_baseline)."""
    out = tempfile.mktemp(prefix="oracle1_", suffix=".json")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "from paper_2510_02635_gb300 import workloads as W; "
            "r = bench.oracle_sample(W.ALL[%r], levels=1); r.pop('wall_s'); "
            "json.dump(r, open(%r, 'w'))" % (ROOT, w.name, out))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.Popen([sys.executable, "-c", code], env=env,
                            stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL), out


def finish_single_thread_baseline(handle, timeout: float = 600.0) -> dict | None:
    proc, out = handle
    try:
        proc.wait(timeout=timeout)
        r = json.load(open(out))
        return {"value": r["value"], "cores": 1, "level_s": r["level_s"],
                "forward_s": r["forward_s"], "sample": r["sample"] + " (one run)"}
    except (subprocess.TimeoutExpired, OSError, ValueError):
        proc.kill()
        return None


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    w = WORKLOAD
    for _ in range(args.warmup):
        oracle_sample(w, levels=1)
    vals, wall = [], 0.0
    for _ in range(args.steps):
        s = oracle_sample(w, levels=1)
        vals.append(s["value"])
        wall += s["wall_s"]
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "d": w.d, "M": w.M, "N": w.N,
                                            "Q": 1, "sample": s["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": s["cores"], "kind": "oracle",
                             "sample": s["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- extras
def _events_ms(fn, repeats: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(repeats):
        fn()
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / repeats


def extra_batched(sample: int = 128) -> dict:
    """The 512-instance uneven batch in one autotuned FP32 plan (one graph launch per
    step), and on a stratified sample of `sample` instances (every fourth instance in the
    order of (d, M): every size class, up to d = 10^4): that batched FP32 plan vs the FP64
    form solving the same instances one at a time (one single-instance plan each, launched
    and completed in turn; capture time excluded on both sides)."""
    import numpy as np
    import torch

    from paper_2510_02635_gb300 import autotune, fbsde
    # FP32 instances whose regression is too ill-conditioned for FP32 rows run in FP64
    inst = autotune.route_precision(W.batch_instances())
    x0s = W.batch_x0(inst)
    t0 = time.perf_counter()
    table = autotune.tune(inst)
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch = autotune.Batch(inst, x0s, table)
    create_s = time.perf_counter() - t0
    ms_full = _events_ms(batch.launch, 2)
    status = int(batch.plan.diagnostics().status)
    # algorithmic bytes of one batch, per instance in units of one pass over its rows
    # (4 B per particle-dim in FP32, 8 B in FP64): the fused step (FP32, d <= 10240) writes
    # the end point once and reads + writes the rows at each of the N - 1 levels; the
    # unfused path writes the end point, reads it for the first moments, and reads +
    # writes + reads again at each level; every CG product reads the rows once
    cg = [int(batch.plan.instance_diagnostics(i).cg_iters_total) for i in range(len(inst))]

    def passes(w, c):
        fused = w.precision == "fp32" and (w.d + 3) // 4 * 4 <= 10240
        return (1 + 2 * (w.N - 1) if fused else 2 + 3 * (w.N - 1)) + c
    nbytes = sum((4.0 if w.precision == "fp32" else 8.0) * w.M * w.d * passes(w, c)
                 for w, c in zip(inst, cg))
    batch.close()
    units_full = sum(w.M * w.d * w.N for w in inst)
    order = sorted(range(len(inst)), key=lambda i: (inst[i].d, inst[i].M, i))
    pick = sorted(order[::max(1, len(inst) // sample)])
    sub, subx = [inst[i] for i in pick], [x0s[i] for i in pick]
    b32 = autotune.Batch(sub, subx, table)
    ms32 = _events_ms(b32.launch, 2)
    u32, g32 = b32.results()
    b32.close()
    all64 = W.batch_instances(precision="fp64")
    inst64 = [all64[i] for i in pick]
    plans = []
    for w, x0 in zip(inst64, subx):
        plans.append(fbsde.Plan([{"problem": autotune.problem_of(w), "Q": 1, "seed": w.seed,
                                  "x0": torch.tensor(x0, device="cuda"),
                                  "solve_index0": w.extra["index"]}]))

    def seq64():
        for pl in plans:
            pl.launch()
            torch.cuda.synchronize()
    ms64 = _events_ms(seq64, 1)
    # accuracy of the batched form against the FP64 per-instance results (the FP64 path
    # matches the oracle to ~1e-13): relative error of u and of grad u (scaled by
    # max(|grad u|, |u|)), with each instance's regression shape M/d
    errs = []
    for i, pl in enumerate(plans):
        u64, g64 = float(pl.u0[0][0]), pl.grad[0][0].cpu().numpy()
        scale = max(float(np.linalg.norm(g64)), abs(u64))
        errs.append((abs(u32[i] - u64) / abs(u64),
                     float(np.linalg.norm(g32[i] - g64)) / scale, sub[i].M / sub[i].d))
    for pl in plans:
        pl.close()
    ok = [e for e in errs if max(e[0], e[1]) <= 1e-4]
    units_sub = sum(w.M * w.d * w.N for w in sub)
    return {"workload": W.BATCH_NAME, "instances": len(inst),
            "fp64_routed": sum(1 for w in inst if w.precision == "fp64"),
            "kappa_fp32_max": autotune.KAPPA_FP32_MAX,
            "value": units_full / (ms_full * 1e-3),
            "unit": UNIT, "ms_per_batch": ms_full, "device_status": status,
            "plan_create_s": create_s, "autotune_s": tune_s, "cg_iters_total": sum(cg),
            "algorithmic_gb": nbytes / 1e9, "effective_gbs": nbytes / (ms_full * 1e-3) / 1e9,
            "speedup_sample": {"instances": len(pick), "selection": "every 4th instance in "
                               "the order of (d, M)", "max_d": max(w.d for w in sub),
                               "fp32_batched_ms": ms32,
                               "fp64_per_instance_ms": ms64, "ratio": ms64 / ms32,
                               "fp64_routed": sum(1 for w in sub if w.precision == "fp64"),
                               "fp32_value": units_sub / (ms32 * 1e-3),
                               "batched_vs_fp64": {
                                   "max_rel_err_u": max(e[0] for e in errs),
                                   "max_rel_err_grad": max(e[1] for e in errs),
                                   "within_1e-4": len(ok),
                                   "worst_M_over_d": max(errs, key=lambda e: max(e[0], e[1]))[2]}}}


def extra_batched_sharded(rank: int, world: int, dist) -> dict:
    """Multi-GPU: the 512-instance uneven batch split over the ranks by estimated cost
    (shard.cost_shard, no collective on the data path); each rank launches its share as one
    autotuned plan; the batch time is the maximum over ranks."""
    import torch

    from paper_2510_02635_gb300 import autotune, shard
    inst = autotune.route_precision(W.batch_instances())
    x0s = W.batch_x0(inst)
    mine = shard.cost_shard(inst, world)[rank]
    sub = [inst[i] for i in mine]
    # each rank tunes its own buckets without the shared cache file (no concurrent writers)
    batch = autotune.Batch(sub, [x0s[i] for i in mine], autotune.tune(sub, cache_path=None))
    dist.barrier()
    ms = _events_ms(batch.launch, 2)
    status = int(batch.plan.diagnostics().status)
    batch.close()
    t = torch.tensor([ms], device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    units = sum(w.M * w.d * w.N for w in inst)
    return {"workload": W.BATCH_NAME, "instances": len(inst), "ranks": world,
            "instances_this_rank": len(sub), "ms_per_batch_max_over_ranks": ms_max,
            "value": units / (ms_max * 1e-3), "unit": UNIT, "device_status_rank0": status,
            "split": "cost_shard (largest estimated cost first onto the least loaded rank)"}


def extra_adjoint() -> dict:
    """The reverse sweep (d u / d x0, d u / d theta) of the log-quadratic workload vs its
    primal solve, both eager, CUDA events."""
    from paper_2510_02635_gb300 import fbsde
    w = W.C4_HJB_D1000
    inp = W.inputs(w)
    solver = fbsde.Solver(w.kind, w.d, w.N, w.M, w.sigma, w.T, Q=w.Q, precision=w.precision,
                          theta=inp["theta"], cg_tol=w.cg_tol)
    ms_primal = _events_ms(lambda: solver.solve(inp["x0"], seed=w.seed, check_status=False), 3)
    ms_adj = _events_ms(lambda: solver.adjoint(inp["x0"], seed=w.seed, with_theta=True,
                                               check_status=False), 3)
    return {"workload": w.name, "primal_ms": ms_primal, "adjoint_ms": ms_adj,
            "adjoint_over_primal": ms_adj / ms_primal,
            "note": "adjoint = re-run of the solve with its tape + the reverse sweep"}


def extra_anchored() -> dict:
    """Algorithm 1 with one regression per particle anchor on the plain-scheme workload
    (Allen-Cahn with manufactured source, d = 100, M = 2048, N = 10, x0 = 0, FP32), against
    the single-anchor solve and the closed form u*(0, x0) = e^{-T} mean_i cos x0_i."""
    import torch

    from paper_2510_02635_gb300 import fbsde
    w = W.C0_AC_D100.with_(precision="fp32", cg_tol=1e-6)
    x0 = torch.zeros(1, w.d, dtype=torch.float64, device="cuda")
    p = fbsde.make_problem(w.kind, w.d, w.N, w.M, w.sigma, w.T, w.precision, h=w.h,
                           ridge_rel=w.ridge_rel, cg_tol=w.cg_tol)
    ws = torch.empty(fbsde.fbsde_anchored_workspace_bytes(p), dtype=torch.uint8, device="cuda")
    u = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(1, w.d, dtype=torch.float64, device="cuda")

    status = [0]

    def run():
        fbsde.check(fbsde.fbsde_solve_anchored(p, 1, x0, w.seed, 0, u, g, ws))

    ms = _events_ms(run, 3)
    dg = fbsde.fbsde_anchored_diagnostics(p, ws)
    status[0] = int(dg.status)
    passes_full = dg.cg_iters_total / w.N
    u_anchored = float(u[0])
    single = fbsde.Solver(w.kind, w.d, w.N, w.M, w.sigma, w.T, Q=1, precision=w.precision,
                          h=w.h, ridge_rel=w.ridge_rel, cg_tol=w.cg_tol)
    u_single = float(single.solve(x0, seed=w.seed)["u0"][0])
    exact = math.exp(-w.T) * 1.0   # mean of cos 0
    out = {"workload": "ac_manufactured_d100_M2048_N10_Q1_fp32_per_anchor", "ms_per_solve": ms,
           "status": status[0], "unit_note": "M^2 d N anchor-particle-dims per solve",
           "u0_single_anchor": u_single, "u0_exact": exact,
           "abs_err_single_anchor": abs(u_single - exact), "cg_passes_per_level": passes_full}
    if status[0] == 0:   # a failed solve reports its status only
        out.update(value=w.M * w.M * w.d * w.N / (ms * 1e-3), u0=u_anchored,
                   abs_err=abs(u_anchored - exact))
    # the same solve with each anchor's regression over a batch of K particles (the
    # batch reading of Remark 2.1: cyclic windows, products restricted to their band), at
    # M = 2048 and M = 4096: the cost per level grows like M (K + 128) d, not M^2 d
    K = 256
    out["batch"] = []
    for Mb in (w.M, 2 * w.M):
        try:
            pb = fbsde.make_problem(w.kind, w.d, w.N, Mb, w.sigma, w.T, w.precision, h=w.h,
                                    ridge_rel=w.ridge_rel, cg_tol=w.cg_tol)
            wsb = ws if Mb == w.M else torch.empty(fbsde.fbsde_anchored_workspace_bytes(pb),
                                                   dtype=torch.uint8, device="cuda")
            st_b = [0]

            def run_batch():
                fbsde.check(fbsde.fbsde_solve_batch(pb, K, 1, x0, w.seed, 0, u, g, wsb))

            ms_b = _events_ms(run_batch, 3)
            dgb = fbsde.fbsde_anchored_diagnostics(pb, wsb)
            st_b[0] = int(dgb.status)
            u_b = float(u[0])
            rec = {"K": K, "M": Mb, "ms_per_solve": ms_b, "status": st_b[0],
                   "cg_passes_per_level": dgb.cg_iters_total / w.N}
            if st_b[0] == 0:
                rec.update(u0=u_b, abs_err=abs(u_b - exact))

            # the same regressions solved directly (L D L^T of each anchor's operator)
            def run_direct():
                fbsde.check(fbsde.fbsde_solve_batch_direct(pb, K, 1, x0, w.seed, 0, u, g, wsb))

            ms_d = _events_ms(run_direct, 3)
            st_d = int(fbsde.fbsde_anchored_diagnostics(pb, wsb).status)
            rec["direct"] = {"ms_per_solve": ms_d, "status": st_d}
            if st_d == 0:
                u_d = float(u[0])
                rec["direct"].update(u0=u_d, abs_err=abs(u_d - exact))
                if st_b[0] == 0:
                    rec["direct"]["rel_diff_u0_vs_cg"] = abs(u_d - u_b) / abs(u_b)
            out["batch"].append(rec)
            del wsb
        except Exception as e:   # reported in the line, never fatal to the bench
            out["batch"].append({"K": K, "M": Mb, "error": repr(e)})
    if out["batch"] and "ms_per_solve" in out["batch"][0]:
        out["batch_speedup_vs_all_particles"] = ms / out["batch"][0]["ms_per_solve"]
        out["batch_direct_speedup_vs_all_particles"] = (
            ms / out["batch"][0]["direct"]["ms_per_solve"])
    return out


def extra_logistic() -> dict:
    """The d = 1000, 64-query logistic workload through a plan (device-side CG loops)."""
    import torch

    from paper_2510_02635_gb300 import autotune, fbsde
    w = W.C1_LOGISTIC_D1000
    x0 = torch.tensor(W.inputs(w)["x0"], device="cuda")
    plan = fbsde.Plan([{"problem": autotune.problem_of(w), "Q": w.Q, "x0": x0, "seed": w.seed}])
    ms = _events_ms(plan.launch, 5)
    plan.close()
    return {"workload": w.name, "value": w.particle_dim_updates / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms}


def extra_drift() -> dict:
    """Row f4: the forward SDE with an Ornstein-Uhlenbeck drift and a state-dependent
    diffusion (Euler-Maruyama paths kept at checkpoints, segments recomputed), d = 1000,
    16 queries, FP32: time per solve, the per-family split of one more solve, the
    Euler-Maruyama kernel's algorithmic bandwidth (8 B per particle-dim per step; the
    first step of a sweep only writes) and the error against the closed form."""
    import numpy as np
    import torch

    from paper_2510_02635_gb300 import fbsde
    w = W.F4_DRIFT_AC_D1000
    inp = W.inputs(w)
    x0 = torch.tensor(inp["x0"], device="cuda")
    solver = fbsde.Solver(w.kind, w.d, w.N, w.M, w.sigma, w.T, Q=w.Q, precision=w.precision,
                          h=w.h, ridge_rel=w.ridge_rel, cg_tol=w.cg_tol, **w.extra)
    ms = _events_ms(lambda: solver.solve(x0, seed=w.seed, check_status=False), 3)
    out = solver.solve(x0, seed=w.seed)
    torch.cuda.synchronize()
    rec = {"workload": w.name, "ms_per_solve": ms, "status": out["status"],
           "value": w.particle_dim_updates / (ms * 1e-3), "unit": UNIT}
    fbsde.fbsde_profile_start(1 << 16)
    solver.solve(x0, seed=w.seed, check_status=False)
    torch.cuda.synchronize()
    split = fbsde.fbsde_profile_stop()
    rec["kernels_ms_per_solve"] = {k: v["total_ms"] for k, v in split.items() if v["launches"]}
    em = split["forward"]
    pdims = w.Q * w.M * w.d
    em_bytes = (8 * em["launches"] - 4) * pdims
    if em["total_ms"] > 0:
        rec["euler_maruyama"] = {"launches_per_solve": em["launches"],
                                 "gbs": em_bytes / (em["total_ms"] * 1e-3) / 1e9,
                                 "note": "N forward steps + the levels recomputed from "
                                         "checkpoints on the way back; timed one by one "
                                         "with the launch profiler"}
    if out["status"] == 0:
        u = out["u0"].cpu().numpy()
        errs = [abs(float(u[q]) - W.exact_solution(w, inp["x0"][q])[0]) /
                abs(W.exact_solution(w, inp["x0"][q])[0]) for q in range(w.Q)]
        rec["rel_err_u_closed_form"] = {"max": max(errs), "mean": float(np.mean(errs))}
    return rec


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank: int, world: int) -> None:
    import numpy as np
    import torch

    from paper_2510_02635_gb300 import build as gbuild
    from paper_2510_02635_gb300 import fbsde

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if not os.path.exists(fbsde.LIB_PATH):
        gbuild.build()
    fbsde.load_library()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = WORKLOAD
    inp = W.inputs(w)
    x0 = torch.tensor(inp["x0"], device="cuda")
    solver = fbsde.Solver(w.kind, w.d, w.N, w.M, w.sigma, w.T, Q=w.Q, precision=w.precision,
                          theta=inp["theta"], h=w.h, ridge_rel=w.ridge_rel, cg_tol=w.cg_tol,
                          cg_max_iter=w.cg_max_iter)
    sidx = rank * w.Q  # each rank owns its own query points / Philox streams
    stream = torch.cuda.current_stream()

    def step():
        out = torch.empty(w.Q, dtype=torch.float64, device="cuda")
        grad = torch.empty(w.Q, w.d, dtype=torch.float64, device="cuda")
        fbsde.check(fbsde.fbsde_solve(solver.problem, w.Q, x0, w.seed, sidx, out, grad,
                                      solver.workspace), "fbsde_solve")
        return out, grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K whole solves, device time by CUDA events on the stream; the
    # library's launch profiler brackets only the matrix-free product (the roofline
    # kernel) with events, so its own event records stay out of the other kernels
    fbsde.fbsde_profile_start(1 << 20)
    fbsde.fbsde_profile_select(["matvec", "step"])
    with ClockSampler(_gpu_uuid(torch)) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            u, g = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    prof = fbsde.fbsde_profile_stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    units = w.particle_dim_updates * world
    value = units / (ms * 1e-3)

    # ---- per-level CG iterations of the same solve (deterministic): algorithmic bytes
    tr = solver.solve(x0, seed=w.seed, solve_index0=sidx, trace=True)
    cg_iters = tr["cg_iters"].cpu().numpy()
    status = tr["status"]
    # matrix-free products per step: one per CG pass of each query (the warm start's
    # product comes out of the moments pass).  While the profiler times the product
    # kernel the library launches the first FBSDE_PROFILED_EAGER_PASSES passes of every
    # CG loop one by one (those are the bracketed launches) and the rest through a CUDA
    # graph, so the timed launches carry min(iters, that many) products per query-level.
    products = int(cg_iters.sum())
    eager = fbsde.FBSDE_PROFILED_EAGER_PASSES
    products_timed = int(np.minimum(cg_iters, eager).sum())
    mv = prof["matvec"]
    mv_ms_step = mv["total_ms"] / args.steps
    bytes_per_product = 4.0 * w.M * w.d   # one FP32 read of the particle cloud
    achieved = bytes_per_product * products_timed / (mv_ms_step * 1e-3) / 1e9
    peaks = _peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    # the fused per-level step (row read + write, 8 B per particle-dim; the forward sweep's
    # end point writes only, 4 B), timed inside the same region
    st_k = prof["step"]
    step_ms = st_k["total_ms"] / args.steps
    step_bytes = 8.0 * w.Q * w.M * w.d * (w.N - 1) + 4.0 * w.Q * w.M * w.d
    step_gbs = step_bytes / (step_ms * 1e-3) / 1e9
    # kernels the library launched one by one, plus those run inside the CG-loop graphs
    # (one reset kernel per level, and three per pass beyond the eager ones, the passes
    # rounded up to the two per iteration of the loop)
    beyond = np.maximum(cg_iters.reshape(w.Q, w.N).max(axis=0) - eager, 0)
    launches = sum(v["launches"] for v in prof.values()) + \
        args.steps * int(w.N + 3 * (2 * ((beyond + 1) // 2)).sum())

    # ---- per-family split: one more solve, every launch bracketed (outside the timed region)
    fbsde.fbsde_profile_start(1 << 18)
    step()
    torch.cuda.synchronize()
    split = fbsde.fbsde_profile_stop()

    # ---- end to end: the host-buffer entry point (copies inside the timed region)
    ps = fbsde.make_problem(w.kind, w.d, w.N, w.M, w.sigma, w.T, w.precision,
                            h=w.h, ridge_rel=w.ridge_rel, cg_tol=w.cg_tol,
                            cg_max_iter=w.cg_max_iter)
    need = fbsde.fbsde_workspace_bytes(ps, w.Q) + fbsde.fbsde_host_staging_bytes(ps, w.Q)
    del solver
    torch.cuda.empty_cache()
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    x0_h = torch.tensor(inp["x0"]).pin_memory().numpy()
    u_h = torch.zeros(w.Q, dtype=torch.float64).pin_memory().numpy()
    g_h = torch.zeros(w.Q, w.d, dtype=torch.float64).pin_memory().numpy()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st = fbsde.fbsde_solve_host(ps, w.Q, x0_h, w.seed, sidx, u_h, g_h, ws)
        if st not in (0,):
            raise RuntimeError(f"fbsde_solve_host: {fbsde.fbsde_status_string(st)}")
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = units / e2e_s

    cpu, single = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(w)
        single = start_single_thread_baseline(w)   # runs while the GPU extras run
    extras = {}
    if world > 1 and not args.no_extras:
        del ws
        torch.cuda.empty_cache()
        extras = {"batched_sharded": extra_batched_sharded(rank, world, dist)}
    if rank == 0 and world == 1 and not args.no_extras:
        del ws
        torch.cuda.empty_cache()
        extras = {"batched": extra_batched(), "adjoint": extra_adjoint(),
                  "logistic_d1000_plan": extra_logistic(), "per_anchor": extra_anchored(),
                  "drift": extra_drift()}

    if single is not None:
        cpu["single_thread"] = finish_single_thread_baseline(single)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "d": w.d, "M": w.M, "N": w.N,
                       "Q_per_gpu": w.Q, "precision": "fp32 stream, fp64 solve/Newton",
                       "cg_tol": w.cg_tol, "l2": "inputs larger than L2 (10.5 GB state)",
                       "u0_per_query_ms": ms / w.Q},
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(x0_h.nbytes),
                    "d2h_bytes_per_step": int(u_h.nbytes + g_h.nbytes),
                    "ms_per_step": 1e3 * e2e_s},
            "gpu_launches": launches,
            "gpu_launches_per_step": launches / args.steps,
            "roofline": {"kernel": "matvec", "bound": "hbm", "achieved": achieved,
                         "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": _matvec_traffic(w),
                         "traffic_source": "ncu capture at Q=4, M=16384 scaled per particle-dim "
                                           "and per CTA (profiles/matvec_traffic.txt)",
                         "algorithmic_bytes_per_product": bytes_per_product,
                         "products_per_step": products,
                         "products_timed_per_step": products_timed,
                         "kernel_ms_per_step": mv_ms_step},
            "kernels_ms_per_step": {k: v["total_ms"] for k, v in split.items()},
            "kernels_ms_note": "one extra solve after the timed region with every launch "
                               "bracketed by events (the timed region brackets only matvec "
                               "and step)",
            "roofline_step": {"kernel": "step", "bound": "hbm", "achieved": step_gbs,
                              "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                              "frac": step_gbs / peak, "traffic": _step_traffic(w),
                              "traffic_source": "ncu capture of the level step at Q=4, "
                                                "M=16384 scaled per particle-dim "
                                                "(profiles/step_traffic.txt); per solve",
                              "algorithmic_bytes_per_solve": step_bytes,
                              "launches_per_solve": st_k["launches"] / args.steps,
                              "kernel_ms_per_step": step_ms},
            "cg_iters_mean": float(cg_iters.mean()), "cg_iters_max": int(cg_iters.max()),
            "device_status": status,
            "u0_sample": float(u[0]),
            "accuracy": _accuracy(w, u.cpu().numpy(), g.cpu().numpy()),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched / adjoint / d=1000 measurements")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
