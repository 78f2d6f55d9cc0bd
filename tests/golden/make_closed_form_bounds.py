#!/usr/bin/env python
"""Writes closed_form_bounds.json: the error of the scheme itself against the closed-form
solution, measured with the FP64 oracle, at the two full-size workloads that have a closed
form (Allen-Cahn with manufactured source at d = 10^4, M = 16384, N = 50; the logistic
gradient-dependent driver at d = 1000, M = 4096, N = 20).

For each workload the oracle solves query 0's point x0 with several independent Philox
streams (solve indices).  The error of the estimator has a bias (the O(dt) time
discretisation of Theorem 3.1 plus the kernel-localisation and ridge bias of the
regression) and a Monte-Carlo spread over the streams.  The stored bound on the error of
any one solve of that workload is |mean error| + 4 (standard deviation over the streams),
for u (signed relative error) and for grad u (relative Euclidean error).  Solve index 0 is
exactly the first query of the benchmark's solve, so its oracle result is stored too: the
benchmark reports the GPU's difference from it.

    python tests/golden/make_closed_form_bounds.py [--streams 6]

Calls only the oracle and the seeded input module; several minutes on 8 cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2510_02635_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "closed_form_bounds.json")


def oracle_hash() -> str:
    return hashlib.sha256(open(os.path.join(ROOT, "oracle", "fbsde_oracle.c"), "rb").read()).hexdigest()


def sweep(w: W.Workload, streams: int) -> dict:
    inp = W.inputs(w)
    x0 = inp["x0"][0]
    p = oracle.Problem(w.kind, w.d, w.sigma, w.T, w.N, w.M, theta=inp["theta"], h=w.h,
                       ridge_rel=w.ridge_rel, cg_tol=1e-12)
    u_star, g_star = W.exact_solution(w, x0)
    eu, eg, runs = [], [], []
    ref = None
    for s in range(streams):
        t0 = time.perf_counter()
        r = oracle.solve(p, x0, w.seed, s)
        assert r["status"] == 0, r["status"]
        eu.append((r["u0"] - u_star) / abs(u_star))
        eg.append(float(np.linalg.norm(r["grad"] - g_star) / np.linalg.norm(g_star)))
        runs.append({"solve_index": s, "u0": r["u0"], "rel_err_u": eu[-1], "rel_err_grad": eg[-1],
                     "seconds": time.perf_counter() - t0})
        print(f"{w.name} stream {s}: u0={r['u0']:.10f} u*={u_star:.10f} "
              f"err_u={eu[-1]:.3e} err_grad={eg[-1]:.3e} ({runs[-1]['seconds']:.0f} s)",
              flush=True)
        if s == 0:
            ref = {"u0": r["u0"], "grad": [float(v) for v in r["grad"]]}
    eu, eg = np.array(eu), np.array(eg)
    return {"workload": w.name, "query": 0, "u_star": u_star, "streams": streams, "runs": runs,
            "u": {"mean": float(eu.mean()), "std": float(eu.std(ddof=1)),
                  "bound": float(abs(eu.mean()) + 4 * eu.std(ddof=1))},
            "grad": {"mean": float(eg.mean()), "std": float(eg.std(ddof=1)),
                     "bound": float(eg.mean() + 4 * eg.std(ddof=1))},
            "oracle_query0": ref}


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--streams", type=int, default=6)
    a = ap.parse_args()
    out = {"oracle_source_sha256": oracle_hash(), "threads": oracle.max_threads(),
           "command": "python tests/golden/make_closed_form_bounds.py --streams %d" % a.streams,
           "bound_rule": "|mean relative error| + 4 std over independent Philox streams "
                         "(u: signed; grad u: Euclidean norm, relative)",
           "workloads": {}}
    for w in (W.C1_LOGISTIC_D1000, W.C2_AC_D10000):
        out["workloads"][w.name] = sweep(w, a.streams)
        with open(OUT, "w") as fh:
            json.dump(out, fh, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
