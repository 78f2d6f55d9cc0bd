"""Test helpers: run one workload through the CPU oracle and through the C-ABI library
on identical seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2510_02635_gb300 import workloads as W

# The u / grad bar of the FP32 path against the FP64 oracle (relative; the gradient
# error is measured against max(|grad u|, |u|)), and of the FP64 path.
TOL_FP32 = 1e-4
TOL_FP64 = 1e-10


def oracle_problem(w: W.Workload, theta=None, cg_tol: float = 1e-12) -> oracle.Problem:
    return oracle.Problem(w.kind, w.d, w.sigma, w.T, w.N, w.M, theta=theta, A=w.A, c0=w.c0,
                          c1=w.c1, c2=w.extra.get("c2", 0.0), c3=w.extra.get("c3", 0.0),
                          h=w.h, ridge_rel=w.ridge_rel, cg_tol=cg_tol,
                          newton_tol=w.newton_tol, newton_max_iter=w.newton_max_iter)


def gpu_solver(w: W.Workload, theta=None, Q: int | None = None, **over):
    from paper_2510_02635_gb300 import fbsde
    params = dict(A=w.A, c0=w.c0, c1=w.c1, c2=w.extra.get("c2", 0.0),
                  c3=w.extra.get("c3", 0.0), h=w.h, ridge_rel=w.ridge_rel, cg_tol=w.cg_tol,
                  cg_max_iter=w.cg_max_iter, newton_max_iter=w.newton_max_iter,
                  newton_tol=w.newton_tol)
    params.update(over)
    return fbsde.Solver(w.kind, w.d, w.N, w.M, w.sigma, w.T, Q=Q or w.Q,
                        precision=w.precision, theta=theta, **params)


def rel_errors(u_gpu: float, g_gpu: np.ndarray, ref: dict) -> tuple[float, float]:
    u_ref = ref["u0"]
    rel_u = abs(u_gpu - u_ref) / abs(u_ref)
    scale = max(np.linalg.norm(ref["grad"]), abs(u_ref))
    rel_g = np.linalg.norm(g_gpu - ref["grad"]) / scale
    return rel_u, rel_g
