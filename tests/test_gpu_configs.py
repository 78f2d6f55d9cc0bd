"""Full-size workloads in the launch configuration the benchmark uses, checked on sampled
query points that the oracle solves one by one (same seeds, same inputs)."""
import numpy as np
import pytest

import oracle
from helpers import TOL_FP32, gpu_solver, oracle_problem, rel_errors
from paper_2510_02635_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _check(w, queries):
    inp = W.inputs(w)
    solver = gpu_solver(w, theta=inp["theta"])
    out = solver.solve(torch.tensor(inp["x0"], device="cuda"), seed=w.seed, trace=True)
    assert out["status"] == 0, out["status"]
    errs = []
    for q in queries:
        ref = oracle.solve(oracle_problem(w, theta=inp["theta"], cg_tol=1e-11), inp["x0"][q],
                           w.seed, q)
        assert ref["status"] == 0
        ru, rg = rel_errors(float(out["u0"][q]), out["grad"][q].cpu().numpy(), ref)
        errs.append((q, ru, rg))
        assert ru <= TOL_FP32 and rg <= TOL_FP32, (q, ru, rg)
    return out, errs


def test_logistic_d1000_64_queries():
    out, errs = _check(W.C1_LOGISTIC_D1000, [0, 37, 63])
    assert int(out["cg_iters"].max()) < 200


def test_hjb_logquad_d1000():
    _check(W.C4_HJB_D1000, [0])


def test_allen_cahn_d10000_16_queries():
    """d = 10^4, M = 16384, N = 50, 16 queries (the benchmark workload): query 5 checked
    against the oracle (about two minutes of CPU time)."""
    out, errs = _check(W.C2_AC_D10000, [5])
    assert int(out["cg_iters"].max()) < 200
