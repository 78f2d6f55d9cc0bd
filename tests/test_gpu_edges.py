"""Edge shapes of the CUDA path against the oracle: the smallest problem (d = 1, M = 2,
N = 1), more queries than CTAs of a streaming pass, the widest rows of each
product-kernel variant (2560 chunks: one 10-warp team; 2561: the 544-thread variant),
the largest dimension accepted in each precision, and the dimension just beyond it
(rejected on the host)."""
import math

import numpy as np
import pytest

import oracle
from helpers import TOL_FP32, TOL_FP64, gpu_solver, oracle_problem, rel_errors
from paper_2510_02635_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _w(kind, d, M, N, Q, prec, seed=11, **kw):
    return W.Workload(f"edge_{kind}_{d}_{M}", kind, d=d, sigma=kw.pop("sigma", 1.0),
                      T=kw.pop("T", 0.5), N=N, M=M, Q=Q, seed=seed, x0_law="normal_1/d",
                      precision=prec, cg_tol=1e-13 if prec == "fp64" else 1e-7,
                      cg_max_iter=2000, **kw)


def _few_particles(d, M):
    """With M < d the regression has rank M - 1 and the default ridge (1e-3 of the mean
    eigenvalue) leaves a condition number near 1e-3 * M / d below one, far beyond what
    FP32 data resolve to 1e-4.  These cases test the kernels at wide rows, so they use
    a ridge of the mean eigenvalue (condition number about d / M)."""
    return {"ridge_rel": 1.0} if M < d else {}


def _check(w, queries=None):
    inp = W.inputs(w)
    out = gpu_solver(w, theta=inp["theta"]).solve(torch.tensor(inp["x0"], device="cuda"),
                                                  seed=w.seed)
    torch.cuda.synchronize()
    assert out["status"] == 0
    tol = TOL_FP64 if w.precision == "fp64" else TOL_FP32
    for q in (queries if queries is not None else range(w.Q)):
        ref = oracle.solve(oracle_problem(w, theta=inp["theta"]), inp["x0"][q], w.seed, q)
        assert ref["status"] == 0
        ru, rg = rel_errors(float(out["u0"][q]), out["grad"][q].cpu().numpy(), ref)
        assert ru <= tol, (q, ru)
        assert rg <= tol, (q, rg)


SHAPES = [
    ("ac_manufactured", 1, 2, 1, 1),
    ("ac_manufactured", 1, 37, 3, 3),
    ("cos_linear_test", 3, 9, 2, 5),
    ("ac_manufactured", 4096, 48, 2, 1),     # FP64: 2048 row chunks, 8-warp team
    ("ac_manufactured", 10240, 48, 2, 1),    # FP32: 2560 row chunks, one 10-warp team;
                                             # FP64: 5120 chunks, 10 warps of 16 chunks
    ("ac_manufactured", 10241, 48, 2, 1),    # FP32: 2561 chunks, 11-warp team (544 threads)
]


# every shape in both precisions, except FP64 rows beyond its limit of 10240 values (the
# library rejects those; tests/test_abi_cpu.py checks it)
EDGE_CASES = [(*shape, prec) for shape in SHAPES for prec in ("fp32", "fp64")
              if not (prec == "fp64" and shape[1] > 10240)]


@pytest.mark.parametrize("kind,d,M,N,Q,prec", EDGE_CASES)
def test_edge_shapes_match_oracle(kind, d, M, N, Q, prec):
    extra = {"c1": 0.3} if kind == "cos_linear_test" else {}
    _check(_w(kind, d, M, N, Q, prec, **_few_particles(d, M), **extra))


def test_more_queries_than_ctas():
    """700 queries of a tiny problem: one CTA per query and streaming pass."""
    _check(_w("ac_manufactured", 5, 16, 2, 700, "fp32"), queries=[0, 1, 350, 699])


@pytest.mark.parametrize("prec,d", [("fp32", 16384), ("fp64", 8192), ("fp64", 10240)])
def test_largest_dimension(prec, d):
    _check(_w("ac_manufactured", d, 40, 2, 1, prec, **_few_particles(d, 40)))


def test_dimension_beyond_the_limit_is_rejected():
    from paper_2510_02635_gb300 import fbsde
    fbsde.load_library()
    for prec, d in (("fp32", 16385), ("fp64", 10241)):
        p = fbsde.make_problem("ac_manufactured", d, 2, 40, 1.0, 0.5, prec)
        assert fbsde.fbsde_workspace_bytes(p, 1) == 0
