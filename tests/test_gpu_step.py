"""The fused per-level step of the FP32 path (one pass over the particle rows: reverse
step, prediction, Newton, weights, moments) against the FP64 oracle, for every geometry
of the kernel: R = 30, 15, 5, 3 and 1 rows per stage, teams of 16 to 480 threads per
row, 1 to 6 chunks of 16 bytes per thread, the column pass in row groups (rows narrower
than 480 chunks) or over whole rows, its sixth chunk in shared memory (rows wider than
9600 floats), ragged d (padding inside the last chunk) and ragged M (stages and CTAs
with fewer rows than R).  The u / grad u bar is the FP32 path's 1e-4."""
import math

import pytest

import oracle
from helpers import TOL_FP32, gpu_solver, oracle_problem, rel_errors
from paper_2510_02635_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _geometry(d):
    """Rows per stage R, threads per row T, chunks per thread VM, column-pass row groups
    RG and chunks vm3, as the library chooses them (host layout)."""
    ld = (d + 3) // 4 * 4
    nch = ld // 4
    R = max(r for r in (1, 3, 5, 15, 30) if r == 1 or r * ld <= 10240)
    T = 480 // R
    tpr = min(480, nch)
    return R, T, -(-nch // T), 480 // tpr, -(-nch // tpr)


# (kind, d, M, N, Q, extra); comments give (R, T, VM, RG, vm3)
CASES = [
    ("ac_manufactured", 1, 61, 3, 2, {}),              # (30, 16, 1, 480, 1)
    ("logistic_grad", 37, 303, 4, 2, {"sigma": 37.0, "T": 1.0}),   # (30, 16, 1, 48, 1)
    ("ac_manufactured", 333, 517, 3, 2, {}),           # (30, 16, 6, 5, 1)
    ("hjb_logquad", 700, 640, 3, 1, {"sigma": math.sqrt(2.0), "T": 1.0,
                                     "theta_law": "uniform_0.5_1.5"}),   # (5, 96, 2, 2, 1)
    ("ac_doublewell", 1501, 1203, 3, 1, {"sigma": math.sqrt(2.0), "T": 0.3}),  # (5, 96, 4, 1, 1)
    ("cos_linear_test", 2500, 777, 3, 1, {"c1": 0.3}),  # (3, 160, 4, 1, 2)
    ("ac_manufactured", 3999, 900, 3, 1, {}),          # (1, 480, 3, 1, 3)
    ("ac_manufactured", 9701, 450, 2, 1, {}),          # (1, 480, 6, 1, 6): shared tail
    ("logistic_grad", 10240, 400, 2, 1, {"sigma": 10240.0, "T": 1.0}),  # (1, 480, 6, 1, 6)
]


@pytest.mark.parametrize("kind,d,M,N,Q,extra", CASES)
def test_fused_step_matches_oracle(kind, d, M, N, Q, extra):
    extra = dict(extra)
    sigma, T = extra.pop("sigma", 1.0), extra.pop("T", 0.5)
    ridge = {"ridge_rel": 1.0} if M < d else {}   # M < d: keep the regression conditioned
    w = W.Workload(f"step_{kind}_{d}", kind, d=d, sigma=sigma, T=T, N=N, M=M, Q=Q, seed=13,
                   x0_law="normal_1/d", precision="fp32", cg_tol=1e-7, cg_max_iter=2000,
                   **ridge, **extra)
    inp = W.inputs(w)
    out = gpu_solver(w, theta=inp["theta"]).solve(torch.tensor(inp["x0"], device="cuda"),
                                                  seed=w.seed)
    torch.cuda.synchronize()
    assert out["status"] == 0
    for q in range(Q):
        ref = oracle.solve(oracle_problem(w, theta=inp["theta"]), inp["x0"][q], w.seed, q)
        assert ref["status"] == 0
        ru, rg = rel_errors(float(out["u0"][q]), out["grad"][q].cpu().numpy(), ref)
        assert ru <= TOL_FP32, (_geometry(d), q, ru)
        assert rg <= TOL_FP32, (_geometry(d), q, rg)


def test_case_geometries_are_the_intended_ones():
    got = [_geometry(c[1]) for c in CASES]
    assert got == [(30, 16, 1, 480, 1), (30, 16, 1, 48, 1), (30, 16, 6, 5, 1), (5, 96, 2, 2, 1),
                   (5, 96, 4, 1, 1), (3, 160, 4, 1, 2), (1, 480, 3, 1, 3), (1, 480, 6, 1, 6),
                   (1, 480, 6, 1, 6)]
