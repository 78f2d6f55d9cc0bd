"""The eager entry point launches a CG loop in three ways: every pass in a cached CUDA
graph (default), the first FBSDE_PROFILED_EAGER_PASSES passes one by one while the
profiler times the product kernel, and every pass one by one on a stream that is being
captured.  All three give the same bits, solve after solve, and the same bits as a plan."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(fb, kind, d, M, N, Q, prec, seed, cg_max_iter=120):
    rng = np.random.default_rng(seed)
    sigma, T = (1.0, 0.5) if kind == "ac_manufactured" else (float(d), 1.0)
    p = fb.make_problem(kind, d, N, M, sigma, T, prec,
                        cg_tol=1e-12 if prec == "fp64" else 1e-6, cg_max_iter=cg_max_iter)
    x0 = torch.tensor(rng.standard_normal((Q, d)) / math.sqrt(d), device="cuda")
    ws = torch.empty(fb.fbsde_workspace_bytes(p, Q), dtype=torch.uint8, device="cuda")
    return p, x0, ws


def _solve(fb, p, Q, x0, ws, seed, stream=None):
    u = torch.empty(Q, dtype=torch.float64, device="cuda")
    g = torch.empty(Q, p.d, dtype=torch.float64, device="cuda")
    fb.check(fb.fbsde_solve(p, Q, x0, seed, 0, u, g, ws, stream=stream))
    return u, g


CASES = [("ac_manufactured", 300, 1200, 6, 3, "fp32", 1),
         ("logistic_grad", 150, 700, 5, 2, "fp64", 2),
         # d close to M: ill-conditioned regressions needing more than the eager passes
         ("ac_manufactured", 900, 1000, 4, 2, "fp32", 3)]


@pytest.mark.parametrize("case", CASES)
def test_profiled_and_graph_tail_solves_agree_bitwise(case):
    from paper_2510_02635_gb300 import fbsde as fb
    kind, d, M, N, Q, prec, seed = case
    p, x0, ws = _setup(fb, kind, d, M, N, Q, prec, seed, cg_max_iter=300)
    u0, g0 = _solve(fb, p, Q, x0, ws, seed)           # every pass in the cached graph
    u1, g1 = _solve(fb, p, Q, x0, ws, seed)           # cache hit
    fb.fbsde_profile_start(1 << 16)
    fb.fbsde_profile_select(["matvec"])
    u2, g2 = _solve(fb, p, Q, x0, ws, seed)           # 48 eager passes + graph tail
    torch.cuda.synchronize()
    prof = fb.fbsde_profile_stop()
    assert prof["matvec"]["launches"] == N * fb.FBSDE_PROFILED_EAGER_PASSES
    assert prof["matvec"]["timed"] == prof["matvec"]["launches"]
    # the FP32 path steps each level with the fused kernel (N launches with the forward
    # sweep's end point), the FP64 path with the row-segment update (N - 1 launches)
    fam, n_step = ("step", N) if prec == "fp32" else ("update", N - 1)
    assert prof[fam]["timed"] == 0 and prof[fam]["launches"] == n_step
    for u, g in ((u1, g1), (u2, g2)):
        assert torch.equal(u, u0) and torch.equal(g, g0)
    assert fb.fbsde_diagnostics(p, Q, ws).status == 0


def test_capture_by_the_caller_replays_the_same_bits():
    from paper_2510_02635_gb300 import fbsde as fb
    kind, d, M, N, Q, prec, seed = CASES[0]
    p, x0, ws = _setup(fb, kind, d, M, N, Q, prec, seed, cg_max_iter=60)
    ref_u, ref_g = _solve(fb, p, Q, x0, ws, seed)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    u = torch.empty(Q, dtype=torch.float64, device="cuda")
    g = torch.empty(Q, d, dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
        fb.check(fb.fbsde_solve(p, Q, x0, seed, 0, u, g, ws,
                                stream=torch.cuda.current_stream()))
    for _ in range(2):
        u.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(u, ref_u) and torch.equal(g, ref_g)


def test_graph_tail_and_plan_agree_bitwise():
    from paper_2510_02635_gb300 import fbsde as fb
    kind, d, M, N, Q, prec, seed = CASES[2]
    p, x0, ws = _setup(fb, kind, d, M, N, Q, prec, seed, cg_max_iter=300)
    u0, g0 = _solve(fb, p, Q, x0, ws, seed)
    plan = fb.Plan([{"problem": p, "Q": Q, "x0": x0, "seed": seed, "solve_index0": 0}])
    plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(plan.u0[0], u0) and torch.equal(plan.grad[0], g0)
    plan.close()
