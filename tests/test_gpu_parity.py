"""CUDA path vs the FP64 oracle, element by element, on identical seeded inputs.

FP64 path: every per-level quantity within 1e-10 (relative).  FP32 path: u(0,x0)
within 1e-4 relative and grad u(0,x0) within 1e-4 max(|grad u|, |u|), the bar of
the method's precision pattern (FP32 streams, FP64 regression combination and
Newton).  Cases span several CTAs and teams, ragged d (not a multiple of the
16-byte chunk), ragged M (not a multiple of the CTA row split) and every kind.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import TOL_FP32, TOL_FP64, gpu_solver, oracle_problem, rel_errors
from paper_2510_02635_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _w(kind, d, M, N, Q=1, prec="fp64", sigma=1.0, T=0.5, seed=3, **kw):
    return W.Workload(f"t_{kind}_{d}", kind, d=d, sigma=sigma, T=T, N=N, M=M, Q=Q, seed=seed,
                      x0_law="normal_1/d", precision=prec,
                      cg_tol=1e-13 if prec == "fp64" else 1e-7, cg_max_iter=400, **kw)


def _run_both(w, theta=None, trace=True, queries=None, solve_index0=0):
    inp = W.inputs(w)
    x0 = inp["x0"]
    th = theta if theta is not None else inp["theta"]
    solver = gpu_solver(w, theta=th)
    out = solver.solve(torch.tensor(x0, device="cuda"), seed=w.seed,
                       solve_index0=solve_index0, trace=trace, trace_forward=trace)
    torch.cuda.synchronize()
    refs = []
    for q in (queries if queries is not None else range(w.Q)):
        refs.append((q, oracle.solve(oracle_problem(w, theta=th), x0[q], w.seed,
                                     solve_index0 + q, trace=trace, keep_forward=trace)))
    return out, refs


CASES = [
    ("ac_manufactured", 37, 300, 4, {}),
    ("ac_manufactured", 100, 2048, 5, {}),
    ("logistic_grad", 33, 257, 4, {"sigma": 33.0, "T": 1.0}),
    ("hjb_logquad", 61, 400, 4, {"sigma": math.sqrt(2.0), "T": 1.0,
                                 "theta_law": "uniform_0.5_1.5"}),
    ("ac_doublewell", 50, 333, 4, {"sigma": math.sqrt(2.0), "T": 0.3}),
    ("cos_linear_test", 29, 211, 3, {"c1": 0.4}),
    ("ac_manufactured", 1500, 1200, 3, {}),   # multi-warp teams (d > 1024 floats)
]


@pytest.mark.parametrize("kind,d,M,N,extra", CASES)
def test_fp64_path_matches_oracle_at_every_level(kind, d, M, N, extra):
    w = _w(kind, d, M, N, Q=2, prec="fp64", **extra)
    out, refs = _run_both(w)
    assert out["status"] == 0
    for q, ref in refs:
        assert ref["status"] == 0
        xN = out["x_N"][q].cpu().numpy()
        x0 = W.inputs(w)["x0"][q]
        assert np.max(np.abs(xN - (ref["X_N"] - x0))) <= 1e-12 * (1 + np.max(np.abs(xN)))
        assert np.max(np.abs(out["y_N"][q].cpu().numpy() - ref["Y_N"])) <= 1e-12
        a = out["alpha"][q].cpu().numpy()
        ax = out["alpha_x"][q].cpu().numpy()
        for k in range(N):
            assert abs(a[k] - ref["alpha"][k]) <= TOL_FP64 * max(1.0, abs(ref["alpha"][k]))
            scale = max(np.linalg.norm(ref["alpha_x"][k]), 1.0)
            assert np.linalg.norm(ax[k] - ref["alpha_x"][k]) <= TOL_FP64 * scale, k
        ru, rg = rel_errors(float(out["u0"][q]), out["grad"][q].cpu().numpy(), ref)
        assert ru <= TOL_FP64 and rg <= TOL_FP64


@pytest.mark.parametrize("kind,d,M,N,extra", CASES)
def test_fp32_path_matches_oracle(kind, d, M, N, extra):
    w = _w(kind, d, M, N, Q=2, prec="fp32", **extra)
    out, refs = _run_both(w, trace=False)
    assert out["status"] == 0
    for q, ref in refs:
        ru, rg = rel_errors(float(out["u0"][q]), out["grad"][q].cpu().numpy(), ref)
        assert ru <= TOL_FP32, ru
        assert rg <= TOL_FP32, rg


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_affine_problem_exact_on_gpu(prec):
    """g = A + theta.x, f = c0 + c1 y + c2 sum z + c3 t: closed recursion of the scheme."""
    d, N, M, sigma, T = 24, 6, 256, 0.9, 0.8
    c0, c1, c2, c3, A = 0.2, -0.7, 0.35, -0.6, -0.4
    rng = np.random.default_rng(21)
    theta = rng.normal(size=d)
    x0 = rng.normal(scale=0.5, size=d)
    w = W.Workload("affine", "affine_test", d=d, sigma=sigma, T=T, N=N, M=M, Q=1, seed=9,
                   x0_law="zero", precision=prec, ridge_rel=0.0, A=A, c0=c0, c1=c1,
                   cg_tol=1e-13 if prec == "fp64" else 1e-8, cg_max_iter=200,
                   extra={"c2": c2, "c3": c3})
    solver = gpu_solver(w, theta=theta)
    out = solver.solve(torch.tensor(x0[None], device="cuda"), seed=9)
    dt = T / N
    a, b = A + theta @ x0, theta.copy()
    for k in range(N - 1, -1, -1):
        a, b = (a + dt * (c0 + c2 * sigma * b.sum() + c3 * k * dt)) / (1 - dt * c1), \
            b / (1 - dt * c1)
    tol = 1e-11 if prec == "fp64" else 2e-5
    assert out["status"] == 0
    assert abs(float(out["u0"][0]) - a) <= tol * max(1, abs(a))
    grad_ref = theta / (1 - dt * c1) ** (N - 1)
    assert np.max(np.abs(out["grad"][0].cpu().numpy() - grad_ref)) <= tol * np.max(np.abs(grad_ref))


def test_config0_plain_scheme_fp64():
    """Allen-Cahn with manufactured source, d = 100, M = 2048, N = 10, x0 = 0, FP64."""
    w = W.C0_AC_D100
    out, refs = _run_both(w, trace=False)
    assert out["status"] == 0
    ru, rg = rel_errors(float(out["u0"][0]), out["grad"][0].cpu().numpy(), refs[0][1])
    assert ru <= TOL_FP64 and rg <= TOL_FP64


def test_solve_index_offsets_the_stream():
    w = _w("ac_manufactured", 40, 256, 3, Q=2, prec="fp64")
    out, refs = _run_both(w, trace=False, solve_index0=1000)
    for q, ref in refs:
        ru, _ = rel_errors(float(out["u0"][q]), out["grad"][q].cpu().numpy(), ref)
        assert ru <= TOL_FP64


def test_deterministic_bits():
    w = _w("ac_manufactured", 300, 1000, 4, Q=3, prec="fp32")
    x0 = torch.tensor(W.inputs(w)["x0"], device="cuda")
    solver = gpu_solver(w)
    a = solver.solve(x0, seed=5)
    b = solver.solve(x0, seed=5)
    assert torch.equal(a["u0"], b["u0"]) and torch.equal(a["grad"], b["grad"])


def test_host_buffer_entry_point_matches_device_entry_point():
    from paper_2510_02635_gb300 import fbsde
    w = _w("hjb_logquad", 64, 512, 4, Q=2, prec="fp32", sigma=math.sqrt(2.0), T=1.0,
           theta_law="uniform_0.5_1.5")
    inp = W.inputs(w)
    solver = gpu_solver(w, theta=inp["theta"])
    dev = solver.solve(torch.tensor(inp["x0"], device="cuda"), seed=w.seed)
    p = fbsde.make_problem(w.kind, w.d, w.N, w.M, w.sigma, w.T, w.precision,
                           theta=np.ascontiguousarray(inp["theta"]), cg_tol=w.cg_tol,
                           cg_max_iter=w.cg_max_iter)
    nbytes = fbsde.fbsde_workspace_bytes(p, w.Q) + fbsde.fbsde_host_staging_bytes(p, w.Q)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    u0 = np.zeros(w.Q)
    g = np.zeros((w.Q, w.d))
    st = fbsde.fbsde_solve_host(p, w.Q, np.ascontiguousarray(inp["x0"]), w.seed, 0, u0, g, ws)
    assert st == 0
    assert np.array_equal(u0, dev["u0"].cpu().numpy())
    assert np.array_equal(g, dev["grad"].cpu().numpy())


def test_device_status_reports_cg_and_newton_exhaustion():
    w = _w("ac_manufactured", 80, 500, 3, Q=1, prec="fp64")
    x0 = torch.tensor(W.inputs(w)["x0"], device="cuda")
    out = gpu_solver(w, cg_max_iter=1).solve(x0, seed=1)
    assert out["status"] == 5 and out["solves_cg_exhausted"] == 1
    out = gpu_solver(w, newton_max_iter=1).solve(x0, seed=1)
    assert out["status"] == 4
    out = gpu_solver(w).solve(x0, seed=1)
    assert out["status"] == 0 and out["max_newton_iters"] >= 2
