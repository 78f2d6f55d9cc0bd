"""CUDA path of the scheme with a drift and a state-dependent diffusion (the forward SDE of
Sec. 2.1 with mu_i(x) = mu0 + mu1 x_i and sigma(x) = diag(sigma + sig1 x_i): Euler-Maruyama
paths (2.7), regressions anchored on the drift path of x0, Z = sigma(X)^T alpha_x per
particle) against the FP64 oracle of the same scheme, on identical seeded inputs.

FP64 path: the end point of the paths, Y_N, every level's alpha and alpha_x, u(0,x0) and
grad u(0,x0) within 1e-10.  FP32 path: u within 1e-4 relative, grad within
1e-4 max(|grad u|, |u|).  The cases span ragged d and M, several row teams (d > 1024),
every kind of the problem table, N = 1 and N = 2 (no stored level, one segment slot),
N = 9, 10, 17 (checkpoints at s, 2s, .. with s = ceil(sqrt N); segments recomputed on the
way back), and rows of 10^4 and 10240 values."""
import math

import numpy as np
import pytest

import oracle
from helpers import TOL_FP32, TOL_FP64, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _theta(kind, d):
    if kind not in ("hjb_logquad", "affine_test"):
        return None
    return np.random.default_rng(17).uniform(0.5, 1.5, size=d)


def _x0(d, Q, seed):
    return np.random.default_rng(seed).standard_normal((Q, d)) / math.sqrt(d)


# kind, d, M, N, sigma, T, (mu0, mu1, sig1), problem extras
CASES = [
    ("drift_ac", 37, 300, 4, 0.7, 0.6, (0.2, -0.6, 0.3), {}),
    ("drift_quad", 130, 257, 9, 0.5, 0.5, (0.1, 0.4, -0.2), {}),
    ("drift_ac", 1500, 600, 5, 0.8, 0.5, (0.0, -0.8, 0.2), {}),
    ("affine_test", 6, 80, 10, 0.3, 0.8, (0.2, -0.4, 0.25),
     {"A": 0.3, "c0": 0.2, "c1": -0.5, "c2": 0.35, "c3": -0.4, "h": 1.5}),
    ("logistic_grad", 33, 257, 4, 2.0, 1.0, (0.0, -0.5, 0.5), {}),
    ("hjb_logquad", 61, 400, 4, math.sqrt(2.0), 1.0, (0.3, -0.2, 0.0), {}),
    ("ac_manufactured", 50, 333, 3, 1.0, 0.5, (0.3, 0.0, 0.2), {}),
    ("ac_doublewell", 20, 290, 2, math.sqrt(2.0), 0.3, (0.1, -0.3, 0.1), {}),
    ("cos_linear_test", 29, 211, 1, 1.0, 0.4, (0.1, 0.2, 0.1), {"c1": 0.4}),
    ("cubic_test", 24, 230, 3, 1.0, 0.3, (0.1, -0.2, 0.1), {"A": 0.5}),
    ("drift_quad", 12, 500, 17, 0.6, 0.5, (-0.2, -1.0, 0.3), {}),
    # wide rows (several warps per row segment walk; FP64 at its largest d): with M < d the
    # regression has rank M - 1, so the ridge is the mean eigenvalue (condition ~ d / M)
    ("drift_ac", 10000, 160, 3, 0.5, 0.5, (0.1, -0.5, 0.2), {"ridge_rel": 1.0}),
    ("drift_quad", 10240, 120, 2, 0.4, 0.5, (0.0, -0.3, 0.1), {"ridge_rel": 1.0}),
]


def _run(case, prec, Q=2, seed=5, trace=True):
    from paper_2510_02635_gb300 import fbsde as fb
    kind, d, M, N, sigma, T, (mu0, mu1, sig1), extra = case
    theta = _theta(kind, d)
    x0 = _x0(d, Q, seed + d)
    kw = dict(ridge_rel=1e-3, h=2.0)
    kw.update(extra)
    solver = fb.Solver(kind, d, N, M, sigma, T, Q=Q, precision=prec, theta=theta,
                       cg_tol=1e-13 if prec == "fp64" else 1e-7, cg_max_iter=400,
                       mu0=mu0, mu1=mu1, sig1=sig1, **kw)
    out = solver.solve(torch.tensor(x0, device="cuda"), seed=seed, trace=trace,
                       trace_forward=trace)
    torch.cuda.synchronize()
    prob = oracle.Problem(kind, d, sigma, T, N, M, theta=theta, cg_tol=1e-13, **kw)
    refs = [oracle.solve_sde(prob, x0[q], seed, q, mu0=mu0, mu1=mu1, sig1=sig1, trace=trace,
                             keep_paths=trace) for q in range(Q)]
    return out, refs, x0, prob


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-d{c[1]}-N{c[3]}" for c in CASES])
def test_fp64_drift_path_matches_oracle_at_every_level(case):
    out, refs, x0, prob = _run(case, "fp64")
    N = prob.N
    assert out["status"] == 0
    for q, ref in enumerate(refs):
        assert ref["status"] == 0
        XN = ref["paths"][N]
        xN = out["x_N"][q].cpu().numpy()
        assert np.max(np.abs(xN - (XN - x0[q]))) <= 1e-12 * (1 + np.max(np.abs(xN)))
        yN = np.array([oracle.sde_g(prob, XN[j]) for j in range(prob.M)])
        assert np.max(np.abs(out["y_N"][q].cpu().numpy() - yN)) <= 1e-12 * (1 + np.max(np.abs(yN)))
        a = out["alpha"][q].cpu().numpy()
        ax = out["alpha_x"][q].cpu().numpy()
        for k in range(N):
            assert abs(a[k] - ref["alpha"][k]) <= TOL_FP64 * max(1.0, abs(ref["alpha"][k])), k
            scale = max(np.linalg.norm(ref["alpha_x"][k]), 1.0)
            assert np.linalg.norm(ax[k] - ref["alpha_x"][k]) <= TOL_FP64 * scale, k
        ru, rg = rel_errors(float(out["u0"][q]), out["grad"][q].cpu().numpy(), ref)
        assert ru <= TOL_FP64 and rg <= TOL_FP64, (ru, rg)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-d{c[1]}-N{c[3]}" for c in CASES])
def test_fp32_drift_path_matches_oracle(case):
    out, refs, _, _ = _run(case, "fp32", trace=False)
    assert out["status"] == 0
    for q, ref in enumerate(refs):
        ru, rg = rel_errors(float(out["u0"][q]), out["grad"][q].cpu().numpy(), ref)
        assert ru <= TOL_FP32 and rg <= TOL_FP32, (q, ru, rg)


def test_drift_kind_without_drift_runs_euler_maruyama_paths():
    """Kind DRIFT_AC with mu = 0 and sig1 = 0 still takes the Euler-Maruyama path (its
    increments are the normals of levels 0..N-1, not the Brownian bridge's), and equals the
    oracle of that scheme."""
    case = ("drift_ac", 40, 400, 5, 0.9, 0.5, (0.0, 0.0, 0.0), {})
    out, refs, _, _ = _run(case, "fp64", trace=False)
    for q, ref in enumerate(refs):
        ru, rg = rel_errors(float(out["u0"][q]), out["grad"][q].cpu().numpy(), ref)
        assert ru <= TOL_FP64 and rg <= TOL_FP64


def test_drift_solve_is_deterministic_and_graph_modes_agree():
    """Two solves, an eager solve with the launch profiler on, and a plan replay give the
    same bits (the stored levels and the recomputed segments are rewritten every solve)."""
    from paper_2510_02635_gb300 import fbsde as fb
    d, N, M, Q, seed = 70, 10, 700, 2, 9
    p = fb.make_problem("drift_quad", d, N, M, 0.6, 0.5, "fp32", cg_tol=1e-7, cg_max_iter=200,
                        mu0=0.1, mu1=-0.5, sig1=0.2)
    x0 = torch.tensor(_x0(d, Q, 3), device="cuda")
    ws = torch.empty(fb.fbsde_workspace_bytes(p, Q), dtype=torch.uint8, device="cuda")
    outs = []
    for prof in (False, False, True):
        u = torch.empty(Q, dtype=torch.float64, device="cuda")
        g = torch.empty(Q, d, dtype=torch.float64, device="cuda")
        if prof:
            fb.fbsde_profile_start(1 << 12)
            fb.fbsde_profile_select(["matvec"])
        fb.check(fb.fbsde_solve(p, Q, x0, seed, 0, u, g, ws))
        torch.cuda.synchronize()
        if prof:
            st = fb.fbsde_profile_stop()
            # forward sweep N steps, then one recompute of every segment but the last
            sq = math.ceil(math.sqrt(N))
            n_seg = (N - 1) // sq   # segments below the last one
            recompute = sum(min(b + sq, N) - b - 1 for b in range(0, n_seg * sq, sq))
            assert st["forward"]["launches"] == N + recompute
            assert st["update"]["launches"] == N
            assert st["step"]["launches"] == 0
        outs.append((u.cpu(), g.cpu()))
    for u, g in outs[1:]:
        assert torch.equal(u, outs[0][0]) and torch.equal(g, outs[0][1])
    plan = fb.Plan([{"problem": p, "Q": Q, "x0": x0, "seed": seed}])
    plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(plan.u0[0].cpu(), outs[0][0])
    assert torch.equal(plan.grad[0].cpu(), outs[0][1])
    plan.close()


def test_drift_kind_error_against_the_closed_form_is_first_order_in_dt():
    """u*(0,x0) = e^{-T} (1/d) sum cos x0_i of DRIFT_AC under an Ornstein-Uhlenbeck drift with
    a state-dependent diffusion, d = 100, M = 4096: the FP32 GPU solve's error falls about
    fourfold from N = 5 to N = 20 (the O(dt) of Theorem 3.1; the oracle at these sizes and
    seeds gives 0.0187 and 0.0050)."""
    from paper_2510_02635_gb300 import fbsde as fb
    d, M, Q, T = 100, 4096, 4, 0.6
    x0 = _x0(d, Q, 21)
    u_star = math.exp(-T) * np.mean(np.cos(x0), axis=1)
    err = {}
    for N in (5, 20):
        solver = fb.Solver("drift_ac", d, N, M, 0.5, T, Q=Q, precision="fp32", cg_tol=1e-7,
                           mu0=0.1, mu1=-0.8, sig1=0.2)
        out = solver.solve(torch.tensor(x0, device="cuda"), seed=4)
        torch.cuda.synchronize()
        assert out["status"] == 0
        err[N] = np.abs(out["u0"].cpu().numpy() - u_star)
    assert np.max(err[5]) < 0.03 and np.max(err[20]) < 0.4 * np.min(err[5]), err


def test_drift_problems_rejected_where_the_scheme_is_driftless():
    from paper_2510_02635_gb300 import fbsde as fb
    d, N, M, Q = 16, 3, 200, 1
    p = fb.make_problem("ac_manufactured", d, N, M, 1.0, 0.5, "fp64", mu1=-0.3)
    x0 = torch.zeros(Q, d, dtype=torch.float64, device="cuda")
    u = torch.empty(Q, dtype=torch.float64, device="cuda")
    g = torch.empty(Q, d, dtype=torch.float64, device="cuda")
    xb = torch.empty(Q, d, dtype=torch.float64, device="cuda")
    ub = torch.ones(Q, dtype=torch.float64, device="cuda")
    ws = torch.empty(fb.fbsde_adjoint_workspace_bytes(p, Q) + 256, dtype=torch.uint8,
                     device="cuda")
    assert fb.fbsde_adjoint(p, Q, x0, 1, 0, ub, u, g, xb, None, ws) == fb.FBSDE_ERR_ARG
    assert fb.fbsde_anchored_workspace_bytes(p) == 0
