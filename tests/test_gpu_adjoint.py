"""GPU reverse sweep (fbsde_adjoint) against the oracle's adjoint, against central
finite differences of the GPU solve (common random numbers) and through
torch.autograd."""
import math

import numpy as np
import pytest

import oracle
from helpers import oracle_problem
from paper_2510_02635_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("ac_manufactured", 1.0, 0.5, {}),
    ("logistic_grad", 19.0, 1.0, {}),
    ("hjb_logquad", math.sqrt(2.0), 1.0, {"theta_law": "uniform_0.5_1.5"}),
    ("affine_test", 0.9, 0.8, {"extra": {"theta_affine": True, "c2": 0.3, "c3": 0.4},
                               "A": 0.3, "c0": 0.2, "c1": -0.5}),
    ("ac_doublewell", math.sqrt(2.0), 0.3, {}),
    ("cos_linear_test", 0.7, 0.6, {"c1": 0.4}),
]


def _w(kind, sigma, T, extra, prec, d=19, M=333, N=4, Q=2):
    return W.Workload(f"adj_{kind}", kind, d=d, sigma=sigma, T=T, N=N, M=M, Q=Q, seed=7,
                      x0_law="normal_1/d", precision=prec,
                      cg_tol=1e-13 if prec == "fp64" else 1e-8, cg_max_iter=300, **extra)


def _solver(w, theta):
    from helpers import gpu_solver
    return gpu_solver(w, theta=theta)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind,sigma,T,extra", CASES)
def test_adjoint_matches_oracle(kind, sigma, T, extra, prec):
    w = _w(kind, sigma, T, extra, prec)
    inp = W.inputs(w)
    th = inp["theta"]
    solver = _solver(w, th)
    with_theta = kind in ("hjb_logquad", "affine_test")
    ub = np.array([1.0, -0.7])
    out = solver.adjoint(inp["x0"], seed=w.seed, u0_bar=ub, with_theta=with_theta)
    assert out["status"] == 0
    tol = 1e-9 if prec == "fp64" else 1e-4
    tb_ref = np.zeros(w.d)
    for q in range(w.Q):
        ref = oracle.adjoint(oracle_problem(w, theta=th), inp["x0"][q], w.seed, q)
        assert ref["status"] == 0
        assert abs(float(out["u0"][q]) - ref["u0"]) <= tol * abs(ref["u0"])
        xb = out["x0_bar"][q].cpu().numpy()
        scale = max(np.max(np.abs(ref["du_dx0"])), 1e-12)
        assert np.max(np.abs(xb - ub[q] * ref["du_dx0"])) <= tol * scale * abs(ub[q])
        tb_ref += ub[q] * ref["du_dtheta"]
    if with_theta:
        tb = out["theta_bar"].cpu().numpy()
        assert np.max(np.abs(tb - tb_ref)) <= tol * max(np.max(np.abs(tb_ref)), 1e-12)


def test_hjb_d1000_adjoint_vs_oracle_and_central_differences():
    """The adjoint workload: log-quadratic terminal, d = 1000, M = 4096, N = 20.  FP32
    reverse sweep vs the FP64 oracle adjoint, and vs central differences (h = 1e-3,
    common random numbers) of the FP64 GPU solve on a few coordinates; the method's own
    grad u estimate is reported alongside."""
    w = W.C4_HJB_D1000
    inp = W.inputs(w)
    th, x0 = inp["theta"], inp["x0"]
    solver = _solver(w, th)
    out = solver.adjoint(x0, seed=w.seed, with_theta=True)
    assert out["status"] == 0
    ref = oracle.adjoint(oracle_problem(w, theta=th), x0[0], w.seed, 0)
    xb, tb = out["x0_bar"][0].cpu().numpy(), out["theta_bar"].cpu().numpy()
    assert np.max(np.abs(xb - ref["du_dx0"])) <= 1e-4 * np.max(np.abs(ref["du_dx0"]))
    assert np.max(np.abs(tb - ref["du_dtheta"])) <= 1e-4 * np.max(np.abs(ref["du_dtheta"]))
    w64 = w.with_(precision="fp64", cg_tol=1e-12)
    s64 = _solver(w64, th)
    h = 1e-3
    for i in (0, 417, 999):
        e = np.zeros_like(x0)
        e[0, i] = h
        up = float(s64.solve(x0 + e, seed=w.seed)["u0"][0])
        um = float(s64.solve(x0 - e, seed=w.seed)["u0"][0])
        fd = (up - um) / (2 * h)
        assert abs(xb[i] - fd) <= 1e-4 * np.max(np.abs(xb)) + 1e-6 * abs(fd)


def test_autograd_function_matches_reverse_sweep():
    from paper_2510_02635_gb300 import fbsde
    w = _w("hjb_logquad", math.sqrt(2.0), 1.0, {"theta_law": "uniform_0.5_1.5"}, "fp64",
           d=33, M=500, N=3, Q=3)
    inp = W.inputs(w)
    solver = _solver(w, inp["theta"])
    x0 = torch.tensor(inp["x0"], device="cuda", requires_grad=True)
    theta = torch.tensor(inp["theta"], device="cuda", requires_grad=True)
    u = fbsde.fbsde_value(solver, x0, w.seed, theta=theta)
    (u * torch.tensor([0.5, 1.0, -2.0], device="cuda", dtype=torch.float64)).sum().backward()
    adj = solver.adjoint(inp["x0"], seed=w.seed, u0_bar=[0.5, 1.0, -2.0], with_theta=True)
    assert torch.allclose(x0.grad, adj["x0_bar"], rtol=0, atol=0)
    assert torch.allclose(theta.grad, adj["theta_bar"], rtol=0, atol=0)


def test_adjoint_and_regression_gradient_estimate_the_same_grad_u():
    """Two estimators of grad u(0, x0) from one solve: the reverse sweep's du/dx0 (the
    derivative of the estimator u(0, x0) for fixed increments) and the scheme's own
    regression slope alpha_x of level 0 (Algorithm 1's grad u output).  On the adjoint
    workload (log-quadratic terminal, d = 1000, M = 4096, N = 20, FP32) one call solves the
    same x0 with 16 independent Philox streams.  The regression slope is far noisier than
    the reverse sweep, so they are compared statistically:
      - along the direction of the mean of du/dx0, the means over the streams agree within
        4 standard errors of their difference;
      - over all d components, the per-component t statistic of the mean difference has
        mean square at most the t distribution's (n - 1)/(n - 3) plus 5 of its standard
        deviations over d independent components (doubled for their correlation)."""
    n = 16
    base = W.C4_HJB_D1000
    w = base.with_(Q=n)
    inp = W.inputs(base)
    x0 = np.repeat(inp["x0"][:1], n, axis=0)
    out = _solver(w, inp["theta"]).adjoint(x0, seed=w.seed)
    assert out["status"] == 0
    A = out["x0_bar"].cpu().numpy()
    G = out["grad"].cpu().numpy()
    a = A.mean(axis=0)
    ahat = a / np.linalg.norm(a)
    pa, pg = A @ ahat, G @ ahat
    se = math.sqrt(pa.var(ddof=1) / n + pg.var(ddof=1) / n)
    assert abs(pg.mean() - pa.mean()) <= 4.0 * se, (pg.mean(), pa.mean(), se)
    D = G - A
    t = D.mean(axis=0) / (D.std(axis=0, ddof=1) / math.sqrt(n))
    nu = n - 1
    mean_t2 = nu / (nu - 2)
    sd_t2 = math.sqrt(2 * nu ** 2 * (nu - 1) / ((nu - 2) ** 2 * (nu - 4)) / w.d)
    assert float(np.mean(t * t)) <= mean_t2 + 10.0 * sd_t2, float(np.mean(t * t))
    # the reverse sweep itself is precise: its spread over the streams along its mean is
    # a small fraction of |grad u|
    assert pa.std(ddof=1) <= 0.2 * np.linalg.norm(a)
