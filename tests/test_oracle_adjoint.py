"""Pins of the oracle's adjoint (reverse-mode derivative of the estimator u(0,x0) of
Algorithm 1 with respect to x0 and theta, same random increments).

References that do not share its code path: central finite differences of the primal
oracle (common random numbers: same seed), numerical derivatives of the problem table,
and the closed form of the affine problem's discrete recursion.
"""
import math
import zlib

import numpy as np
import pytest

import oracle


def _fd_x0(p, x0, seed, h=1e-5, idx=None):
    idx = range(p.d) if idx is None else idx
    out = []
    for i in idx:
        e = np.zeros(p.d)
        e[i] = h
        out.append((oracle.solve(p, x0 + e, seed)["u0"] - oracle.solve(p, x0 - e, seed)["u0"])
                   / (2 * h))
    return np.array(out)


def _fd_theta(make, theta, x0, seed, h=1e-5):
    out = []
    for i in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        out.append((oracle.solve(make(tp), x0, seed)["u0"] - oracle.solve(make(tm), x0, seed)["u0"])
                   / (2 * h))
    return np.array(out)


CASES = [
    ("ac_manufactured", 1.0, 0.5, {}),
    ("logistic_grad", 7.0, 1.0, {}),
    ("hjb_logquad", math.sqrt(2.0), 1.0, {"theta": True}),
    ("affine_test", 0.9, 0.8, {"theta": True, "A": 0.3, "c0": 0.2, "c1": -0.5, "c2": 0.3, "c3": 0.4}),
    ("ac_doublewell", math.sqrt(2.0), 0.3, {}),
    ("cos_linear_test", 0.7, 0.6, {"c1": 0.4}),
    ("cubic_test", 1.0, 0.5, {"A": 0.6}),
]


@pytest.mark.parametrize("kind,sigma,T,extra", CASES)
def test_adjoint_matches_central_differences(kind, sigma, T, extra):
    rng = np.random.default_rng(zlib.crc32(kind.encode()))
    d, N, M, seed = 7, 4, 160, 11
    extra = dict(extra)
    theta = rng.uniform(0.5, 1.5, d) if extra.pop("theta", False) else None

    def make(th):
        return oracle.Problem(kind, d, sigma, T, N, M, theta=th, h=1.7, **extra)

    p = make(theta)
    x0 = rng.normal(scale=0.4, size=d)
    a = oracle.adjoint(p, x0, seed)
    assert a["status"] == 0
    assert a["u0"] == pytest.approx(oracle.solve(p, x0, seed)["u0"], rel=1e-12)
    fd = _fd_x0(p, x0, seed)
    scale = max(np.max(np.abs(fd)), 1e-3)
    assert np.max(np.abs(a["du_dx0"] - fd)) <= 1e-6 * scale
    if theta is not None:
        fdt = _fd_theta(make, theta, x0, seed)
        assert np.max(np.abs(a["du_dtheta"] - fdt)) <= 1e-6 * max(np.max(np.abs(fdt)), 1e-3)
    else:
        assert np.all(a["du_dtheta"] == 0.0)


def test_adjoint_of_affine_problem_closed_form():
    """g = A + theta.x, f = c0 + c1 y + c2 sum z + c3 t: u = a_0 with
    a_k = r (a_{k+1} + s_k), s_k = dt (c0 + c2 sigma sum b_{k+1} + c3 t_k),
    b_k = r b_{k+1}, a_N = A + theta.x0, b_N = theta, r = 1/(1 - dt c1).  Unrolled,
    a_0 = r^N a_N + sum_k r^(k+1) s_k with sum b_{k+1} = r^(N-1-k) sum theta, so
    du/dx0 = theta r^N and du/dtheta = x0 r^N + N dt c2 sigma r^N."""
    d, N, M, sigma, T = 5, 6, 64, 0.9, 0.8
    c0, c1, c2, c3 = 0.2, -0.6, 0.35, 0.1
    rng = np.random.default_rng(3)
    theta = rng.normal(size=d)
    x0 = rng.normal(size=d)
    p = oracle.Problem("affine_test", d, sigma, T, N, M, theta=theta, A=0.1, c0=c0, c1=c1,
                       c2=c2, c3=c3, ridge_rel=0.0)
    a = oracle.adjoint(p, x0, 4)
    dt = T / N
    r = 1.0 / (1.0 - dt * c1)
    assert np.allclose(a["du_dx0"], theta * r ** N, rtol=1e-10, atol=1e-12)
    extra = N * dt * c2 * sigma * r ** N
    assert np.allclose(a["du_dtheta"], x0 * r ** N + extra, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("kind", ["ac_manufactured", "logistic_grad", "hjb_logquad",
                                  "affine_test", "ac_doublewell", "cos_linear_test"])
def test_problem_table_derivatives_match_numerical_differentiation(kind):
    rng = np.random.default_rng(5)
    d, h = 5, 1e-6
    theta = rng.uniform(0.5, 1.5, d)
    p = oracle.Problem(kind, d, 0.8, 1.0, 4, 16, theta=theta, c2=0.3)
    x = rng.normal(size=d)
    z = rng.normal(scale=0.3, size=d)
    t, y = 0.4, 0.37
    gx, gt = oracle.g_grad(p, x)
    fx, fz = oracle.f_grads(p, t, x, y, z)
    for i in range(d):
        e = np.zeros(d)
        e[i] = h
        assert gx[i] == pytest.approx((oracle.g(p, x + e) - oracle.g(p, x - e)) / (2 * h),
                                      rel=1e-6, abs=1e-9)
        assert fx[i] == pytest.approx((oracle.f(p, t, x + e, y, z)[0]
                                       - oracle.f(p, t, x - e, y, z)[0]) / (2 * h),
                                      rel=1e-6, abs=1e-9)
        assert fz[i] == pytest.approx((oracle.f(p, t, x, y, z + e)[0]
                                       - oracle.f(p, t, x, y, z - e)[0]) / (2 * h),
                                      rel=1e-6, abs=1e-9)
        if kind in ("hjb_logquad", "affine_test"):
            tp, tm = theta.copy(), theta.copy()
            tp[i] += h
            tm[i] -= h
            pp = oracle.Problem(kind, d, 0.8, 1.0, 4, 16, theta=tp)
            pm = oracle.Problem(kind, d, 0.8, 1.0, 4, 16, theta=tm)
            assert gt[i] == pytest.approx((oracle.g(pp, x) - oracle.g(pm, x)) / (2 * h),
                                          rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("kind,d,M,sigma,T", [
    ("hjb_logquad", 200, 800, math.sqrt(2.0), 1.0),
    ("ac_manufactured", 200, 800, 1.0, 1.0),
])
def test_adjoint_solution_moves_between_levels(kind, d, M, sigma, T):
    """The adjoint regression's solution v changes by a large fraction from one level to
    the next (its right-hand side sums per-particle noise), unlike the primal alpha_x; a
    start from the previous level's v saves few CG passes and a linear extrapolation over two
    levels is worse.  This is why the GPU reverse sweep needs about twice the primal's CG
    passes."""
    N = 20
    rng = np.random.default_rng(1)
    theta = rng.uniform(0.5, 1.5, d) if kind == "hjb_logquad" else None
    x0 = rng.normal(scale=1 / math.sqrt(d), size=d)
    p = oracle.Problem(kind, d, sigma, T, N, M, theta=theta, cg_tol=1e-12)
    V = oracle.adjoint(p, x0, 4, 0, trace=True)["v_levels"]
    const = [np.linalg.norm(V[k] - V[k - 1]) / np.linalg.norm(V[k]) for k in range(2, N)]
    linear = [np.linalg.norm(V[k] - 2 * V[k - 1] + V[k - 2]) / np.linalg.norm(V[k])
              for k in range(2, N)]
    assert 0.2 < np.median(const) < 0.8
    assert np.median(linear) > np.median(const)
    prim = oracle.solve(p, x0, 4, 0, trace=True)["alpha_x"]
    steady = [np.linalg.norm(prim[k] - prim[k + 1]) / np.linalg.norm(prim[k]) for k in range(N - 1)]
    assert np.median(steady) < np.median(const)


def test_adjoint_derivatives_against_cole_hopf_monte_carlo():
    """sigma = sqrt 2, f = -|z|^2/2, g = log((1 + sum theta_i x_i^2)/2): v = e^{-u} solves the
    heat equation, so u(0,x0) = -ln E[e^{-g(X_T)}], X_T = x0 + sqrt 2 W_T, and its
    derivatives are ratios of expectations,
        du/dx0_i   = E[e^{-g} 2 theta_i X_i / (1 + sum theta X^2)] / E[e^{-g}],
        du/dtheta_i = E[e^{-g} X_i^2 / (1 + sum theta X^2)] / E[e^{-g}],
    which plain Monte Carlo estimates independently of the scheme (800k samples).  The
    oracle's reverse sweep differentiates the scheme's estimator for fixed increments; on
    average over its cloud that is the derivative of u, so both must agree up to the
    scheme's error (time step, regression) and the Monte-Carlo spread of each side."""
    rng = np.random.default_rng(13)
    d, T = 200, 1.0
    theta = rng.uniform(0.5, 1.5, d)
    x0 = rng.standard_normal(d) / math.sqrt(d)
    num_x, num_t, den = np.zeros(d), np.zeros(d), 0.0
    for _ in range(8):
        X = x0 + math.sqrt(2.0 * T) * rng.standard_normal((100_000, d))
        q = 1.0 + (theta * X * X).sum(axis=1)
        v = 2.0 / q
        den += v.sum()
        num_x += ((v / q)[:, None] * (2.0 * theta * X)).sum(axis=0)
        num_t += ((v / q)[:, None] * (X * X)).sum(axis=0)
    ref_x, ref_t = num_x / den, num_t / den
    p = oracle.Problem("hjb_logquad", d, math.sqrt(2.0), T, 10, 4096, theta=theta)
    r = oracle.adjoint(p, x0, seed=9)
    assert r["status"] == 0
    err_x = np.linalg.norm(r["du_dx0"] - ref_x) / np.linalg.norm(ref_x)
    err_t = np.linalg.norm(r["du_dtheta"] - ref_t) / np.linalg.norm(ref_t)
    # measured (seeds 9-11): err_t 0.020-0.023 and err_x 0.069-0.072, with Monte-Carlo
    # standard errors of the reference of 0.0015 and 0.021; a sign or factor error in
    # either derivative lands near 1 or 2
    assert err_t < 0.04, err_t
    assert err_x < 0.12, err_x
    assert 0.9 < float(r["du_dx0"] @ ref_x) / float(ref_x @ ref_x) < 1.1
