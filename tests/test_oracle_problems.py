"""Pins of the oracle's problem table (terminal g, driver f) and of its Newton solve.

Each closed form is checked against the PDE (2.1) itself with symbolic derivatives:
the residual d_t u + 1/2 sigma^2 Lap u + f(t, x, u, sigma grad u), with f taken from
the oracle, must vanish.  A dropped term or a wrong sign in the driver fails here.
"""
import math

import numpy as np
import pytest

import oracle

sp = pytest.importorskip("sympy")


def _residual_fn(u_expr, xs, t, sigma):
    """Return callables for u, sigma grad u and d_t u + 1/2 sigma^2 Lap u."""
    ut = sp.diff(u_expr, t)
    lap = sum(sp.diff(u_expr, xi, 2) for xi in xs)
    grad = [sp.diff(u_expr, xi) for xi in xs]
    lin = sp.lambdify((t, *xs), ut + sp.Rational(1, 2) * sigma ** 2 * lap, "math")
    uf = sp.lambdify((t, *xs), u_expr, "math")
    gf = sp.lambdify((t, *xs), [sigma * gi for gi in grad], "math")
    return uf, gf, lin


def _pde_residuals(prob, u_expr, xs, t, sigma, rng, n=12, scale=1.0):
    uf, gf, lin = _residual_fn(u_expr, xs, t, sigma)
    out = []
    for _ in range(n):
        tt = rng.uniform(0, prob.T)
        x = rng.normal(0, scale, len(xs))
        u = uf(tt, *x)
        z = np.array(gf(tt, *x), dtype=float)
        fval, _ = oracle.f(prob, tt, x, u, z)
        out.append(lin(tt, *x) + fval)
    return np.array(out)


def test_ac_manufactured_solution_solves_the_pde():
    """u* = e^{t-T} (1/d) sum cos x_i with the driver y - y^3 + q(t,x)."""
    rng = np.random.default_rng(0)
    for d, sigma in [(3, 1.0), (5, 0.7)]:
        t = sp.Symbol("t")
        xs = sp.symbols(f"x0:{d}")
        T = 0.5
        u = sp.exp(t - T) * sum(sp.cos(x) for x in xs) / d
        prob = oracle.Problem("ac_manufactured", d, sigma, T, 10, 16)
        r = _pde_residuals(prob, u, xs, t, sigma, rng)
        assert np.max(np.abs(r)) < 1e-12
        # terminal condition is u*(T, .)
        x = rng.normal(size=d)
        assert oracle.g(prob, x) == pytest.approx(float(u.subs({t: T, **dict(zip(xs, x))})),
                                                  rel=1e-14)


def test_logistic_closed_form_needs_sigma_equal_d():
    """u = logistic(t + sum x_i / d) solves the PDE with f = (y - (2+d)/(2d)) sum z_i
    exactly when sigma = d; with sigma = d/sqrt(2) the residual does not vanish."""
    rng = np.random.default_rng(1)
    d = 4
    t = sp.Symbol("t")
    xs = sp.symbols(f"x0:{d}")
    s = t + sum(xs) / d
    u = 1 / (1 + sp.exp(-s))
    prob = oracle.Problem("logistic_grad", d, float(d), 1.0, 10, 16)
    r = _pde_residuals(prob, u, xs, t, float(d), rng, scale=0.5)
    assert np.max(np.abs(r)) < 1e-12
    x = rng.normal(size=d)
    assert oracle.g(prob, x) == pytest.approx(float(u.subs({t: 1.0, **dict(zip(xs, x))})),
                                              rel=1e-14)
    sig2 = d / math.sqrt(2.0)
    prob2 = oracle.Problem("logistic_grad", d, sig2, 1.0, 10, 16)
    r2 = _pde_residuals(prob2, u, xs, t, sig2, rng, scale=0.5)
    assert np.max(np.abs(r2)) > 1e-3


def test_quadratic_gradient_driver_via_cole_hopf():
    """With sigma = sqrt 2 and f = -|z|^2/2, u = -ln v solves the PDE for every solution v
    of the backward heat equation d_t v + Lap v = 0; v = 1 + sum c_i (x_i^2 + 2(T-t))."""
    rng = np.random.default_rng(2)
    d, T = 3, 1.0
    t = sp.Symbol("t")
    xs = sp.symbols(f"x0:{d}")
    c = rng.uniform(0.5, 1.5, d)
    v = 1 + sum(float(ci) * (xi ** 2 + 2 * (T - t)) for ci, xi in zip(c, xs))
    u = -sp.log(v)
    theta = rng.uniform(0.5, 1.5, d)
    prob = oracle.Problem("hjb_logquad", d, math.sqrt(2.0), T, 10, 16, theta=theta)
    r = _pde_residuals(prob, u, xs, t, math.sqrt(2.0), rng)
    assert np.max(np.abs(r)) < 1e-12
    # terminal: g(x) = -ln(2 / (1 + sum theta_i x_i^2)), the Cole-Hopf image of v_T
    x = rng.normal(size=d)
    assert oracle.g(prob, x) == pytest.approx(-math.log(2.0 / (1.0 + np.sum(theta * x * x))),
                                              rel=1e-14)


@pytest.mark.parametrize("kind", ["ac_manufactured", "logistic_grad", "hjb_logquad",
                                  "cubic_test", "affine_test"])
def test_newton_root_matches_bracketing_solver(kind):
    """Newton (2.17) on F(Y) = Y - E_hat - dt f(t,x,Y,z) (2.16) lands on the root that a
    bracketing solver finds from the same F."""
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(3)
    d = 6
    theta = rng.uniform(0.5, 1.5, d)
    prob = oracle.Problem(kind, d, 1.0 if kind != "logistic_grad" else float(d), 1.0, 10, 16,
                          theta=theta, c0=0.3, c1=-0.7)
    for _ in range(20):
        E_hat = rng.uniform(-0.8, 0.8)
        dt = rng.uniform(0.01, 0.1)
        t = rng.uniform(0, 1)
        x = rng.normal(size=d)
        z = rng.normal(scale=0.2, size=d)
        y, it = oracle.newton(prob, E_hat, dt, t, x, z)
        assert it > 0

        def F(yy):
            return yy - E_hat - dt * oracle.f(prob, t, x, yy, z)[0]
        root = opt.brentq(F, E_hat - 1.0, E_hat + 1.0, xtol=1e-15, rtol=1e-15)
        assert y == pytest.approx(root, abs=1e-12)
        if kind in ("logistic_grad", "hjb_logquad", "affine_test"):
            assert it <= 2   # linear in y: one step, one confirming step
