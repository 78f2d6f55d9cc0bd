"""Pins of the oracle's literal Algorithm 1 (one regression per particle anchor):
the uniform-kernel limit equals the single-anchor solve (a shift of the regressors moves
only the intercept), the affine problem's closed recursion holds for any kernel weights,
and on the manufactured Allen-Cahn problem the per-particle anchors remove the bias that
a single anchor leaves when f depends on x."""
import math

import numpy as np
import pytest

import oracle


def _p(kind, d, N, M, h, **kw):
    sigma = kw.pop("sigma", 1.0)
    T = kw.pop("T", 0.5)
    return oracle.Problem(kind, d, sigma, T, N, M, h=h, cg_tol=1e-13, **kw)


@pytest.mark.parametrize("kind,extra", [
    ("ac_manufactured", {}),
    ("logistic_grad", {"sigma": 6.0, "T": 1.0}),
    ("hjb_logquad", {"sigma": math.sqrt(2.0), "T": 1.0}),
    ("ac_doublewell", {"sigma": math.sqrt(2.0), "T": 0.3}),
    ("cos_linear_test", {"c1": 0.4}),
])
def test_uniform_kernel_limit_equals_single_anchor(kind, extra):
    d, N, M = 6, 4, 120
    rng = np.random.default_rng(7)
    theta = rng.uniform(0.5, 1.5, d) if kind == "hjb_logquad" else None
    x0 = rng.normal(scale=0.4, size=d)
    p = _p(kind, d, N, M, math.inf, theta=theta, **extra)
    a = oracle.solve_anchored(p, x0, 5, 2)
    b = oracle.solve(p, x0, 5, 2)
    assert a["status"] == 0 and b["status"] == 0
    assert abs(a["u0"] - b["u0"]) <= 1e-11 * max(1.0, abs(b["u0"]))
    assert np.max(np.abs(a["grad"] - b["grad"])) <= 1e-11 * max(1.0, np.max(np.abs(b["grad"])))


def test_affine_problem_exact_with_per_anchor_weights():
    """g = A + theta.x, f = c0 + c1 y + c2 sum z + c3 t: every weighted fit recovers the
    affine Y_{k+1} exactly, whatever the anchor's weights, so the closed recursion holds."""
    d, N, M, sigma, T = 5, 5, 90, 0.8, 0.7
    c0, c1, c2, c3, A = 0.2, -0.6, 0.3, -0.5, -0.4
    rng = np.random.default_rng(21)
    theta = rng.normal(size=d)
    x0 = rng.normal(scale=0.5, size=d)
    p = oracle.Problem("affine_test", d, sigma, T, N, M, theta=theta, A=A, c0=c0, c1=c1,
                       c2=c2, c3=c3, h=1.5, ridge_rel=0.0, cg_tol=1e-14)
    r = oracle.solve_anchored(p, x0, 9, 0)
    dt = T / N
    a, b = A + theta @ x0, theta.copy()
    for k in range(N - 1, -1, -1):
        a, b = (a + dt * (c0 + c2 * sigma * b.sum() + c3 * k * dt)) / (1 - dt * c1), \
            b / (1 - dt * c1)
    assert r["status"] == 0
    assert abs(r["u0"] - a) <= 1e-10 * max(1.0, abs(a))
    assert np.max(np.abs(r["grad"] - theta / (1 - dt * c1) ** (N - 1))) <= 1e-9


def test_per_particle_anchors_remove_the_single_anchor_bias():
    """Manufactured Allen-Cahn (f depends on x through sum cos x_i), d = 8, M = 800, h = 2:
    the single-anchor solve is biased by ~1.5e-2; the per-anchor solve is within 2e-3."""
    d, N, M = 8, 8, 800
    x0 = np.random.default_rng(1).normal(scale=0.3, size=d)
    exact = math.exp(-0.5) * np.cos(x0).mean()
    p = _p("ac_manufactured", d, N, M, 2.0)
    a = oracle.solve_anchored(p, x0, 3, 1)
    b = oracle.solve(p, x0, 3, 1)
    assert a["status"] == 0
    assert abs(a["u0"] - exact) < 2e-3
    assert abs(b["u0"] - exact) > 5 * abs(a["u0"] - exact)
