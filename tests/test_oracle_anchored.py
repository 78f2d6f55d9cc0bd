"""Pins of the oracle's literal Algorithm 1 (one regression per particle anchor):
the uniform-kernel limit equals the single-anchor solve (a shift of the regressors moves
only the intercept), the affine problem's closed recursion holds for any kernel weights,
on the manufactured Allen-Cahn problem the per-particle anchors remove the bias that
a single anchor leaves when f depends on x, and at tiny sizes the solve equals a brute
force of the definitions (dense least squares per anchor).  The same pins hold for the
regressions over a subset of K particles per anchor (Remark 2.1: nearest subset, and the
random batch as a cyclic window), plus the nearest subset's bias against the batch."""
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


def _brute_force_anchored(p, x0, seed, s, select=None):
    """Algorithm 1 with one regression per particle anchor, from the definitions at tiny
    sizes: the particle paths, then per level and anchor m the Gaussian weights of
    D_j = X_{k+1}^j - X_k^m with eps_k^2 = h^2 sigma^2 d (t_k + t_{k+1}) (normalised), the
    weighted least squares of Y_{k+1} on [1, D] with the ridge lambda = ridge_rel tr(Gamma_c)/d
    on the slope only (Remark 2.2) solved by a dense lstsq of the augmented system, the
    anchor's intercept and Z = sigma slope, and Newton on Y = alpha + dt f (Eq. 2.16) to
    full precision."""
    d, N, M = p.d, p.N, p.M
    dt = p.T / N
    X = np.stack([oracle.path(p, x0, seed, s, j) for j in range(M)], axis=1)   # [N+1, M, d]
    Y = np.array([oracle.g(p, X[N, j]) for j in range(M)])
    slope0 = None
    for k in range(N - 1, -1, -1):
        t_k = k * dt
        rho_ref = p.sigma ** 2 * d * (t_k + (k + 1) * dt)
        Yk = np.empty(M)
        for m in range(M):
            D = X[k + 1] - X[k, m]
            rho = np.sum(D * D, axis=1)
            if select is not None:   # regression over a subset of the particles
                idx = select(m, rho)
                D, rho, Ysub = D[idx], rho[idx], Y[idx]
            else:
                Ysub = Y
            w = np.exp(-(rho - rho_ref) / (p.h ** 2 * rho_ref))
            w /= w.sum()
            S = w @ D
            lam = p.ridge_rel * (w @ rho - S @ S) / d
            sw = np.sqrt(w)
            rows = np.vstack([np.hstack([sw[:, None], sw[:, None] * D]),
                              np.hstack([np.zeros((d, 1)), math.sqrt(lam) * np.eye(d)])])
            rhs = np.concatenate([sw * Ysub, np.zeros(d)])
            coef = np.linalg.lstsq(rows, rhs, rcond=None)[0]
            alpha, slope = coef[0], coef[1:]
            z = p.sigma * slope
            y = alpha
            for _ in range(100):
                fv, dfdy = oracle.f(p, t_k, X[k, m], y, z)
                step = (y - alpha - dt * fv) / (1.0 - dt * dfdy)
                y -= step
                if abs(step) <= 1e-15 * max(1.0, abs(y)):
                    break
            Yk[m] = y
            if k == 0 and m == 0:
                slope0 = slope
        Y = Yk
    return float(Y.mean()), slope0


@pytest.mark.parametrize("kind,extra", [
    ("ac_manufactured", {}),
    ("logistic_grad", {"sigma": 3.0, "T": 1.0}),
    ("hjb_logquad", {"sigma": math.sqrt(2.0), "T": 1.0}),
])
def test_per_anchor_solve_equals_dense_least_squares_brute_force(kind, extra):
    """Same u(0,x0) and grad u as the brute force above (1e-10 relative): the per-anchor
    bandwidth, the normalisation, the ridge, the intercept and Newton per anchor."""
    d, N, M = 3, 3, 40
    rng = np.random.default_rng(11)
    theta = rng.uniform(0.5, 1.5, d) if kind == "hjb_logquad" else None
    x0 = rng.normal(scale=0.5, size=d)
    p = _p(kind, d, N, M, 2.0, theta=theta, **extra)
    ref_u, ref_g = _brute_force_anchored(p, x0, 3, 1)
    a = oracle.solve_anchored(p, x0, 3, 1)
    assert a["status"] == 0
    assert abs(a["u0"] - ref_u) <= 1e-10 * max(1.0, abs(ref_u)), (a["u0"], ref_u)
    assert np.max(np.abs(a["grad"] - ref_g)) <= 1e-9 * max(1.0, np.max(np.abs(ref_g)))


# Regression over a subset of K particles per anchor (Remark 2.1): the K nearest (ties by
# the smaller index) or the cyclic window j = (m + q) mod M (a random batch in law).
def _nearest(K):
    return lambda m, rho: np.lexsort((np.arange(len(rho)), rho))[:K]


def _window(K, M):
    return lambda m, rho: (m + np.arange(K)) % M


@pytest.mark.parametrize("which", ["nearest", "batch"])
def test_subset_solves_with_all_particles_equal_the_per_anchor_solve(which):
    d, N, M = 5, 3, 90
    x0 = np.random.default_rng(2).normal(scale=0.4, size=d)
    for kind, extra in (("ac_manufactured", {}), ("logistic_grad", {"sigma": 3.0, "T": 1.0})):
        p = _p(kind, d, N, M, 2.0, **extra)
        fn = oracle.solve_neighbours if which == "nearest" else oracle.solve_batch
        a, b = fn(p, M, x0, 7, 1), oracle.solve_anchored(p, x0, 7, 1)
        assert a["status"] == 0 and b["status"] == 0
        assert abs(a["u0"] - b["u0"]) <= 1e-11 * max(1.0, abs(b["u0"]))
        assert np.max(np.abs(a["grad"] - b["grad"])) <= 1e-10 * max(1.0, np.max(np.abs(b["grad"])))


@pytest.mark.parametrize("which", ["nearest", "batch"])
def test_subset_solves_equal_the_brute_force(which):
    """K = 12 of M = 40: the selection, the weights normalised over the subset, the
    regression and Newton per anchor, against the dense brute force (1e-10)."""
    d, N, M, K = 3, 3, 40, 12
    rng = np.random.default_rng(11)
    x0 = rng.normal(scale=0.5, size=d)
    p = _p("ac_manufactured", d, N, M, 2.0)
    sel = _nearest(K) if which == "nearest" else _window(K, M)
    ref_u, ref_g = _brute_force_anchored(p, x0, 3, 1, select=sel)
    fn = oracle.solve_neighbours if which == "nearest" else oracle.solve_batch
    r = fn(p, K, x0, 3, 1)
    assert r["status"] == 0
    assert abs(r["u0"] - ref_u) <= 1e-10 * max(1.0, abs(ref_u)), (r["u0"], ref_u)
    assert np.max(np.abs(r["grad"] - ref_g)) <= 1e-9 * max(1.0, np.max(np.abs(ref_g)))


def test_nearest_subset_is_biased_and_the_batch_is_not():
    """Manufactured Allen-Cahn, d = 8, M = 800, N = 8, T = 0.5, x0 = 0 (u* = e^-T): the
    regression over each anchor's 200 nearest particles misses u* by more than 0.2; a batch of
    200 (the cyclic window) and all particles are within 0.01."""
    d, N, M, K = 8, 8, 800, 200
    p = _p("ac_manufactured", d, N, M, 2.0)
    x0 = np.zeros(d)
    exact = math.exp(-0.5)
    near = oracle.solve_neighbours(p, K, x0, 3, 0)
    batch = oracle.solve_batch(p, K, x0, 3, 0)
    full = oracle.solve_anchored(p, x0, 3, 0)
    assert near["status"] == batch["status"] == full["status"] == 0
    assert abs(near["u0"] - exact) > 0.2
    assert abs(batch["u0"] - exact) < 0.01 and abs(full["u0"] - exact) < 0.01
