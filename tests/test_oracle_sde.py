"""Pins of the oracle of the scheme with a drift and a state-dependent diffusion (the
forward SDE of Sec. 2.1 with mu_i(x) = mu0 + mu1 x_i, sigma(x) = diag(sig0 + sig1 x_i);
Euler-Maruyama paths (2.7); anchor on the drift path of x0; Z = sigma(X)^T alpha_x per
particle).  References that do not share its code path:
  - the closed recursion of the discrete scheme for affine g and affine f (exact);
  - the PDE (2.1) itself for the manufactured drift kinds, with the derivatives of the
    closed forms taken by finite differences and f from the oracle's own table;
  - the law of the Euler-Maruyama increments;
  - a brute force of the scheme's definitions at tiny sizes (dense weighted least squares);
  - first-order convergence to the closed form as dt shrinks.
"""
import math

import numpy as np
import pytest

import oracle


def _prob(kind, d, sig0, T, N, M, **kw):
    return oracle.Problem(kind, d, sig0, T, N, M, **kw)


@pytest.mark.parametrize("coef", [(0.2, -0.4, 0.25), (0.0, 0.3, 0.0), (-0.1, 0.0, 0.4)])
def test_affine_problem_closed_recursion_under_drift_and_diffusion(coef):
    """g = A + theta . x, f = c0 + c1 y + c2 sum_i z_i + c3 t, no ridge: every regression is
    exact, the prediction at the drifted position and Z = sigma(X)^T b are affine in X, so
    Y_k = a_k + b_k . X_k with
        b_k = (1 + mu1 dt + c2 sig1 dt) b_{k+1} / (1 - c1 dt),
        a_k = (a_{k+1} + dt (mu0 sum b + c0 + c2 sig0 sum b + c3 t_k)) / (1 - c1 dt),
    b = b_{k+1} the slope of level k, u(0,x0) = a_0 + b_0 . x0 and grad u = b_1."""
    mu0, mu1, sig1 = coef
    d, N, M, T, sig0 = 6, 5, 80, 0.8, 0.3
    A, c0, c1, c2, c3 = 0.3, 0.2, -0.5, 0.35, -0.4
    rng = np.random.default_rng(3)
    theta = rng.normal(size=d)
    x0 = rng.normal(scale=0.5, size=d)
    p = _prob("affine_test", d, sig0, T, N, M, theta=theta, A=A, c0=c0, c1=c1, c2=c2, c3=c3,
              ridge_rel=0.0, cg_tol=1e-14, h=1.5)
    r = oracle.solve_sde(p, x0, 7, 0, mu0=mu0, mu1=mu1, sig1=sig1)
    assert r["status"] == 0
    dt = T / N
    a, b = A, theta.copy()
    grad_ref = None
    for k in range(N - 1, -1, -1):
        sb = b.sum()
        a = (a + dt * (mu0 * sb + c0 + c2 * sig0 * sb + c3 * k * dt)) / (1 - c1 * dt)
        grad_ref = b.copy()
        b = b * (1 + mu1 * dt + c2 * sig1 * dt) / (1 - c1 * dt)
    assert abs(r["u0"] - (a + b @ x0)) <= 1e-12 * max(1.0, abs(a))
    assert np.max(np.abs(r["grad"] - grad_ref)) <= 1e-11 * np.max(np.abs(grad_ref))


def _closed(kind, t, x, T):
    e = math.exp(t - T)
    return e * np.mean(np.cos(x)) if kind == "drift_ac" else e * np.mean(x * x)


@pytest.mark.parametrize("kind", ["drift_ac", "drift_quad"])
@pytest.mark.parametrize("coef", [(0.2, -0.7, 0.3), (0.0, 0.4, 0.0), (0.5, 0.0, -0.2)])
def test_drift_kinds_manufactured_solution_solves_the_pde(kind, coef):
    """d_t u + 1/2 sum_i s_i(x)^2 d_ii u + sum_i m_i(x) d_i u + f(t, x, u, sigma^T grad u) = 0
    at u = u*, with s_i = sig0 + sig1 x_i, m_i = mu0 + mu1 x_i, the derivatives of u* by
    central differences and f from the oracle's table: the residual is the difference
    error only.  A sign or a factor in the source moves it by O(0.1)."""
    mu0, mu1, sig1 = coef
    d, T, sig0 = 4, 1.0, 0.6
    p = _prob(kind, d, sig0, T, 4, 8)
    rng = np.random.default_rng(5)
    h = 1e-3
    for _ in range(5):
        x = rng.uniform(-1.5, 1.5, size=d)
        t = rng.uniform(0.0, T)
        u = _closed(kind, t, x, T)
        ut = (_closed(kind, t + h, x, T) - _closed(kind, t - h, x, T)) / (2 * h)
        grad, lap = np.zeros(d), 0.0
        s = sig0 + sig1 * x
        m = mu0 + mu1 * x
        for i in range(d):
            e = np.zeros(d)
            e[i] = h
            up, um = _closed(kind, t, x + e, T), _closed(kind, t, x - e, T)
            grad[i] = (up - um) / (2 * h)
            lap += 0.5 * s[i] ** 2 * (up - 2 * u + um) / h ** 2
        f, _ = oracle.sde_f(p, t, x, u, s * grad, mu0=mu0, mu1=mu1, sig1=sig1)
        assert abs(ut + lap + m @ grad + f) < 1e-5


def test_euler_maruyama_increments_have_the_law_of_2_7():
    """(X_{k+1} - X_k - mu(X_k) dt) / (sigma(X_k) sqrt dt) is a standard normal, independent
    across levels, particles and dimensions, and X_0 = x0."""
    d, N, M, T, sig0 = 8, 4, 3000, 0.8, 0.5
    mu0, mu1, sig1 = 0.3, -0.6, 0.2
    p = _prob("drift_quad", d, sig0, T, N, M)
    x0 = np.linspace(-0.5, 0.5, d)
    r = oracle.solve_sde(p, x0, 11, 2, mu0=mu0, mu1=mu1, sig1=sig1, keep_paths=True)
    X = r["paths"]
    assert np.array_equal(X[0], np.broadcast_to(x0, (M, d)))
    dt = T / N
    xi = (X[1:] - X[:-1] - (mu0 + mu1 * X[:-1]) * dt) / ((sig0 + sig1 * X[:-1]) * math.sqrt(dt))
    n = xi.size
    assert abs(xi.mean()) < 4 / math.sqrt(n)
    assert abs(xi.var() - 1.0) < 4 * math.sqrt(2.0 / n)
    assert abs(np.mean(xi[1:] * xi[:-1])) < 4 / math.sqrt(xi[1:].size)   # levels independent
    assert abs(np.mean(xi ** 4) - 3.0) < 0.15


def _brute_force(p, x0, seed, s, mu0, mu1, sig1):
    """The scheme from its definitions at tiny sizes: the drift path a_k of x0; per level the
    Gaussian weights of D_j = X_{k+1}^j - a_k with eps_k^2 = h^2 mean_j |D_j|^2
    (normalised), the weighted least squares of Y_{k+1} on [1, D] with the ridge
    ridge_rel tr(Gamma_c)/d on the slope, by a dense lstsq of the augmented system; per
    particle Z = sigma(X_k^j) slope, the prediction alpha + slope . (X_k^j + mu(X_k^j) dt
    - a_k), and Newton on Y = prediction + dt f(t_k, X_k^j, Y, Z)."""
    d, N, M = p.d, p.N, p.M
    dt = p.T / N
    X = oracle.solve_sde(p, x0, seed, s, mu0=mu0, mu1=mu1, sig1=sig1, keep_paths=True)["paths"]
    a = [np.array(x0, dtype=float)]
    for k in range(N):
        a.append(a[-1] + (mu0 + mu1 * a[-1]) * dt)
    Y = np.array([oracle.sde_g(p, X[N, j]) for j in range(M)])
    slope = None
    for k in range(N - 1, -1, -1):
        D = X[k + 1] - a[k]
        rho = np.sum(D * D, axis=1)
        rho_ref = rho.mean()
        w = np.exp(-(rho - rho_ref) / (p.h ** 2 * rho_ref))
        w /= w.sum()
        S = w @ D
        lam = p.ridge_rel * (w @ rho - S @ S) / d
        sw = np.sqrt(w)
        rows = np.vstack([np.hstack([sw[:, None], sw[:, None] * D]),
                          np.hstack([np.zeros((d, 1)), math.sqrt(lam) * np.eye(d)])])
        coef = np.linalg.lstsq(rows, np.concatenate([sw * Y, np.zeros(d)]), rcond=None)[0]
        alpha, slope = coef[0], coef[1:]
        Yk = np.empty(M)
        for j in range(M):
            x = X[k, j]
            e = alpha + slope @ (x + (mu0 + mu1 * x) * dt - a[k])
            z = (p.sigma + sig1 * x) * slope
            y = e
            for _ in range(100):
                fv, dfdy = oracle.sde_f(p, k * dt, x, y, z, mu0=mu0, mu1=mu1, sig1=sig1)
                step = (y - e - dt * fv) / (1.0 - dt * dfdy)
                y -= step
                if abs(step) <= 1e-15 * max(1.0, abs(y)):
                    break
            Yk[j] = y
        Y = Yk
    return float(Y.mean()), slope


@pytest.mark.parametrize("kind,sig0,coef", [("drift_ac", 0.7, (0.2, -0.6, 0.3)),
                                             ("drift_quad", 0.5, (0.1, 0.4, -0.2)),
                                             ("logistic_grad", 3.0, (0.0, -0.5, 0.5)),
                                             ("ac_doublewell", 1.2, (0.3, 0.0, 0.2))])
def test_solve_equals_brute_force_of_the_definitions(kind, sig0, coef):
    mu0, mu1, sig1 = coef
    d, N, M, T = 3, 4, 50, 0.6
    p = _prob(kind, d, sig0, T, N, M, h=1.8, ridge_rel=1e-2, cg_tol=1e-14)
    x0 = np.array([0.3, -0.2, 0.5])
    r = oracle.solve_sde(p, x0, 21, 1, mu0=mu0, mu1=mu1, sig1=sig1)
    assert r["status"] == 0
    u_bf, g_bf = _brute_force(p, x0, 21, 1, mu0, mu1, sig1)
    assert abs(r["u0"] - u_bf) <= 1e-10 * max(1.0, abs(u_bf))
    assert np.max(np.abs(r["grad"] - g_bf)) <= 1e-9 * max(1.0, np.max(np.abs(g_bf)))


def test_drift_kind_error_decays_with_the_time_step():
    """Allen-Cahn-type source with an Ornstein-Uhlenbeck drift and a state-dependent
    diffusion: the mean error against u* over independent streams decays as dt shrinks
    (the O(dt) of Theorem 3.1) until the Monte-Carlo floor."""
    d, M, T, sig0 = 4, 1500, 0.6, 0.5
    mu0, mu1, sig1 = 0.1, -0.8, 0.2
    x0 = np.array([0.4, -0.3, 0.1, 0.2])
    u_star = math.exp(-T) * float(np.mean(np.cos(x0)))
    errs = []
    for N in (2, 8):
        p = _prob("drift_ac", d, sig0, T, N, M, h=2.0)
        e = [oracle.solve_sde(p, x0, 3, s, mu0=mu0, mu1=mu1, sig1=sig1)["u0"] - u_star
             for s in range(6)]
        errs.append(abs(float(np.mean(e))))
    assert errs[1] < 0.6 * errs[0], errs
