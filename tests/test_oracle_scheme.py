"""End-to-end pins of the oracle's Algorithm 1 against results the paper or the
mathematics fix: exact closed forms of the discrete scheme, a value the paper prints,
an exact Monte-Carlo representation (Cole-Hopf), the first-order time convergence, and at
tiny sizes a brute force of the definitions with nonlinear drivers.
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _prob(kind, d, sigma, T, N, M, **kw):
    return oracle.Problem(kind, d, sigma, T, N, M, **kw)


@pytest.mark.parametrize("h", [2.0, math.inf])
def test_affine_terminal_constant_driver_exact(h):
    """g = A + theta.x, f = c0: the regression is exact at every level, so
    u(0,x0) = A + theta.x0 + T c0 and grad u(0,x0) = theta (left Riemann sum of a
    constant is exact)."""
    rng = np.random.default_rng(10)
    d, T, N = 8, 0.6, 6
    theta = rng.normal(size=d)
    x0 = rng.normal(scale=0.3, size=d)
    p = _prob("affine_test", d, 0.8, T, N, 64, theta=theta, A=0.3, c0=0.25, c1=0.0, h=h,
              ridge_rel=0.0)
    r = oracle.solve(p, x0, seed=1, solve_index=3)
    assert r["status"] == 0
    assert r["u0"] == pytest.approx(0.3 + theta @ x0 + T * 0.25, abs=1e-11)
    assert np.max(np.abs(r["grad"] - theta)) < 1e-10


def test_affine_terminal_linear_driver_closed_recursion():
    """f = c0 + c1 y + c2 sum_i z_i + c3 t keeps Y_k affine in X_k.  With the slope
    b_{k+1} of Y_{k+1} the level-k regression returns (a_{k+1}, b_{k+1}), Z_k = sigma b_{k+1},
    and Y_k = (E_hat + dt (c0 + c2 sigma sum b_{k+1} + c3 t_k)) / (1 - dt c1), so
    a_k = (a_{k+1} + dt (c0 + c2 sigma sum b_{k+1} + c3 t_k)) / (1 - dt c1),
    b_k = b_{k+1} / (1 - dt c1); output u = a_0 and grad = b_1."""
    rng = np.random.default_rng(11)
    d, T, N, sigma = 5, 1.0, 7, 1.1
    c0, c1, c2, c3 = 0.2, -0.7, 0.35, -0.6
    theta = rng.normal(size=d)
    x0 = rng.normal(scale=0.5, size=d)
    p = _prob("affine_test", d, sigma, T, N, 48, theta=theta, A=-0.4, c0=c0, c1=c1, c2=c2,
              c3=c3, ridge_rel=0.0)
    r = oracle.solve(p, x0, seed=2, trace=True)
    dt = T / N
    a, b = -0.4 + theta @ x0, theta.copy()
    for k in range(N - 1, -1, -1):
        # level k regresses Y_{k+1}: intercept a, slope b
        assert r["alpha"][k] == pytest.approx(a, abs=1e-11)
        assert np.max(np.abs(r["alpha_x"][k] - b)) < 1e-10
        src = c0 + c2 * sigma * b.sum() + c3 * k * dt
        a, b = (a + dt * src) / (1 - dt * c1), b / (1 - dt * c1)
    assert r["u0"] == pytest.approx(a, abs=1e-11)


def test_constant_terminal_reduces_to_implicit_euler_ode():
    """g = A, f = y - y^3: every particle carries the same value, the regression slope is
    zero and each level is one backward implicit Euler step of y' = -(y - y^3)."""
    opt = pytest.importorskip("scipy.optimize")
    d, T, N, A = 12, 0.8, 9, 0.8
    p = _prob("cubic_test", d, 1.0, T, N, 32, A=A)
    r = oracle.solve(p, np.zeros(d), seed=3)
    dt = T / N
    y = A
    for _ in range(N):
        y = opt.brentq(lambda v, yn=y: v - dt * (v - v ** 3) - yn, -2, 2, xtol=1e-15)
    assert r["status"] == 0
    assert r["u0"] == pytest.approx(y, abs=1e-13)
    assert np.max(np.abs(r["grad"])) < 1e-12


@pytest.mark.parametrize("c1", [0.0, 0.4])
def test_linear_driver_equals_one_weighted_regression(c1):
    """f = c1 y, uniform weights, no ridge: the lower levels fit affine data exactly, so
    u(0,x0) = alpha/(1 - dt c1)^N and grad = alpha_x/(1 - dt c1)^(N-1), where
    (alpha, alpha_x) is the least-squares fit of g(X_N^j) on X_N^j - x0."""
    rng = np.random.default_rng(12)
    d, T, N, M, sigma, seed, s = 6, 0.9, 5, 80, 0.5, 4, 2
    x0 = rng.normal(scale=0.4, size=d)
    p = _prob("cos_linear_test", d, sigma, T, N, M, c1=c1, h=math.inf, ridge_rel=0.0)
    r = oracle.solve(p, x0, seed=seed, solve_index=s, keep_forward=True)
    XN = r["X_N"]
    # forward sweep (2.7) with mu = 0: X_N^j = x0 + sigma W^j(T), W^j(T) = sqrt(T) xi_{s,N,j}
    dt = T / N
    for j in (0, 17, M - 1):
        end = oracle.normals(seed, s, N, j, d)
        assert np.allclose(XN[j], x0 + sigma * math.sqrt(T) * end, rtol=0, atol=1e-13)
        assert np.array_equal(oracle.path(p, x0, seed, s, j)[N], XN[j])
    gN = np.cos(XN).mean(axis=1)
    assert np.allclose(r["Y_N"], gN, rtol=0, atol=1e-15)
    design = np.hstack([np.ones((M, 1)), XN - x0])
    sol = np.linalg.lstsq(design, gN, rcond=None)[0]
    fac = 1.0 / (1.0 - dt * c1)
    assert r["u0"] == pytest.approx(sol[0] * fac ** N, abs=1e-10)
    assert np.max(np.abs(r["grad"] - sol[1:] * fac ** (N - 1))) < 1e-9


def _mean_err(kind, d, sigma, T, N, M, ref, seeds, h=math.inf, x0=None):
    x0 = np.zeros(d) if x0 is None else x0
    us = [oracle.solve(_prob(kind, d, sigma, T, N, M, h=h), x0, seed=s)["u0"] for s in seeds]
    return float(np.mean(us) - ref), float(np.std(us))


def test_allen_cahn_case1_printed_reference_and_first_order():
    """Sec. 4.1, case 1: d = 100, T = 0.3, x0 = 0, Lap u (sigma = sqrt 2), f = u - u^3,
    g = 1/(2 + 0.4|x|^2); the paper prints u(0,0) ~ 0.0528 and first-order decay in dt."""
    ref = None
    for line in open(os.path.join(ROOT, "tests", "golden", "ac_case1_reference.txt")):
        if line.startswith("u0"):
            ref = float(line.split()[1])
    errs = [_mean_err("ac_doublewell", 100, math.sqrt(2.0), 0.3, N, 2048, ref, range(4))[0]
            for N in (10, 20, 40)]
    assert errs[0] > errs[1] > errs[2]
    assert abs(errs[2]) < 3e-4            # 0.6% of u; the printed value has 3 digits
    slope = np.polyfit(np.log([0.03, 0.015, 0.0075]), np.log(np.abs(errs)), 1)[0]
    assert 0.5 < slope < 1.6


def test_manufactured_allen_cahn_first_order_in_dt():
    """u* = e^{t-T} (1/d) sum cos x_i at x0 = 0: the mean error over seeds decays like dt
    (Theorem 3.1 and the slopes reported in Sec. 4)."""
    ref = math.exp(-0.5)
    errs = [_mean_err("ac_manufactured", 100, 1.0, 0.5, N, 2048, ref, range(4))[0]
            for N in (5, 10, 20)]
    assert all(e > 0 for e in errs) and errs[0] > errs[1] > errs[2]
    slope = np.polyfit(np.log([0.1, 0.05, 0.025]), np.log(errs), 1)[0]
    assert 0.6 < slope < 1.3


def test_particle_count_sets_the_monte_carlo_spread():
    """Seed-to-seed spread shrinks as M grows (the M_eff term of Lemma 3.10)."""
    sd = [_mean_err("ac_manufactured", 100, 1.0, 0.5, 10, M, 0.0, range(24), h=2.0)[1]
          for M in (256, 1024)]
    assert 1.3 < sd[0] / sd[1] < 3.5


def test_cole_hopf_monte_carlo_reference():
    """sigma = sqrt 2, f = -|z|^2/2: v = e^{-u} solves the heat equation, so
    u(0,x0) = -ln E[exp(-g(x0 + sqrt 2 W_T))] exactly; plain Monte Carlo estimates it."""
    rng = np.random.default_rng(13)
    d, T = 200, 1.0
    theta = rng.uniform(0.5, 1.5, d)
    x0 = rng.standard_normal(d) / math.sqrt(d)
    acc = []
    for _ in range(8):
        X = x0 + math.sqrt(2.0 * T) * rng.standard_normal((100_000, d))
        acc.append(2.0 / (1.0 + (theta * X * X).sum(axis=1)))
    v = np.concatenate(acc)
    ref = -math.log(v.mean())
    p = _prob("hjb_logquad", d, math.sqrt(2.0), T, 10, 4096, theta=theta)
    r = oracle.solve(p, x0, seed=9)
    assert r["status"] == 0
    assert abs(r["u0"] - ref) / abs(ref) < 5e-4


def test_result_does_not_depend_on_thread_count():
    code = ("import numpy as np, oracle;"
            "p=oracle.Problem('ac_manufactured',37,1.0,0.5,4,300);"
            "r=oracle.solve(p,np.linspace(-1,1,37),seed=5,solve_index=1);"
            "print(repr(r['u0']), r['grad'].tobytes().hex())")
    outs = []
    for nt in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=nt, PYTHONPATH=ROOT)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT,
                                   capture_output=True, text=True, check=True).stdout)
    assert outs[0] == outs[1]


def test_partial_sweep_and_argument_errors():
    p = _prob("ac_manufactured", 10, 1.0, 0.5, 6, 64)
    r = oracle.solve(p, np.zeros(10), seed=0, max_levels=2, trace=True)
    assert r["status"] == 0 and math.isnan(r["u0"])
    assert np.isfinite(r["alpha"][4:]).all() and np.isnan(r["alpha"][:4]).all()
    bad = _prob("ac_manufactured", 10, 1.0, 0.5, 6, 1)
    assert oracle.solve(bad, np.zeros(10), seed=0)["status"] == 1


def test_top_level_regression_uses_the_forward_cloud_and_its_spread():
    """Level N-1 regresses Y_N = g(X_N) on D = X_N - x0 with kernel scale
    eps^2 = h^2 E|D|^2 and E|D|^2 = sigma^2 d T (the variance of the forward SDE (2.3)
    with mu = 0); the empirical spread of the cloud agrees with that expectation."""
    rng = np.random.default_rng(14)
    d, T, N, M, sigma, h = 30, 0.7, 4, 2000, 1.7, 1.2
    x0 = rng.normal(size=d)
    p = _prob("ac_manufactured", d, sigma, T, N, M, h=h)
    r = oracle.solve(p, x0, seed=6, solve_index=1, trace=True, keep_forward=True)
    D = r["X_N"] - x0
    spread = np.mean(np.sum(D * D, axis=1))
    assert spread == pytest.approx(sigma ** 2 * d * T, rel=4 * math.sqrt(2.0 / (d * M)))
    alpha, ax, _, _, st = oracle.llr(D, r["Y_N"], sigma ** 2 * d * T, h=h, ridge_rel=1e-3)
    assert st == 0
    assert r["alpha"][N - 1] == pytest.approx(alpha, rel=1e-12)
    assert np.max(np.abs(r["alpha_x"][N - 1] - ax)) < 1e-12 * np.max(np.abs(ax))


def _increments(p, x0, seed, s, M):
    paths = np.stack([oracle.path(p, x0, seed, s, j) for j in range(M)])  # [M, N+1, d]
    assert np.array_equal(paths[:, 0], np.broadcast_to(x0, (M, p.d)))      # X_0 = x0
    return np.diff(paths, axis=1) / p.sigma                                 # dW_k, [M, N, d]


def test_bridge_path_has_the_increment_law_of_the_forward_scheme():
    """Eq. 2.7 asks for independent increments dW_k ~ N(0, dt I).  The path is drawn
    backwards by the Brownian bridge, so check the law of its increments over many
    particles: mean 0, variance dt at every level, no covariance between levels or
    dimensions, Gaussian fourth moment.  A wrong bridge weight or variance (e.g. t_k in
    place of t_k dt / t_{k+1}, or the weight 1) breaks the per-level variances."""
    d, T, N, M, sigma = 3, 0.9, 6, 6000, 0.7
    dt = T / N
    p = _prob("cos_linear_test", d, sigma, T, N, M)
    x0 = np.array([0.3, -1.1, 2.0])
    dW = _increments(p, x0, 21, 4, M)
    n = M * d
    z = dW / math.sqrt(dt)                      # should be iid N(0,1)
    se = 1.0 / math.sqrt(n)
    for k in range(N):
        zk = z[:, k].ravel()
        assert abs(zk.mean()) < 5 * se, k
        assert abs(zk.var() - 1.0) < 5 * math.sqrt(2.0) * se, k
        assert abs(np.mean(zk ** 4) - 3.0) < 5 * math.sqrt(96.0) * se, k
        for k2 in range(k):
            c = np.mean(z[:, k] * z[:, k2])
            assert abs(c) < 5 * se, (k, k2)
    # dimensions are independent too
    zz = z.reshape(M, N * d)
    assert abs(np.mean(zz[:, 0] * zz[:, 1])) < 5 / math.sqrt(M)


def test_bridge_path_ends_and_levels():
    """W(T) = sqrt(T) xi_{s,N,j} exactly; the level-k position uses the level-k normals
    only through the bridge step (changing the seed moves every level; the same seed
    repeats the path bit for bit); X_0 = x0 for every particle."""
    d, T, N = 5, 1.3, 4
    p = _prob("cos_linear_test", d, 1.7, T, N, 8)
    x0 = np.linspace(-1, 1, d)
    a = oracle.path(p, x0, 3, 2, 5)
    assert np.array_equal(a, oracle.path(p, x0, 3, 2, 5))
    assert np.allclose(a[N], x0 + 1.7 * math.sqrt(T) * oracle.normals(3, 2, N, 5, d),
                       rtol=0, atol=1e-15)
    assert np.array_equal(a[0], x0)
    b = oracle.path(p, x0, 4, 2, 5)
    assert np.all(np.abs(a[1:] - b[1:]) > 0)


def _brute_force_single_anchor(p, x0, seed, s):
    """Algorithm 1 with one anchor per level (the query's drift path a_k = x0), from the
    definitions at tiny sizes: the particle paths; per level the Gaussian weights of
    D_j = X_{k+1}^j - x0 with eps_k^2 = h^2 sigma^2 d t_{k+1} (normalised), the weighted
    least squares of Y_{k+1} on [1, D] with the ridge lambda = ridge_rel tr(Gamma_c)/d on the
    slope only, solved by a dense lstsq of the augmented system; Z_k = sigma slope; and per
    particle Newton on Y = alpha + slope . (X_k^j - x0) + dt f(t_k, X_k^j, Y, Z_k)."""
    d, N, M = p.d, p.N, p.M
    dt = p.T / N
    X = np.stack([oracle.path(p, x0, seed, s, j) for j in range(M)], axis=1)   # [N+1, M, d]
    Y = np.array([oracle.g(p, X[N, j]) for j in range(M)])
    slope = None
    for k in range(N - 1, -1, -1):
        t_k = k * dt
        rho_ref = p.sigma ** 2 * d * (k + 1) * dt
        D = X[k + 1] - x0
        rho = np.sum(D * D, axis=1)
        w = np.exp(-(rho - rho_ref) / (p.h ** 2 * rho_ref)) if math.isfinite(p.h) else np.ones(M)
        w /= w.sum()
        S = w @ D
        lam = p.ridge_rel * (w @ rho - S @ S) / d
        sw = np.sqrt(w)
        rows = np.vstack([np.hstack([sw[:, None], sw[:, None] * D]),
                          np.hstack([np.zeros((d, 1)), math.sqrt(lam) * np.eye(d)])])
        coef = np.linalg.lstsq(rows, np.concatenate([sw * Y, np.zeros(d)]), rcond=None)[0]
        alpha, slope = coef[0], coef[1:]
        z = p.sigma * slope
        Yk = np.empty(M)
        for j in range(M):
            e = alpha + slope @ (X[k, j] - x0)
            y = e
            for _ in range(100):
                fv, dfdy = oracle.f(p, t_k, X[k, j], y, z)
                step = (y - e - dt * fv) / (1.0 - dt * dfdy)
                y -= step
                if abs(step) <= 1e-15 * max(1.0, abs(y)):
                    break
            Yk[j] = y
        Y = Yk
    return float(Y.mean()), slope


@pytest.mark.parametrize("kind,extra", [
    ("ac_manufactured", {}),
    ("logistic_grad", {"sigma": 3.0, "T": 1.0}),
    ("hjb_logquad", {"sigma": math.sqrt(2.0), "T": 1.0}),
    ("ac_doublewell", {"sigma": math.sqrt(2.0), "T": 0.3}),
])
def test_solve_equals_dense_least_squares_brute_force(kind, extra):
    """Nonlinear drivers: orc_solve equals the brute force above to 1e-10 (the bandwidth,
    the normalisation, the ridge on the slope only, the prediction at X_k^j and Newton)."""
    d, N, M = 4, 4, 60
    rng = np.random.default_rng(17)
    theta = rng.uniform(0.5, 1.5, d) if kind == "hjb_logquad" else None
    x0 = rng.normal(scale=0.5, size=d)
    sigma, T = extra.get("sigma", 1.0), extra.get("T", 0.5)
    p = _prob(kind, d, sigma, T, N, M, theta=theta, h=2.0, cg_tol=1e-14)
    ref_u, ref_g = _brute_force_single_anchor(p, x0, 5, 2)
    r = oracle.solve(p, x0, 5, 2)
    assert r["status"] == 0
    assert abs(r["u0"] - ref_u) <= 1e-10 * max(1.0, abs(ref_u)), (r["u0"], ref_u)
    assert np.max(np.abs(r["grad"] - ref_g)) <= 1e-9 * max(1.0, np.max(np.abs(ref_g)))
