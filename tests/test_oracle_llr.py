"""Pins of the oracle's weighted local linear regression (Eqs. 2.10-2.15, Remarks 2.2-2.3)
and its Schur-complement conjugate-gradient solve (Lemma 3.7).

The reference solution is an independent dense weighted least-squares solve of the
full (d+1)-parameter problem (numpy's lstsq on the sqrt(w)-scaled design with the
ridge rows appended), so a wrong sign or a dropped term in the Schur complement,
the right-hand side or the intercept recovery fails here.
"""
import math

import numpy as np
import pytest

import oracle


def _dense_wls(D, Y, w, lam):
    """argmin_{a, b} sum_j w_j (Y_j - a - b.D_j)^2 + lam |b|^2 (intercept not penalised)."""
    M, d = D.shape
    sw = np.sqrt(w)
    A = np.zeros((M + d, d + 1))
    A[:M, 0] = sw
    A[:M, 1:] = sw[:, None] * D
    A[M:, 1:] = math.sqrt(lam) * np.eye(d)
    rhs = np.concatenate([sw * Y, np.zeros(d)])
    sol = np.linalg.lstsq(A, rhs, rcond=None)[0]
    return sol[0], sol[1:]


def _cloud(rng, M, d, scale=0.3):
    D = rng.normal(scale=scale, size=(M, d))
    Y = np.sin(D @ rng.normal(size=d)) + 0.1 * rng.normal(size=M)
    return D, Y


@pytest.mark.parametrize("M,d,h,ridge", [(50, 5, 2.0, 1e-3), (50, 5, math.inf, 0.0),
                                         (200, 30, 1.5, 1e-2), (40, 60, 2.0, 1e-3)])
def test_llr_matches_dense_weighted_least_squares(M, d, h, ridge):
    rng = np.random.default_rng(M * 1000 + d)
    D, Y = _cloud(rng, M, d)
    rho_ref = float(np.mean(np.sum(D * D, axis=1)))
    alpha, ax, w, iters, st = oracle.llr(D, Y, rho_ref, h=h, ridge_rel=ridge, cg_tol=1e-13)
    assert st == 0 and iters > 0
    # ridge scale: trace of the weighted covariance of the cloud, per dimension
    lam = ridge * np.trace(np.cov(D, rowvar=False, aweights=w, bias=True)) / d
    a_ref, b_ref = _dense_wls(D, Y, w, lam)
    assert alpha == pytest.approx(a_ref, rel=1e-9, abs=1e-11)
    assert np.linalg.norm(ax - b_ref) <= 1e-8 * np.linalg.norm(b_ref)


def test_kernel_weights_follow_remark_2_3():
    """w_j / w_i = exp(-(|D_j|^2 - |D_i|^2) / eps^2), eps^2 = h^2 rho_ref; sum w = 1;
    h = inf gives equal weights."""
    rng = np.random.default_rng(5)
    D, Y = _cloud(rng, 64, 8)
    rho = np.sum(D * D, axis=1)
    rho_ref, h = 0.7, 1.3
    _, _, w, _, _ = oracle.llr(D, Y, rho_ref, h=h, ridge_rel=1e-3)
    assert w.sum() == pytest.approx(1.0, rel=1e-14)
    eps2 = h * h * rho_ref
    for i, j in [(0, 1), (3, 17), (40, 63)]:
        assert w[j] / w[i] == pytest.approx(math.exp(-(rho[j] - rho[i]) / eps2), rel=1e-12)
    _, _, wu, _, _ = oracle.llr(D, Y, rho_ref, h=math.inf, ridge_rel=1e-3)
    assert np.allclose(wu, 1.0 / 64, rtol=1e-15)


def test_symmetric_cloud_has_zero_first_moment():
    """For a cloud closed under D -> -D the weighted first moment S vanishes (the finite
    form of xi_1 = 0 in Lemma 3.4), so the intercept equals the weighted mean of Y."""
    rng = np.random.default_rng(6)
    half = rng.normal(size=(40, 7))
    D = np.concatenate([half, -half])
    Y = rng.normal(size=80)
    alpha, ax, w, _, st = oracle.llr(D, Y, 7.0, h=2.0, ridge_rel=1e-3)
    assert st == 0
    assert alpha == pytest.approx(float(np.dot(w, Y)), rel=1e-13, abs=1e-15)
    # equal weights within each +/- pair
    assert np.allclose(w[:40], w[40:], rtol=1e-15)


def test_affine_data_recovered_exactly():
    rng = np.random.default_rng(7)
    M, d = 120, 9
    D = rng.normal(size=(M, d))
    a, b = 0.37, rng.normal(size=d)
    Y = a + D @ b
    alpha, ax, _, _, st = oracle.llr(D, Y, float(d), h=2.0, ridge_rel=0.0, cg_tol=1e-14)
    assert st == 0
    assert alpha == pytest.approx(a, abs=1e-12)
    assert np.max(np.abs(ax - b)) < 1e-11


def test_cg_stops_at_tolerance_and_reports_exhaustion():
    rng = np.random.default_rng(8)
    D, Y = _cloud(rng, 100, 20)
    rho_ref = float(np.mean(np.sum(D * D, axis=1)))
    _, ax_loose, w, it_loose, st = oracle.llr(D, Y, rho_ref, cg_tol=1e-3)
    _, ax_tight, _, it_tight, st2 = oracle.llr(D, Y, rho_ref, cg_tol=1e-13)
    assert st == 0 and st2 == 0 and it_tight > it_loose
    # residual of the dense centred system at the loose solution
    S = w @ D
    G = (D * w[:, None]).T @ D - np.outer(S, S)
    lam = 1e-3 * np.trace(G) / 20
    rhs = (w * Y) @ D - float(w @ Y) * S
    res = np.linalg.norm((G + lam * np.eye(20)) @ ax_loose - rhs)
    assert res <= 1e-3 * np.linalg.norm(rhs) * (1 + 1e-9)
    _, _, _, it1, st3 = oracle.llr(D, Y, rho_ref, cg_tol=1e-13, cg_max_iter=2)
    assert st3 == 5 and it1 == 2
