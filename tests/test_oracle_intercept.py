"""Pins for the oracle's centring, standardisation and intercept.

Checks against things fixed outside the oracle's algebra: statistics of an
explicitly centred and scaled copy of X, ordinary least squares with a column
of ones (numpy lstsq) as the lambda -> 0 limit, the KKT conditions of the
intercept model on the original scale (mean residual zero, penalised
gradient bounded by lambda sd_j), invariance of the slopes under shifts of a
column or of y, a constant column dropping out, and a direct held-out
residual pass for the CV error.
"""
import numpy as np
import pytest

import synthgen
from oracle import (Penalty, augmented_sums, back_transform, centered_stats, cv_mse_intercept,
                    fit, lambda_grid, lambda_max, lanczos_d, oem_path, xval_intercept)


def _data(n=300, p=6, seed=3, shift=0.0):
    X = synthgen.ar1_design(n, p, 0.5, seed, np.float64)
    X = X * np.linspace(0.5, 3.0, p) + np.linspace(-2.0, 5.0, p) + shift
    beta = synthgen.leading_beta(p, [1.0, -0.7, 0.0, 0.4])
    y = synthgen.response(X, beta, 0.5, seed, np.float64) + 3.0
    return X, y


@pytest.mark.parametrize("intercept,standardize", [(True, True), (True, False), (False, True)])
def test_centered_stats_match_an_explicitly_centred_copy(intercept, standardize):
    X, y = _data()
    n = X.shape[0]
    G, c, N, mu, sd, ybar, const = centered_stats(*augmented_sums(X, y), intercept, standardize)
    Xc = X - X.mean(0) if intercept else X.copy()
    yc = y - y.mean() if intercept else y.copy()
    s = np.sqrt((Xc * Xc).mean(0)) if standardize else np.ones(X.shape[1])
    Xs = Xc / s
    np.testing.assert_allclose(G, Xs.T @ Xs / n, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(c, Xs.T @ yc / n, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(N, yc @ yc / n, rtol=1e-12)
    np.testing.assert_allclose(sd, s, rtol=1e-12)
    assert not const.any()
    if standardize:
        np.testing.assert_allclose(np.diag(G), 1.0, rtol=1e-12)


def test_small_lambda_limit_is_least_squares_with_intercept():
    X, y = _data(n=400, p=5, seed=8)
    Gr, cr, Nr, s, t, n = augmented_sums(X, y)
    G, c, N, mu, sd, ybar, _ = centered_stats(Gr, cr, Nr, s, t, n, True, True)
    d = lanczos_d(G)[0]
    lam = 1e-9 * lambda_max(c, Penalty("lasso"))
    pr = oem_path(G, c, d, Penalty("lasso"), [lam], tol=1e-14, max_iter=200_000)
    beta, beta0 = back_transform(pr.beta[0], mu, sd, ybar)
    A = np.column_stack([np.ones(n), X])
    ref = np.linalg.lstsq(A, y, rcond=None)[0]
    np.testing.assert_allclose(beta0, ref[0], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(beta, ref[1:], rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("kind,kw", [("lasso", {}), ("enet", {"alpha": 0.5})])
def test_kkt_of_the_intercept_model_on_the_original_scale(kind, kw):
    X, y = _data(n=500, p=8, seed=21)
    n = X.shape[0]
    pen = Penalty(kind, **kw)
    res = fit(X, y, [pen], True, True, nlambda=12, lambda_min_ratio=1e-2, tol=1e-12,
              max_iter=100_000)
    sd = np.sqrt(((X - X.mean(0)) ** 2).mean(0))
    alpha = kw.get("alpha", 1.0)
    for l, lam in enumerate(res.lambdas[0]):
        b, b0 = res.beta[0, l], res.beta0[0, l]
        r = y - b0 - X @ b
        assert abs(r.mean()) <= 1e-10 * max(1.0, abs(y).max())
        # standardized coefficient bs_j = b_j sd_j; gradient of the scaled
        # loss: g_j = -x_sj^T r / n with x_sj = (x_j - mean) / sd_j
        g = -((X - X.mean(0)) / sd).T @ r / n
        bs = b * sd
        gl = g + (1 - alpha) * lam * bs  # ridge part of the elastic net
        on = bs != 0
        assert np.all(np.abs(gl[on] + alpha * lam * np.sign(bs[on])) <= 1e-7 * max(1.0, lam))
        assert np.all(np.abs(gl[~on]) <= alpha * lam * (1 + 1e-7) + 1e-10)


def test_slopes_do_not_move_when_a_column_or_y_is_shifted():
    X, y = _data(seed=5)
    pen = Penalty("mcp", gamma=3.0)
    a = fit(X, y, [pen], True, True, nlambda=10, lambda_min_ratio=1e-2, tol=1e-12)
    X2 = X.copy()
    X2[:, 2] += 7.5
    b = fit(X2, y + 11.0, [pen], True, True, nlambda=10, lambda_min_ratio=1e-2, tol=1e-12)
    np.testing.assert_allclose(b.lambdas, a.lambdas, rtol=1e-10)
    np.testing.assert_allclose(b.beta, a.beta, rtol=1e-8, atol=1e-10)
    # the intercept absorbs the shifts: beta0' = beta0 + 11 - 7.5 beta_2
    np.testing.assert_allclose(b.beta0, a.beta0 + 11.0 - 7.5 * a.beta[..., 2], rtol=1e-8, atol=1e-8)


def test_constant_column_drops_out():
    X, y = _data(seed=9)
    Xc = np.column_stack([X, np.full(X.shape[0], 4.25)])
    pen = Penalty("lasso")
    a = fit(X, y, [pen], True, True, nlambda=8, lambda_min_ratio=1e-2, tol=1e-12)
    b = fit(Xc, y, [pen], True, True, nlambda=8, lambda_min_ratio=1e-2, tol=1e-12)
    G, c, N, mu, sd, ybar, const = centered_stats(*augmented_sums(Xc, y), True, True)
    assert const[-1] and not const[:-1].any()
    assert np.all(b.beta[..., -1] == 0.0)
    np.testing.assert_allclose(b.beta[..., :-1], a.beta, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(b.beta0, a.beta0, rtol=1e-9, atol=1e-12)


def test_cv_mse_intercept_matches_direct_residuals():
    X, y = _data(n=240, p=5, seed=13)
    rng = np.random.default_rng(2)
    fold = rng.integers(0, 4, size=X.shape[0])
    rows = fold == 1
    Gk, ck, Nk, sk, tk, nk = augmented_sums(X[rows], y[rows])
    B = rng.normal(size=(3, 5))
    b0 = rng.normal(size=3)
    direct = np.array([np.mean((y[rows] - b0[i] - X[rows] @ B[i]) ** 2) for i in range(3)])
    np.testing.assert_allclose(cv_mse_intercept(Gk, ck, Nk, sk, tk, nk, B, b0), direct, rtol=1e-11)


def test_xval_intercept_full_fit_equals_fit_and_mse_is_held_out():
    X, y = _data(n=360, p=6, seed=17)
    rng = np.random.default_rng(4)
    fold = rng.integers(0, 3, size=X.shape[0])
    pens = [Penalty("lasso"), Penalty("scad", gamma=3.7)]
    full, mse, cvm, cvsd, imin, i1se, best = xval_intercept(X, y, fold, 3, pens, nlambda=8,
                                                            lambda_min_ratio=1e-2, tol=1e-10)
    ref = fit(X, y, pens, True, True, nlambda=8, lambda_min_ratio=1e-2, tol=1e-10)
    np.testing.assert_allclose(full.beta, ref.beta, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(full.beta0, ref.beta0, rtol=1e-12, atol=1e-14)
    # fold 2's error: refit on the other folds, residuals on fold 2 directly
    tr = fold != 2
    for i in range(2):
        # the folds use the full-data grid: refit the training rows on it
        G, c, N, mu, sd, ybar, _ = centered_stats(*augmented_sums(X[tr], y[tr]), True, True)
        pr = oem_path(G, c, lanczos_d(G)[0], pens[i], full.lambdas[i], tol=1e-10)
        b, b0 = back_transform(pr.beta, mu, sd, ybar)
        direct = np.mean((y[~tr][None, :] - b0[:, None] - b @ X[~tr].T) ** 2, axis=1)
        np.testing.assert_allclose(mse[i, 2], direct, rtol=1e-8)
