"""Pins for the oracle's penalised logistic regression (Section 4).

Checks against things fixed outside the oracle's iteration: the null model at
lambda_max, the KKT conditions of the penalised log-likelihood (score of the
unpenalised intercept zero, |x_j^T (y - mu)| / n <= lambda on the inactive
set, equal with the sign of beta_j on the active set), the maximum-likelihood
estimate of an independent Newton-Raphson solver with the exact Hessian as
lambda -> 0, the majorise-minimise decrease of the objective at every outer
step, and the objective against a direct evaluation.
"""
import math

import numpy as np
import pytest

import synthgen
from oracle import Penalty, logistic_loss, logistic_path, sigmoid


def _data(n=600, p=6, seed=3):
    X = synthgen.ar1_design(n, p, 0.5, seed, np.float64)
    beta = np.zeros(p)
    beta[:3] = [1.2, -0.8, 0.5]
    rng = np.random.default_rng(seed)
    prob = 1.0 / (1.0 + np.exp(-(X @ beta - 0.4)))
    y = (rng.random(n) < prob).astype(np.float64)
    return X, y


def _newton_mle(X, y, iters=50):
    Z = np.column_stack([X, np.ones(X.shape[0])])
    b = np.zeros(Z.shape[1])
    for _ in range(iters):
        mu = 1.0 / (1.0 + np.exp(-(Z @ b)))
        H = Z.T @ (Z * (mu * (1 - mu))[:, None])
        b = b + np.linalg.solve(H, Z.T @ (y - mu))
    return b


def test_sigmoid_and_loss_are_the_textbook_forms():
    t = np.array([-800.0, -3.0, 0.0, 2.5, 800.0])
    np.testing.assert_allclose(sigmoid(t), [0.0, 1 / (1 + math.exp(3)), 0.5, 1 / (1 + math.exp(-2.5)), 1.0])
    Z = np.array([[1.0, 2.0], [0.5, -1.0], [-2.0, 0.3]])
    y = np.array([1.0, 0.0, 1.0])
    b = np.array([0.3, -0.7])
    eta = Z @ b
    direct = -np.mean(y * np.log(1 / (1 + np.exp(-eta))) + (1 - y) * np.log(1 - 1 / (1 + np.exp(-eta))))
    assert abs(logistic_loss(Z, y, b) - direct) <= 1e-14


def test_null_model_at_lambda_max():
    X, y = _data()
    r = logistic_path(X, y, Penalty("lasso"), nlambda=5, lambda_min_ratio=0.1, tol=1e-10)
    assert np.all(r.beta[0] == 0.0)
    assert abs(r.beta0[0] - math.log(y.mean() / (1 - y.mean()))) <= 1e-12
    assert np.any(r.beta[1] != 0.0)


@pytest.mark.parametrize("kind,alpha", [("lasso", 1.0), ("enet", 0.5)])
def test_kkt_of_the_penalised_likelihood(kind, alpha):
    X, y = _data(n=800, p=8, seed=11)
    n = X.shape[0]
    r = logistic_path(X, y, Penalty(kind, alpha=alpha), nlambda=10, lambda_min_ratio=0.02, tol=1e-11,
                      max_iter=200_000)
    assert r.converged.all()
    for l, lam in enumerate(r.lambdas):
        b, b0 = r.beta[l], r.beta0[l]
        res = y - sigmoid(X @ b + b0)
        assert abs(res.mean()) <= 1e-8
        g = X.T @ res / n - (1 - alpha) * lam * b  # score minus the ridge part
        on = b != 0
        assert np.all(np.abs(g[on] - alpha * lam * np.sign(b[on])) <= 1e-7)
        assert np.all(np.abs(g[~on]) <= alpha * lam + 1e-7)


def test_small_lambda_limit_is_the_mle():
    X, y = _data(n=1000, p=5, seed=7)
    mle = _newton_mle(X, y)
    r = logistic_path(X, y, Penalty("lasso"), lambdas=[1e-10], tol=1e-13, max_iter=500_000,
                      max_outer=2000)
    np.testing.assert_allclose(r.beta[0], mle[:5], rtol=1e-6, atol=1e-7)
    assert abs(r.beta0[0] - mle[5]) <= 1e-6


@pytest.mark.parametrize("kind", ["lasso", "mcp", "scad"])
def test_outer_steps_decrease_the_objective(kind):
    X, y = _data(n=500, p=10, seed=5)
    r = logistic_path(X, y, Penalty(kind, gamma=3.7 if kind == "scad" else 3.0), nlambda=8,
                      lambda_min_ratio=0.05, tol=1e-10, max_iter=100_000)
    for l in range(len(r.lambdas)):
        vals = [v for (ll, v) in r.trace if ll == l]
        assert all(b <= a + 1e-12 * max(1.0, abs(a)) for a, b in zip(vals, vals[1:])), (l, vals)
