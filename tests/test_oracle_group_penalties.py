"""Pins of the oracle's group MCP, group SCAD and sparse group lasso
(Section 2.2, Eqs. gmcp, gscad, sglasso; Table 1 penalty forms).

* Orthonormal design (G = I, d = 1): one update from any start is the exact
  solution, and it equals the textbook rules written out here independently:
  the group firm threshold (group MCP), the group SCAD rule, and the sparse
  group lasso prox S(c, lambda tau w) (1 - lambda (1 - tau) c_k / ||S||)_+.
* The update is the prox of d/2 ||beta - u/d||^2 + P(beta): checked by a grid
  search over a two-variable group.
* Special cases: tau = 0 is the group lasso, tau = 1 the lasso; groups of
  one variable turn group MCP / SCAD into MCP / SCAD.
* lambda >= lambda_max gives beta = 0 and 0.99 lambda_max does not.
* Converged paths satisfy the KKT conditions; the objective never rises for
  the convex sparse group lasso when d >= lambda_1.
"""
import math

import numpy as np
import pytest

import oracle
from oracle.oem import _sgl_group_lambda

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _orthonormal(n, p, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, p)))
    return Q * math.sqrt(n)


def _groups(p, size):
    return np.arange(p) // size


def _firm_group(cg, lk, gam):
    nrm = np.linalg.norm(cg)
    if nrm <= gam * lk:
        return gam / (gam - 1.0) * max(0.0, 1.0 - lk / nrm) * cg
    return cg.copy()


def _scad_group(cg, lk, gam):
    nrm = np.linalg.norm(cg)
    if nrm <= 2.0 * lk:
        return max(0.0, 1.0 - lk / nrm) * cg
    if nrm <= gam * lk:
        return ((gam - 1.0) * nrm - gam * lk) / ((gam - 2.0) * nrm) * cg
    return cg.copy()


def _sgl_prox(cg, lt_w, lk):
    s = np.sign(cg) * np.maximum(np.abs(cg) - lt_w, 0.0)
    ns = np.linalg.norm(s)
    return s * max(0.0, 1.0 - lk / ns) if ns > 0 else s


@pytest.mark.parametrize("kind", ["grp.mcp", "grp.scad", "sgl"])
def test_orthonormal_design_one_update_is_the_textbook_rule(kind):
    n, p, size = 400, 12, 3
    X = _orthonormal(n, p, 3)
    rng = np.random.default_rng(4)
    y = X @ np.repeat([1.5, 0.4, 0.0, 2.5], size) + 0.3 * rng.standard_normal(n)
    G, c = X.T @ X / n, X.T @ y / n
    np.testing.assert_allclose(G, np.eye(p), atol=1e-12)
    pen = oracle.Penalty(kind, gamma=3.7 if kind == "grp.scad" else 3.0, groups=_groups(p, size),
                         tau=0.4)
    members, cgw = pen.group_list(p)
    lam = 0.3
    beta0 = rng.standard_normal(p)
    got = oracle.threshold(c + 1.0 * beta0 - G @ beta0, lam, 1.0, pen)
    want = np.zeros(p)
    for k, m in enumerate(members):
        if kind == "grp.mcp":
            want[m] = _firm_group(c[m], lam * cgw[k], pen.gamma)
        elif kind == "grp.scad":
            want[m] = _scad_group(c[m], lam * cgw[k], pen.gamma)
        else:
            want[m] = _sgl_prox(c[m], lam * pen.tau, lam * (1 - pen.tau) * cgw[k])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    # and the path converges to it in one step at every lambda
    res = oracle.oem_path(G, c, 1.0, pen, [lam], tol=1e-14)
    np.testing.assert_allclose(res.beta[0], want, atol=1e-12)


@pytest.mark.parametrize("kind,par", [("grp.mcp", {"gamma": 3.0}), ("grp.scad", {"gamma": 3.7}),
                                      ("sgl", {"tau": 0.3}), ("sgl", {"tau": 0.8})])
def test_group_update_is_the_prox_by_grid_search(kind, par):
    d, lam = 1.7, 0.45
    pen = oracle.Penalty(kind, groups=np.array([0, 0]), **par)
    rng = np.random.default_rng(7)
    xs = np.linspace(-3, 3, 1201)
    B1, B2 = np.meshgrid(xs, xs, indexing="ij")
    flat = np.stack([B1.ravel(), B2.ravel()], 1)
    for _ in range(6):
        u = rng.uniform(-2.5, 2.5, 2) * d  # minimiser inside the grid
        got = oracle.threshold(u, lam, d, pen)
        # the penalty of the group on the grid (Table 1 forms, c_k = sqrt 2)
        nb = np.linalg.norm(flat, axis=1)
        ck = math.sqrt(2.0)
        if kind == "grp.mcp":
            pv = np.where(nb <= par["gamma"] * lam * ck, lam * ck * nb - nb ** 2 / (2 * par["gamma"]),
                          par["gamma"] * (lam * ck) ** 2 / 2)
        elif kind == "grp.scad":
            lk, g = lam * ck, par["gamma"]
            pv = np.where(nb <= lk, lk * nb, np.where(nb <= g * lk, -(nb ** 2 - 2 * g * lk * nb + lk ** 2) / (2 * (g - 1)),
                                                      (g + 1) * lk ** 2 / 2))
        else:
            t = par["tau"]
            pv = lam * (1 - t) * ck * nb + lam * t * np.abs(flat).sum(1)
        f = 0.5 * d * np.sum((flat - u / d) ** 2, 1) + pv
        best = flat[np.argmin(f)]
        fg = 0.5 * d * np.sum((got - u / d) ** 2) + oracle.penalty_value(got, lam, pen)
        assert fg <= f.min() + 1e-9
        assert np.abs(got - best).max() <= 2 * (xs[1] - xs[0])


def test_special_cases_reduce_to_known_penalties():
    rng = np.random.default_rng(11)
    p = 10
    u = rng.standard_normal(p) * 2
    groups = _groups(p, 5)
    for lam, d in [(0.3, 1.0), (0.7, 2.5)]:
        g0 = oracle.threshold(u, lam, d, oracle.Penalty("sgl", groups=groups, tau=0.0))
        gl = oracle.threshold(u, lam, d, oracle.Penalty("grp.lasso", groups=groups))
        np.testing.assert_allclose(g0, gl, atol=1e-14)
        g1 = oracle.threshold(u, lam, d, oracle.Penalty("sgl", groups=groups, tau=1.0))
        la = oracle.threshold(u, lam, d, oracle.Penalty("lasso"))
        np.testing.assert_allclose(g1, la, atol=1e-14)
        single = np.arange(p)
        for gk, k in (("grp.mcp", "mcp"), ("grp.scad", "scad")):
            a = oracle.threshold(u, lam, d, oracle.Penalty(gk, groups=single, gamma=3.5))
            b = oracle.threshold(u, lam, d, oracle.Penalty(k, gamma=3.5))
            np.testing.assert_allclose(a, b, atol=1e-14)


@pytest.mark.parametrize("kind", ["grp.mcp", "grp.scad", "sgl"])
def test_lambda_max_gives_zero_and_is_tight(kind):
    rng = np.random.default_rng(13)
    p = 12
    c = rng.standard_normal(p)
    pen = oracle.Penalty(kind, groups=_groups(p, 4), tau=0.35,
                         w=rng.uniform(0.5, 1.5, p), gamma=3.0 if kind != "grp.scad" else 3.7)
    lm = oracle.lambda_max(c, pen)
    assert np.all(oracle.threshold(c, lm * (1 + 1e-12), 1.5, pen) == 0)
    assert np.any(oracle.threshold(c, 0.99 * lm, 1.5, pen) != 0)


def test_sgl_group_lambda_by_brute_force():
    rng = np.random.default_rng(17)
    for _ in range(5):
        cg = rng.standard_normal(4)
        w = rng.uniform(0.3, 2.0, 4)
        lamk = _sgl_group_lambda(cg, w, 1.3, 0.6)
        grid = np.linspace(0, 3 * lamk, 30001)
        ok = [np.linalg.norm(np.maximum(np.abs(cg) - l * 0.6 * w, 0)) <= l * 0.4 * 1.3 for l in grid]
        first = grid[np.argmax(ok)]
        assert abs(first - lamk) <= 2 * (grid[1] - grid[0])


@pytest.mark.parametrize("kind", ["grp.mcp", "grp.scad", "sgl"])
def test_paths_satisfy_kkt(kind):
    rng = np.random.default_rng(19)
    n, p = 600, 15
    X = rng.standard_normal((n, p))
    X[:, 1:] += 0.4 * X[:, :-1]
    y = X @ np.concatenate([[1.0, -0.8, 0.6], np.zeros(p - 3)]) + 0.5 * rng.standard_normal(n)
    G, c = X.T @ X / n, X.T @ y / n
    pen = oracle.Penalty(kind, groups=_groups(p, 3), tau=0.5,
                         gamma=3.0 if kind != "grp.scad" else 3.7)
    d = oracle.lanczos_d(G)[0]
    lams = oracle.lambda_grid(oracle.lambda_max(c, pen), 15, 1e-2)
    res = oracle.oem_path(G, c, d, pen, lams, tol=1e-12, max_iter=100000)
    assert res.converged.all()
    for l, lam in enumerate(lams):
        assert oracle.kkt_violation(G, c, res.beta[l], lam, pen) <= 1e-8, (kind, l)
    # a wrong point is caught
    bad = res.beta[-1].copy()
    bad[0] += 0.05
    assert oracle.kkt_violation(G, c, bad, lams[-1], pen) > 1e-3


def test_sgl_objective_monotone():
    rng = np.random.default_rng(23)
    n, p = 300, 9
    X = rng.standard_normal((n, p))
    y = X[:, 0] - X[:, 4] + rng.standard_normal(n)
    G, c, N = X.T @ X / n, X.T @ y / n, float(y @ y) / n
    pen = oracle.Penalty("sgl", groups=_groups(p, 3), tau=0.3)
    d = oracle.lanczos_d(G)[0]
    lam = 0.2 * oracle.lambda_max(c, pen)
    b = np.zeros(p)
    prev = oracle.objective(G, c, N, b, lam, pen)
    for _ in range(200):
        b = oracle.threshold(c + d * b - G @ b, lam, d, pen)
        cur = oracle.objective(G, c, N, b, lam, pen)
        assert cur <= prev + 1e-13
        prev = cur
