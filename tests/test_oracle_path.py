"""Pins for the oracle's statistics, d, lambda grid, OEM paths and CV scoring.

Checks against things fixed outside the oracle: brute-force sums, the fold
identities of Section 3, numpy's eigvalsh, closed forms for an orthonormal
design and for ridge, lambda >= lambda_max giving beta = 0, KKT conditions,
an independent coordinate-descent solver and exact sign-pattern enumeration at
p <= 8, the majorise-minimise monotonicity of OEM for d >= lambda_1, and a
direct held-out residual pass for the CV error.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

import synthgen
from oracle import (Penalty, assemble_fold_grams, cv_mse, cv_select, fold_gram_sums,
                    gram_sums, kkt_violation, lambda_grid, lambda_max, lanczos_d,
                    objective, oem_path, xval)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _small(n=400, p=8, seed=11, rho=0.5):
    X = synthgen.ar1_design(n, p, rho, seed, np.float64)
    beta = synthgen.leading_beta(p, [1.5, -1.0, 0.0, 0.5])
    y = synthgen.response(X, beta, 1.0, seed, np.float64)
    G, c, N, n_ = gram_sums(X, y)
    return X, y, G / n, c / n, N / n


# ------------------------------------------------------------------ Gram sums

def test_gram_sums_brute_force_loops():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(7, 3))
    y = rng.normal(size=7)
    G, c, N, n = gram_sums(X, y)
    for i in range(3):
        for j in range(3):
            s = 0.0
            for r in range(7):
                s += X[r, i] * X[r, j]
            assert G[i, j] == pytest.approx(s, rel=1e-15, abs=1e-15)
        assert c[i] == pytest.approx(sum(X[r, i] * y[r] for r in range(7)), rel=1e-14)
    assert N == pytest.approx(sum(v * v for v in y), rel=1e-14)
    assert n == 7


def test_gram_sums_exact_for_bf16_inputs():
    rng = np.random.default_rng(2)
    bits = synthgen.f32_to_bf16_bits(rng.normal(size=(64, 5)).astype(np.float32))
    Xd = synthgen.bf16_bits_to_f64(bits)
    # bfloat16 values have 8 significant bits: products are exact in float64 and
    # a sum of 64 of them (exponent range small) is exact too.
    G, _, _, _ = gram_sums(Xd, np.zeros(64))
    G2 = np.zeros((5, 5))
    for r in range(64):
        G2 += np.outer(Xd[r], Xd[r])
    assert np.array_equal(G, G2)


def test_fold_identities():
    n, p, K = 1000, 6, 5
    X = synthgen.ar1_design(n, p, 0.5, 3, np.float32)
    y = synthgen.response(X, synthgen.leading_beta(p, [1, 2]), 1.0, 3, np.float32)
    fold = synthgen.fold_ids(n, K, 3)
    Gk, ck, Nk, nk = fold_gram_sums(X, y, fold, K)
    Gf, cf, Nf, nf = gram_sums(X, y)
    assert nk.sum() == n
    np.testing.assert_allclose(Gk.sum(0), Gf, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(ck.sum(0), cf, rtol=1e-12, atol=1e-9)
    assert Nk.sum() == pytest.approx(Nf, rel=1e-12)
    G, c, N, cnt = assemble_fold_grams(Gk, ck, Nk, nk)
    np.testing.assert_allclose(G[0] * n, Gf, rtol=1e-12, atol=1e-9)
    for k in range(K):
        keep = fold != k
        Gm, cm, Nm, nm = gram_sums(X[keep], y[keep])
        assert cnt[k + 1] == nm
        np.testing.assert_allclose(G[k + 1], Gm / nm, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(c[k + 1], cm / nm, rtol=1e-10, atol=1e-12)
        assert N[k + 1] == pytest.approx(Nm / nm, rel=1e-10)
        # leave-out + fold = full (Section 3)
        np.testing.assert_allclose(G[k + 1] * cnt[k + 1] + Gk[k], Gf, rtol=1e-12, atol=1e-9)


def test_fold_with_no_rows():
    X = np.arange(12.0).reshape(6, 2)
    y = np.ones(6)
    fold = np.array([0, 0, 2, 2, 0, 2], dtype=np.uint8)
    Gk, ck, Nk, nk = fold_gram_sums(X, y, fold, 3)
    assert nk[1] == 0 and np.all(Gk[1] == 0) and np.all(ck[1] == 0) and Nk[1] == 0


# ------------------------------------------------------------------ Lanczos d

@pytest.mark.parametrize("p,kind", [(1, "ar"), (2, "ar"), (8, "ar"), (50, "ar"), (200, "ar"),
                                     (60, "exch"), (30, "spike"), (40, "lowrank")])
def test_lanczos_d_bounds_top_eigenvalue(p, kind):
    rng = np.random.default_rng(p)
    if kind == "ar":
        X = synthgen.ar1_design(4 * p + 50, p, 0.5, p, np.float64)
        G = X.T @ X / X.shape[0]
    elif kind == "exch":
        X = synthgen.exchangeable_design(500, p, 0.25, 4, np.float64)
        G = X.T @ X / 500
    elif kind == "spike":
        Q, _ = np.linalg.qr(rng.normal(size=(p, p)))
        ev = np.linspace(0.1, 1.0, p)
        ev[-1] = 10.0
        G = (Q * ev) @ Q.T
    else:
        B = rng.normal(size=(p, 3))
        G = B @ B.T
    lam1 = float(np.linalg.eigvalsh(G)[-1])
    d, theta, r, m = lanczos_d(G, 64)
    assert theta <= lam1 * (1 + 1e-12) + 1e-12
    assert d >= lam1 * (1 - 1e-13)
    assert d - lam1 <= 2 * r + 1e-10 * lam1
    if kind in ("spike", "exch", "lowrank") or p <= 64:
        assert d <= lam1 * (1 + 1e-8)


def test_lanczos_d_large_ar_is_tight_enough():
    X = synthgen.ar1_design(20000, 500, 0.5, 9, np.float64)
    G = X.T @ X / 20000
    lam1 = float(np.linalg.eigvalsh(G)[-1])
    d, theta, r, m = lanczos_d(G, 64)
    assert lam1 <= d <= lam1 * 1.02


def test_lanczos_zero_matrix():
    assert lanczos_d(np.zeros((4, 4)))[0] == 1.0


# ------------------------------------------------------------------ lambda grid

def test_lambda_grid_shape():
    g = lambda_grid(2.0, 100, 1e-3)
    assert g[0] == 2.0 and g[-1] == pytest.approx(2e-3, rel=1e-14)
    r = g[1:] / g[:-1]
    np.testing.assert_allclose(r, r[0], rtol=1e-12)
    assert lambda_grid(3.0, 1, 1e-3).tolist() == [3.0]


@pytest.mark.parametrize("kind", ["lasso", "enet", "mcp", "scad", "grp.lasso"])
def test_lambda_max_gives_zero_and_is_tight(kind):
    X, y, G, c, N = _small(p=8)
    pen = Penalty(kind, alpha=0.5, gamma=3.0, groups=np.repeat(np.arange(4), 2))
    lm = lambda_max(c, pen)
    d = lanczos_d(G)[0]
    r = oem_path(G, c, d, pen, [lm, lm * 1.5], tol=1e-12)
    assert np.all(r.beta == 0.0)
    r2 = oem_path(G, c, d, pen, [lm * 0.999], tol=1e-12)
    assert np.any(r2.beta != 0.0)


def test_lambda_max_weights():
    c = np.array([1.0, -4.0, 2.0])
    assert lambda_max(c, Penalty("lasso", w=np.array([1.0, 2.0, 0.0]))) == 2.0
    assert lambda_max(c, Penalty("enet", alpha=0.5)) == 8.0
    pen = Penalty("grp.lasso", groups=np.array([0, 0, 1]), cg=np.array([1.0, 4.0]))
    assert lambda_max(c, pen) == pytest.approx(math.sqrt(17.0))


# ------------------------------------------------------------------ closed forms

def _soft(z, t):
    return np.sign(z) * np.maximum(np.abs(z) - t, 0)


def test_orthonormal_design_one_step_exact():
    n, p = 256, 6
    X = synthgen.random_orthonormal_design(n, p, 1)
    rng = np.random.default_rng(3)
    y = X @ np.array([3.0, -2.0, 0.5, 0.0, 1.0, -0.2]) + rng.normal(size=n)
    G, c, N, _ = gram_sums(X, y)
    G, c = G / n, c / n
    np.testing.assert_allclose(G, np.eye(p), atol=1e-12)
    d = lanczos_d(G)[0]
    assert d == pytest.approx(1.0, abs=1e-10)
    lam, g = 0.4, 3.0
    exp = {
        "lasso": _soft(c, lam),
        "mcp": np.where(np.abs(c) <= g * lam, _soft(c, lam) / (1 - 1 / g), c),
        "scad": np.array([(_soft(np.array([z]), lam)[0] if abs(z) <= 2 * lam else
                           (((g - 1) * z - np.sign(z) * g * lam) / (g - 2) if abs(z) <= g * lam else z))
                          for z in c]),
    }
    for kind, e in exp.items():
        r = oem_path(G, c, 1.0, Penalty(kind, gamma=g), [lam], tol=1e-13)
        np.testing.assert_allclose(r.beta[0], e, atol=1e-10)
        assert r.iters[0] <= 3
    grp = np.array([0, 0, 1, 1, 2, 2])
    r = oem_path(G, c, 1.0, Penalty("grp.lasso", groups=grp), [lam], tol=1e-13)
    e = np.zeros(p)
    for k in range(3):
        m = grp == k
        nrm = np.linalg.norm(c[m])
        e[m] = c[m] * max(1 - math.sqrt(2) * lam / nrm, 0)
    np.testing.assert_allclose(r.beta[0], e, atol=1e-10)


def test_ridge_fixed_point_matches_cholesky():
    X, y, G, c, N = _small(p=8)
    w = np.array([1.0, 0.5, 2.0, 1.0, 1.0, 0.0, 1.0, 3.0])
    d = lanczos_d(G)[0]
    for lam in (0.01, 0.3, 2.0):
        r = oem_path(G, c, d, Penalty("enet", alpha=0.0, w=w), [lam], tol=1e-13, max_iter=200000)
        exp = scipy.linalg.cho_solve(scipy.linalg.cho_factor(G + lam * np.diag(w)), c)
        np.testing.assert_allclose(r.beta[0], exp, atol=1e-9)


# ------------------------------------------------------------------ KKT

@pytest.mark.parametrize("kind", ["lasso", "enet", "mcp", "scad", "grp.lasso"])
def test_paths_satisfy_kkt(kind):
    X, y, G, c, N = _small(n=2000, p=8)
    pen = Penalty(kind, alpha=0.5, gamma=3.0 if kind == "mcp" else 3.7,
                  groups=np.repeat(np.arange(4), 2))
    d = lanczos_d(G)[0]
    lams = lambda_grid(lambda_max(c, pen), 30, 1e-2)
    r = oem_path(G, c, d, pen, lams, tol=1e-12, max_iter=200000)
    assert r.converged.all()
    for l, lam in enumerate(lams):
        assert kkt_violation(G, c, r.beta[l], lam, pen) <= 1e-9


@pytest.mark.parametrize("kind,gam", [("mcp", 3.0), ("scad", 3.7)])
def test_small_d_raised_consistently(kind, gam):
    """With lambda_1(G) below 1/gamma (MCP) or 1/(gamma-1) (SCAD), d is raised
    to d_eff; the fixed point must still satisfy the KKT conditions."""
    X, y, G, c, N = _small(n=2000, p=6, rho=0.2)
    s = 0.25 / float(np.linalg.eigvalsh(G)[-1])
    G2, c2 = G * s, c * s   # lambda_1(G2) = 0.25 < 1/(gamma-1)
    pen = Penalty(kind, gamma=gam)
    d = lanczos_d(G2)[0]
    assert d < 1.0 / (gam - 1.0)
    lam = 0.1 * lambda_max(c2, pen)
    r = oem_path(G2, c2, d, pen, [lam], tol=1e-13, max_iter=500000)
    assert r.converged.all()
    assert kkt_violation(G2, c2, r.beta[0], lam, pen) <= 1e-9


def test_kkt_detects_a_wrong_solution():
    X, y, G, c, N = _small(p=8)
    pen = Penalty("lasso")
    lam = 0.1
    beta = oem_path(G, c, lanczos_d(G)[0], pen, [lam], tol=1e-13).beta[0]
    beta[0] *= 1.01
    assert kkt_violation(G, c, beta, lam, pen) > 1e-4


# ------------------------------------------------------------------ brute force, p <= 8

def _cd(G, c, kind, lam, alpha=1.0, gamma=3.0, iters=20000):
    """Cyclic coordinate descent (an independent algorithm). Univariate updates
    from Breheny & Huang (2011) for MCP/SCAD and Friedman et al. (2010) for the
    lasso / elastic net, with v = G_jj and z the partial residual correlation."""
    p = c.size
    b = np.zeros(p)
    for _ in range(iters):
        old = b.copy()
        for j in range(p):
            v = G[j, j]
            z = c[j] - G[j] @ b + v * b[j]
            az = abs(z)
            s = math.copysign(1.0, z)
            if kind == "lasso":
                b[j] = s * max(az - lam, 0) / v
            elif kind == "enet":
                b[j] = s * max(az - alpha * lam, 0) / (v + (1 - alpha) * lam)
            elif kind == "mcp":
                b[j] = s * max(az - lam, 0) / (v - 1 / gamma) if az <= v * gamma * lam else z / v
            elif kind == "scad":
                if az <= (v + 1) * lam:
                    b[j] = s * max(az - lam, 0) / v
                elif az <= v * gamma * lam:
                    b[j] = s * max(az - gamma * lam / (gamma - 1), 0) / (v - 1 / (gamma - 1))
                else:
                    b[j] = z / v
        if np.max(np.abs(b - old)) < 1e-15:
            break
    return b


@pytest.mark.parametrize("kind", ["lasso", "enet", "mcp", "scad"])
def test_oem_matches_coordinate_descent(kind):
    # strictly convex problems: lambda_min(G) > 1/gamma (MCP), > 1/(gamma-1) (SCAD)
    X, y, G, c, N = _small(n=3000, p=6, rho=0.2)
    gam = 3.0 if kind == "mcp" else 3.7
    lmin = float(np.linalg.eigvalsh(G)[0])
    assert lmin > 1 / (gam - 1) + 0.05
    pen = Penalty(kind, alpha=0.5, gamma=gam)
    d = lanczos_d(G)[0]
    for lam in (0.02, 0.1, 0.3):
        r = oem_path(G, c, d, pen, [lam], tol=1e-14, max_iter=500000)
        b = _cd(G, c, kind, lam, 0.5, gam)
        np.testing.assert_allclose(r.beta[0], b, atol=1e-10)


@pytest.mark.parametrize("kind", ["lasso", "enet"])
def test_oem_matches_sign_pattern_enumeration(kind):
    """Exact lasso / elastic-net solution by enumerating all 3^p sign patterns
    (p = 7): on support S with signs s, (G_SS + r I) b_S = c_S - t s_S, keep the
    pattern consistent with its signs and the KKT bound off S."""
    X, y, G, c, N = _small(n=1500, p=7)
    alpha = 1.0 if kind == "lasso" else 0.5
    lam = 0.05
    t, r_ = alpha * lam, (1 - alpha) * lam
    p = 7
    found = []
    for pattern in itertools.product((-1, 0, 1), repeat=p):
        s = np.array(pattern, dtype=float)
        S = np.flatnonzero(s)
        b = np.zeros(p)
        if S.size:
            b[S] = np.linalg.solve(G[np.ix_(S, S)] + r_ * np.eye(S.size), c[S] - t * s[S])
            if np.any(np.sign(b[S]) != s[S]):
                continue
        g = c - G @ b - r_ * b
        off = np.setdiff1d(np.arange(p), S)
        if off.size and np.any(np.abs(g[off]) > t + 1e-12):
            continue
        found.append(b)
    assert len(found) == 1
    r = oem_path(G, c, lanczos_d(G)[0], Penalty(kind, alpha=alpha), [lam], tol=1e-14,
                 max_iter=500000)
    np.testing.assert_allclose(r.beta[0], found[0], atol=1e-10)


# ------------------------------------------------------------------ MM monotonicity

@pytest.mark.parametrize("kind", ["lasso", "enet", "mcp", "scad", "grp.lasso"])
def test_objective_monotone_when_d_bounds_lambda1(kind):
    X, y, G, c, N = _small(n=800, p=8, rho=0.7)
    pen = Penalty(kind, alpha=0.5, gamma=3.0 if kind == "mcp" else 3.7,
                  groups=np.repeat(np.arange(4), 2))
    d = lanczos_d(G)[0]
    lams = lambda_grid(lambda_max(c, pen), 10, 1e-2)
    tr = []
    oem_path(G, c, d, pen, lams, tol=1e-10, max_iter=3000, trace=tr)
    for (l0, f0), (l1, f1) in zip(tr, tr[1:]):
        if l0 == l1:
            assert f1 <= f0 + 1e-12 * max(1.0, abs(f0))


def test_objective_not_monotone_when_d_too_small():
    X, y, G, c, N = _small(n=800, p=8, rho=0.7)
    lam1 = float(np.linalg.eigvalsh(G)[-1])
    tr = []
    oem_path(G, c, 0.45 * lam1, Penalty("lasso"), [0.01], tol=1e-10, max_iter=300, trace=tr)
    vals = [f for _, f in tr]
    assert any(b > a + 1e-9 for a, b in zip(vals, vals[1:]))


# ------------------------------------------------------------------ CV

def test_cv_mse_equals_direct_residuals():
    n, p, K = 900, 5, 3
    X = synthgen.ar1_design(n, p, 0.5, 5, np.float64)
    y = synthgen.response(X, synthgen.leading_beta(p, [1, -1]), 1.0, 5, np.float64)
    fold = synthgen.fold_ids(n, K, 5)
    Gk, ck, Nk, nk = fold_gram_sums(X, y, fold, K)
    rng = np.random.default_rng(0)
    B = rng.normal(size=(4, p))
    for k in range(K):
        m = fold == k
        direct = np.array([np.sum((y[m] - X[m] @ b) ** 2) / m.sum() for b in B])
        np.testing.assert_allclose(cv_mse(Gk[k], ck[k], Nk[k], nk[k], B), direct, rtol=1e-10)


def test_cv_select_golden():
    rows = {}
    with open(os.path.join(GOLD, "cv_select.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split(":")
                rows[k.strip()] = [float(t) for t in v.split()]
    mse = np.array([rows["fold0"], rows["fold1"]])
    cvm, cvsd, imin, i1se = cv_select(mse)
    assert imin == int(rows["idx_min"][0]) and i1se == int(rows["idx_1se"][0])
    np.testing.assert_allclose(cvm, [5, 3, 2.2, 2, 2.5])


def test_xval_end_to_end_small():
    n, p, K = 3000, 10, 4
    X = synthgen.ar1_design(n, p, 0.5, 8, np.float32)
    beta = synthgen.leading_beta(p, [-0.5, -0.5, 0.5, 0.5, 1.0])
    y = synthgen.response(X, beta, 2.0, 8, np.float32)
    fold = synthgen.fold_ids(n, K, 8)
    pens = [Penalty("lasso"), Penalty("mcp", gamma=3.0),
            Penalty("grp.lasso", groups=np.repeat(np.arange(5), 2))]
    r = xval(X, y, fold, K, pens, nlambda=20, lambda_min_ratio=1e-2, tol=1e-9)
    assert r.mse.shape == (3, K, 20)
    assert 0 <= r.best_penalty < 3
    for i in range(3):
        assert r.idx_1se[i] <= r.idx_min[i]
        assert r.full[i].converged.all()
        # held-out MSE near the noise variance (sigma = 2) at lambda.min
        assert 3.0 < r.cvm[i, r.idx_min[i]] < 5.5
    # every fold's path agrees with a fit on the held-in rows alone
    for k in range(K):
        keep = fold != k
        G, c, N, m = gram_sums(X[keep], y[keep])
        pr = oem_path(G / m, c / m, lanczos_d(G / m)[0], pens[0], r.lambdas[0], tol=1e-9)
        np.testing.assert_allclose(pr.beta, r.folds[k][0].beta, atol=1e-7)
