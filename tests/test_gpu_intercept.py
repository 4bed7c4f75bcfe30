"""GPU parity for the intercept / standardize options: the CUDA path (column
shifts, a column of ones in the same Gram pass, centring and scaling in the
assembly, paths on the standardized problem, back to the original scale)
against the oracle's ``fit`` / ``xval_intercept`` on the same data.

Tolerances: lambda grid 2e-6 relative (float32-input Gram modes; 1e-9 in
float64 mode); coefficients and intercepts 1e-5 * max(1, ||beta||_inf) (as
for the paths without centring); CV error 1e-5 relative. Columns have means
up to 40 standard deviations and scales from 0.3 to 4; one case puts the
means at 1e4 standard deviations, where centring after an unshifted split
Gram would lose every digit.
"""
import numpy as np
import pytest

import synthgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oem():
    import paper_1801_09661_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


@pytest.fixture(scope="module")
def ctx(oem):
    c = oem.Context(0)
    yield c
    c.close()


def _data(n, p, seed, mean_scale=40.0, dtype=np.float32):
    X = synthgen.ar1_design(n, p, 0.5, seed, np.float64)
    X = X * np.linspace(0.3, 4.0, p) + mean_scale * np.sin(np.arange(p) + 0.5)
    beta = synthgen.leading_beta(p, [1.0, -0.8, 0.5, 0.0, 0.3])
    y = synthgen.response(X, beta, 1.0, seed, np.float64) + 7.0
    return X.astype(dtype), y.astype(np.float32 if dtype != np.float64 else np.float64)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _xdev(X):
    from paper_1801_09661_gb300 import padded
    return padded(X)


def _close(a, ref, scale_floor=1.0, rel=1e-5):
    return float(np.abs(a - ref).max()) <= rel * max(scale_floor, float(np.abs(ref).max()))


@pytest.mark.parametrize("mode", ["auto", "fp32", "fp64"])
@pytest.mark.parametrize("intercept,standardize", [(True, True), (True, False), (False, True)])
def test_fit_matches_oracle(oem, ctx, mode, intercept, standardize):
    # Without standardisation the column scales 0.3..4 make the problem
    # ill-conditioned (d / lambda_min(G) ~ 500): the 1e-7 stopping rule then
    # leaves ~tol * 500 between two runs that stop at different iterations, so
    # those cases iterate in float64 to tol 1e-10. Without an intercept the
    # columns are zero-mean (scaling by the root second moment of columns with
    # large means would make G nearly rank one).
    n, p, L = 6007, 70, 20
    X, y = _data(n, p, 31, mean_scale=40.0 if intercept else 0.0,
                 dtype=np.float64 if mode == "fp64" else np.float32)
    kinds = [("lasso", {}), ("enet", {"alpha": 0.5}), ("mcp", {"gamma": 3.0})]
    gp = [oem.Penalty(k, **kw) for k, kw in kinds]
    op = [oracle.Penalty(k, **kw) for k, kw in kinds]
    tol, prec = (1e-7, "f32") if standardize else (1e-10, "f64")
    beta, lam, its, conv, d, beta0 = oem.oem_fit(ctx, _xdev(X), _dev(y), gp, nlambda=L,
                                                 lambda_min_ratio=1e-2, tol=tol, gram_mode=mode,
                                                 iter_precision=prec, max_iter=200_000,
                                                 intercept=intercept, standardize=standardize)
    assert ctx.sync() == 0
    ref = oracle.fit(X, y, op, intercept, standardize, nlambda=L, lambda_min_ratio=1e-2, tol=tol,
                     max_iter=200_000)
    np.testing.assert_allclose(lam.cpu().numpy(), ref.lambdas, rtol=1e-9 if mode == "fp64" else 2e-6)
    assert abs(float(d.cpu()[0]) - ref.d) <= 1e-6 * ref.d
    b, b0 = beta.cpu().numpy(), beta0.cpu().numpy()
    for i in range(len(kinds)):
        assert _close(b[i], ref.beta[i]), (kinds[i], float(np.abs(b[i] - ref.beta[i]).max()))
        assert _close(b0[i], ref.beta0[i]), (kinds[i], float(np.abs(b0[i] - ref.beta0[i]).max()))
    if not intercept:
        assert np.all(b0 == 0.0)


def test_bfloat16_input_with_intercept_runs_split(oem, ctx):
    n, p, L = 5003, 40, 15
    X, y = _data(n, p, 5, mean_scale=10.0)
    Xb = torch.from_numpy(X).cuda().to(torch.bfloat16)
    Xr = Xb.float().cpu().numpy()  # the bfloat16 values the GPU sees
    pen = [oem.Penalty("lasso")]
    beta, lam, its, conv, d, beta0 = oem.oem_fit(ctx, Xb, _dev(y), pen, nlambda=L,
                                                 lambda_min_ratio=1e-2, tol=1e-7, intercept=True,
                                                 standardize=True)
    assert ctx.sync() == 0
    ref = oracle.fit(Xr, y, [oracle.Penalty("lasso")], True, True, nlambda=L, lambda_min_ratio=1e-2,
                     tol=1e-7)
    assert _close(beta.cpu().numpy()[0], ref.beta[0])
    assert _close(beta0.cpu().numpy()[0], ref.beta0[0])


def test_large_means_keep_their_digits(oem, ctx):
    # column means 1e4 standard deviations away: the Gram pass runs on the
    # shifted data, so the centred statistics keep full precision (paths to
    # tol 1e-10 in float64 so that only the statistics can differ; convex
    # penalties, whose solutions move in proportion to the statistics)
    n, p, L = 8009, 24, 15
    X, y = _data(n, p, 12, mean_scale=1e4)
    pen = [oem.Penalty("lasso"), oem.Penalty("enet", alpha=0.5)]
    beta, lam, its, conv, d, beta0 = oem.oem_fit(ctx, _xdev(X), _dev(y), pen, nlambda=L,
                                                 lambda_min_ratio=1e-2, tol=1e-10, iter_precision="f64",
                                                 max_iter=100_000, intercept=True, standardize=True)
    assert ctx.sync() == 0
    ref = oracle.fit(X, y, [oracle.Penalty("lasso"), oracle.Penalty("enet", alpha=0.5)], True, True,
                     nlambda=L, lambda_min_ratio=1e-2, tol=1e-10, max_iter=100_000)
    np.testing.assert_allclose(lam.cpu().numpy(), ref.lambdas, rtol=2e-6)
    b = beta.cpu().numpy()
    for i in range(2):
        assert _close(b[i], ref.beta[i]), (i, float(np.abs(b[i] - ref.beta[i]).max()))
        # the intercept carries the 1e4 means: compare relative to them
        assert _close(beta0.cpu().numpy()[i], ref.beta0[i], scale_floor=1e4), \
            (i, float(np.abs(beta0.cpu().numpy()[i] - ref.beta0[i]).max()))


def test_constant_column_gets_zero(oem, ctx):
    n, p, L = 4001, 20, 10
    X, y = _data(n, p, 8)
    X[:, 7] = 3.25
    beta, lam, its, conv, d, beta0 = oem.oem_fit(ctx, _xdev(X), _dev(y), [oem.Penalty("lasso")],
                                                 nlambda=L, lambda_min_ratio=1e-2, tol=1e-7,
                                                 intercept=True, standardize=True)
    assert ctx.sync() == 0
    b = beta.cpu().numpy()
    assert np.all(b[0, :, 7] == 0.0)
    ref = oracle.fit(X, y, [oracle.Penalty("lasso")], True, True, nlambda=L, lambda_min_ratio=1e-2,
                     tol=1e-7)
    assert _close(b[0], ref.beta[0])
    assert _close(beta0.cpu().numpy()[0], ref.beta0[0])


@pytest.mark.parametrize("mode", ["auto", "fp64"])
def test_cv_with_intercept_matches_oracle(oem, ctx, mode):
    n, p, K, L = 9001, 40, 4, 15
    X, y = _data(n, p, 44, dtype=np.float64 if mode == "fp64" else np.float32)
    fold = synthgen.fold_ids(n, K, 44)
    kinds = [("lasso", {}), ("mcp", {"gamma": 3.0})]
    gp = [oem.Penalty(k, **kw) for k, kw in kinds]
    op = [oracle.Penalty(k, **kw) for k, kw in kinds]
    out = oem.oem_cv(ctx, _xdev(X), _dev(y), _dev(fold), K, gp, nlambda=L, lambda_min_ratio=1e-2,
                     tol=1e-7, gram_mode=mode, intercept=True, standardize=True)
    assert ctx.sync() == 0
    full, mse, cvm, cvsd, imin, i1se, best = oracle.xval_intercept(X, y, fold, K, op, True, True,
                                                                   nlambda=L, lambda_min_ratio=1e-2,
                                                                   tol=1e-7)
    np.testing.assert_allclose(out["lambdas"].cpu().numpy(), full.lambdas,
                               rtol=1e-9 if mode == "fp64" else 2e-6)
    b, b0 = out["beta"].cpu().numpy(), out["beta0"].cpu().numpy()
    for i in range(len(kinds)):
        assert _close(b[i], full.beta[i])
        assert _close(b0[i], full.beta0[i])
    np.testing.assert_allclose(out["cvm"].cpu().numpy(), cvm, rtol=1e-5)
    g_imin = out["idx_min"].cpu().numpy()
    for i in range(len(kinds)):
        if g_imin[i] != imin[i]:
            assert abs(cvm[i, g_imin[i]] - cvm[i, imin[i]]) <= 1e-6 * cvm[i].min()
