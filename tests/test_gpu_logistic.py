"""GPU parity for penalised logistic regression (Section 4, Hessian bound
1/4): the CUDA path (Gram pass over [X | y | 1], Lanczos d, one pass over X
per outer step for the score, resumed OEM launches for the surrogates)
against the oracle's ``logistic_path`` on the same data, plus the KKT
conditions of the penalised log-likelihood checked in float64 on the GPU's
own result.

Tolerances: lambda grid 1e-5 relative (the score at the null model uses a
float32 sigmoid, ~1e-7 relative); coefficients and intercepts
1e-5 * max(1, ||beta||_inf); KKT within 1e-5 (the outer stopping rule is
tol = 1e-7 on successive iterates, the inner iteration float32).
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


def _data(n, p, seed, dtype=np.float32):
    X = synthgen.ar1_design(n, p, 0.5, seed, np.float64)
    beta = np.zeros(p)
    beta[:4] = [1.0, -0.8, 0.6, 0.4]
    rng = np.random.default_rng(seed)
    prob = 1.0 / (1.0 + np.exp(-(X @ beta - 0.5)))
    y = (rng.random(n) < prob).astype(np.float64)
    return X.astype(dtype), y.astype(np.float64 if dtype == np.float64 else np.float32)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _xdev(X):
    from paper_1801_09661_gb300 import padded
    return padded(X)


def _close(a, ref, rel=1e-5):
    return float(np.abs(a - ref).max()) <= rel * max(1.0, float(np.abs(ref).max()))


KINDS = [("lasso", {}), ("enet", {"alpha": 0.5}), ("mcp", {"gamma": 3.0})]


@pytest.mark.parametrize("mode", ["auto", "fp64"])
@pytest.mark.parametrize("intercept", [True, False])
def test_logistic_matches_oracle(oem, ctx, mode, intercept):
    n, p, L = 6007, 30, 15
    X, y = _data(n, p, 21, dtype=np.float64 if mode == "fp64" else np.float32)
    gp = [oem.Penalty(k, **kw) for k, kw in KINDS]
    beta, beta0, lam, its, conv, d = oem.oem_fit_logistic(ctx, _xdev(X), _dev(y), gp, nlambda=L,
                                                          lambda_min_ratio=2e-2, tol=1e-7,
                                                          gram_mode=mode, intercept=intercept)
    assert ctx.sync() == 0
    b, b0, lm = beta.cpu().numpy(), beta0.cpu().numpy(), lam.cpu().numpy()
    assert conv.cpu().numpy().all()
    for i, (k, kw) in enumerate(KINDS):
        ref = oracle.logistic_path(X, y, oracle.Penalty(k, **kw), nlambda=L, lambda_min_ratio=2e-2,
                                   intercept=intercept, tol=1e-7)
        np.testing.assert_allclose(lm[i], ref.lambdas, rtol=1e-5)
        assert abs(float(d.cpu()[0]) - ref.d) <= 1e-6 * ref.d
        assert _close(b[i], ref.beta), (k, float(np.abs(b[i] - ref.beta).max()))
        assert _close(b0[i], ref.beta0), (k, float(np.abs(b0[i] - ref.beta0).max()))
    if not intercept:
        assert np.all(b0 == 0.0)


def test_logistic_kkt_on_the_gpu_result(oem, ctx):
    n, p, L = 8009, 40, 12
    X, y = _data(n, p, 5)
    beta, beta0, lam, its, conv, d = oem.oem_fit_logistic(ctx, _xdev(X), _dev(y), [oem.Penalty("lasso")],
                                                          nlambda=L, lambda_min_ratio=2e-2, tol=1e-9,
                                                          iter_precision="f64", intercept=True)
    assert ctx.sync() == 0
    Xd, yd = X.astype(np.float64), y.astype(np.float64)
    for l, lm in enumerate(lam.cpu().numpy()[0]):
        bb, b0 = beta.cpu().numpy()[0, l], float(beta0.cpu().numpy()[0, l])
        r = yd - oracle.sigmoid(Xd @ bb + b0)
        assert abs(r.mean()) <= 1e-6
        g = Xd.T @ r / n
        on = bb != 0
        assert np.all(np.abs(g[on] - lm * np.sign(bb[on])) <= 1e-5 * max(1.0, lm))
        assert np.all(np.abs(g[~on]) <= lm * (1 + 1e-5) + 1e-7)


def test_logistic_bfloat16_input(oem, ctx):
    n, p, L = 5003, 24, 10
    X, y = _data(n, p, 9)
    Xb = torch.from_numpy(X).cuda().to(torch.bfloat16)
    Xr = Xb.float().cpu().numpy()
    beta, beta0, lam, its, conv, d = oem.oem_fit_logistic(ctx, Xb, _dev(y), [oem.Penalty("lasso")],
                                                          nlambda=L, lambda_min_ratio=2e-2, tol=1e-7,
                                                          intercept=True)
    assert ctx.sync() == 0
    ref = oracle.logistic_path(Xr, y, oracle.Penalty("lasso"), nlambda=L, lambda_min_ratio=2e-2,
                               intercept=True, tol=1e-7)
    assert _close(beta.cpu().numpy()[0], ref.beta)
    assert _close(beta0.cpu().numpy()[0], ref.beta0)


def test_logistic_rejects_what_it_does_not_support(oem, ctx):
    X, y = _data(500, 10, 1)
    with pytest.raises(oem.OemError):
        oem.oem_fit_logistic(ctx, _xdev(X), _dev(y), [oem.Penalty("lasso")], standardize=True)
    with pytest.raises(oem.OemError):
        oem.oem_fit_logistic(ctx, _xdev(X), _dev(y),
                             [oem.Penalty("grp.lasso", groups=np.repeat(np.arange(5), 2))])
