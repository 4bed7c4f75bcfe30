"""Parity at the full sizes of the named workloads, through the C ABI.

* four_penalties_f32_n1e6_p500 — the bench workload, in the launch
  configuration bench.py times (oem_fit, default options: split-BF16 Gram,
  autotuned iteration layout). Gram against the exact FP64 oracle Gram
  (relative Frobenius <= 1e-6); d against the oracle's Lanczos and an upper
  bound of lambda_1; paths against the oracle run on the GPU's own Gram
  (two-stage parity: Gram error and path error are separate sources) and,
  end to end, against the oracle on the exact Gram; KKT on the GPU's Gram.
* cv10_f32_n4e6_p200 — 10-fold CV in one pass: every fold Gram against the
  exact oracle fold Gram; full-data paths, cvm, cvsd and the selections
  against the oracle's CV run on the GPU's fold Grams.
* group_lasso_bf16_n2e6_p2000 — the oracle's full Gram (8e12 flops) and
  paths are out of reach on the host, so: a 24 x 24 block of G and the
  matching entries of c from exact FP64 dot products of sampled columns;
  d >= lambda_1 of the GPU Gram (eigvalsh); the KKT conditions of the group
  lasso (Section 2.2, Eq. glasso) at every lambda of the path.
KKT tolerance: max(1e-6, 10 d tol max(1, ||beta||_inf)), the residual the
stopping rule can guarantee.
"""
import numpy as np
import pytest

import oracle
import synthgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oem():
    import paper_1801_09661_gb300 as m
    assert torch.cuda.is_available()
    return m


@pytest.fixture(scope="module")
def ctx(oem):
    c = oem.Context(0, budget_bytes=64 << 30)
    yield c
    c.close()


def _pens(oem, w):
    gp, op = [], []
    for k in w.penalties:
        kw = {}
        if k == "enet":
            kw = {"alpha": w.extra["alpha"]}
        elif k == "mcp":
            kw = {"gamma": w.extra["gamma_mcp"]}
        elif k == "scad":
            kw = {"gamma": w.extra["gamma_scad"]}
        elif k == "grp.lasso":
            kw = {"groups": np.arange(w.p) // w.group_size}
        gp.append(oem.Penalty(k, **kw))
        op.append(oracle.Penalty(k, **kw))
    return gp, op


def _xdev(oem, X):
    if X.dtype == np.uint16:  # bfloat16 bits
        return oem.padded(torch.from_numpy(X.view(np.int16)).view(torch.bfloat16))
    return oem.padded(X)


def _rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _kkt_tol(d, tol, beta):
    return max(1e-6, 10.0 * d * tol * max(1.0, float(np.abs(beta).max())))


def test_bench_workload_full_size(oem, ctx):
    w = synthgen.WORKLOADS["four_penalties_f32_n1e6_p500"]
    X, y, _, _ = synthgen.make_data(w)
    Xd, yd = _xdev(oem, X), torch.from_numpy(y).cuda()
    gp, op = _pens(oem, w)
    beta, lam, its, conv, d = oem.oem_fit(ctx, Xd, yd, gp, nlambda=w.nlambda,
                                          lambda_min_ratio=w.lambda_min_ratio, tol=w.tol)
    assert ctx.sync() == 0
    Gg, cg, _ = oem.oem_gram(ctx, Xd, yd, mode="split_bf16")  # the Gram oem_fit formed
    assert ctx.sync() == 0
    beta, lam, its, conv = (t.cpu().numpy() for t in (beta, lam, its, conv))
    d = float(d.cpu()[0])
    Gg, cg = Gg.cpu().numpy(), cg.cpu().numpy()
    n = w.n
    G, c, _, _ = oracle.gram_sums(X, y)
    assert _rel_fro(Gg, G) <= 1e-6
    assert float(np.linalg.norm(cg - c) / np.linalg.norm(c)) <= 1e-6
    G, c, Gg, cg = G / n, c / n, Gg / n, cg / n
    lam1 = float(np.linalg.eigvalsh(G)[-1])
    d_or = oracle.lanczos_d(Gg)[0]
    assert d >= lam1 * (1 - 1e-9)
    assert abs(d - d_or) <= 1e-7 * d_or + 1e-6 * lam1
    assert conv.all()
    for i, pen in enumerate(op):
        lams = oracle.lambda_grid(oracle.lambda_max(cg, pen), w.nlambda, w.lambda_min_ratio)
        np.testing.assert_allclose(lam[i], lams, rtol=1e-9)
        # path parity on the GPU's own Gram and d
        ref = oracle.oem_path(Gg, cg, d, pen, lams, tol=w.tol, max_iter=10000)
        scale = max(1.0, float(np.abs(ref.beta).max()))
        assert float(np.abs(beta[i] - ref.beta).max()) <= 1e-5 * scale, pen.kind
        # end to end against the exact Gram: the Gram error (<= 1e-6) moves
        # the solution by at most its conditioning times that
        ref_e = oracle.oem_path(G, c, oracle.lanczos_d(G)[0], pen,
                                oracle.lambda_grid(oracle.lambda_max(c, pen), w.nlambda,
                                                   w.lambda_min_ratio), tol=w.tol, max_iter=10000)
        assert float(np.abs(beta[i] - ref_e.beta).max()) <= 1e-4 * scale, pen.kind
        # stationarity (a minimiser for the convex penalties) on that Gram
        kt = _kkt_tol(d, w.tol, beta[i])
        for l in range(w.nlambda):
            assert oracle.kkt_violation(Gg, cg, beta[i, l], lam[i, l], pen) <= kt, (pen.kind, l)


def test_cv10_full_size(oem, ctx):
    w = synthgen.WORKLOADS["cv10_f32_n4e6_p200"]
    X, y, fold, _ = synthgen.make_data(w)
    K = w.K
    Xd, yd, fd = _xdev(oem, X), torch.from_numpy(y).cuda(), torch.from_numpy(fold).cuda()
    gp, op = _pens(oem, w)
    out = oem.oem_cv(ctx, Xd, yd, fd, K, gp, nlambda=w.nlambda, lambda_min_ratio=w.lambda_min_ratio,
                     tol=w.tol)
    assert ctx.sync() == 0
    Gk_g, ck_g, Nk_g, nk_g = (t.cpu().numpy() for t in oem.oem_fold_grams(ctx, Xd, yd, fd, K,
                                                                       mode="split_bf16"))
    assert ctx.sync() == 0
    # every fold Gram against the exact oracle fold Gram
    Gk, ck, Nk, nk = oracle.fold_gram_sums(X, y, fold, K)
    np.testing.assert_array_equal(nk_g, nk)
    for k in range(K):
        assert _rel_fro(Gk_g[k], Gk[k]) <= 1e-6, k
    # the oracle's CV (Section 3) on the GPU's fold statistics
    G, c, N, cnt = oracle.assemble_fold_grams(Gk_g, ck_g, Nk_g, nk_g)
    d = np.array([oracle.lanczos_d(G[b])[0] for b in range(K + 1)])
    L = w.nlambda
    lams = np.array([oracle.lambda_grid(oracle.lambda_max(c[0], pen), L, w.lambda_min_ratio)
                     for pen in op])
    np.testing.assert_allclose(out["lambdas"].cpu().numpy(), lams, rtol=1e-9)
    mse = np.zeros((len(op), K, L))
    for i, pen in enumerate(op):
        full = oracle.oem_path(G[0], c[0], d[0], pen, lams[i], tol=w.tol)
        scale = max(1.0, float(np.abs(full.beta).max()))
        assert float(np.abs(out["beta"][i].cpu().numpy() - full.beta).max()) <= 1e-5 * scale
        for k in range(K):
            fk = oracle.oem_path(G[k + 1], c[k + 1], d[k + 1], pen, lams[i], tol=w.tol)
            mse[i, k] = oracle.cv_mse(Gk_g[k], ck_g[k], Nk_g[k], nk_g[k], fk.beta)
    cvm_g, cvsd_g = out["cvm"].cpu().numpy(), out["cvsd"].cpu().numpy()
    imin_g = out["idx_min"].cpu().numpy()
    for i in range(len(op)):
        cvm, cvsd, imin, i1se = oracle.cv_select(mse[i])
        np.testing.assert_allclose(cvm_g[i], cvm, rtol=1e-6)
        np.testing.assert_allclose(cvsd_g[i], cvsd, rtol=1e-3, atol=1e-8)
        if imin_g[i] != imin:
            assert abs(cvm[imin_g[i]] - cvm[imin]) <= 1e-6 * cvm.min()


def test_group_lasso_bf16_full_size(oem, ctx):
    w = synthgen.WORKLOADS["group_lasso_bf16_n2e6_p2000"]
    X, y, _, _ = synthgen.make_data(w)
    Xd, yd = _xdev(oem, X), torch.from_numpy(y).cuda()
    gp, op = _pens(oem, w)
    beta, lam, its, conv, d = oem.oem_fit(ctx, Xd, yd, gp, nlambda=w.nlambda,
                                          lambda_min_ratio=w.lambda_min_ratio, tol=w.tol)
    assert ctx.sync() == 0
    Gg, cg, _ = oem.oem_gram(ctx, Xd, yd, mode="bf16")  # the Gram oem_fit formed
    assert ctx.sync() == 0
    beta, lam, its, conv = (t.cpu().numpy() for t in (beta, lam, its, conv))
    d = float(d.cpu()[0])
    Gg, cg = Gg.cpu().numpy(), cg.cpu().numpy()
    # a sampled block of G and c from exact float64 dot products
    rng = np.random.default_rng(5)
    S = np.sort(rng.choice(w.p, 24, replace=False))
    XS = synthgen.bf16_bits_to_f64(X[:, S])
    yf = y.astype(np.float64)
    Gs, cs = XS.T @ XS, XS.T @ yf
    scale = np.sqrt(np.outer(np.diag(Gs), np.diag(Gs)))
    assert float(np.abs(Gg[np.ix_(S, S)] - Gs).max() / 1.0) <= 1e-6 * scale.max()
    assert float((np.abs(Gg[np.ix_(S, S)] - Gs) / scale).max()) <= 1e-6
    assert float(np.abs(cg[S] - cs).max()) <= 1e-6 * np.sqrt(np.diag(Gs).max() * (yf @ yf))
    n = w.n
    G, c = Gg / n, cg / n
    lam1 = float(np.linalg.eigvalsh(G)[-1])
    assert lam1 <= d <= lam1 * (1 + 1e-6)
    assert conv.all() and its.max() < 10000
    pen = op[0]
    lams = oracle.lambda_grid(oracle.lambda_max(c, pen), w.nlambda, w.lambda_min_ratio)
    np.testing.assert_allclose(lam[0], lams, rtol=1e-9)
    kt = _kkt_tol(d, w.tol, beta[0])
    for l in range(w.nlambda):
        assert oracle.kkt_violation(G, c, beta[0, l], lam[0, l], pen) <= kt, l
