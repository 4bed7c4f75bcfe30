"""Parity at the full sizes of the named workloads, through the C ABI.

The bar (each against the FP64 oracle): Gram relative Frobenius <= 1e-6;
coefficients max |beta_gpu - beta_oracle| <= 1e-5 max(1, ||beta||_inf) at
every lambda; KKT violation <= 1e-6 (the raw bar; where the stopping rule
cannot guarantee it the test says so and holds the residual that rule
bounds, max(1e-6, 10 d tol max(1, ||beta||_inf))); supports identical except
where the oracle's |u| / d is within 1e-6 of a threshold (support_band).
Two error sources are checked apart and together: the Gram pass (GPU Gram
against the exact oracle Gram), the iteration (the oracle re-run on the GPU's
own Gram against the GPU path), and end to end (the oracle on the exact Gram
against the GPU path).

* four_penalties_f32_n1e6_p500 — oem_fit with default options (split-BF16
  Gram, autotuned iteration layout), as bench.py times it.
* cv10_f32_n4e6_p200 — 10-fold CV in one pass: every fold Gram against the
  exact oracle fold Gram; full-data paths, cvm, cvsd, selections against the
  oracle's CV on the GPU's fold statistics and on the exact ones.
* group_lasso_bf16_n2e6_p2000 — the oracle's float64 Gram of all 2e6 rows
  (row blocks), d, and the first 30 lambdas of the group lasso path
  (Section 2.2, Eq. glasso) on the GPU's Gram and on the exact one, held to
  1e-5 or to twice the oracle's own stopping band where that is larger (the
  band, measured here against the oracle at tol 1e-10, exceeds 1e-5 on this
  ill-conditioned design); KKT at every lambda of the GPU path.
Each test prints its measured errors (pytest -s shows them).
"""
import time

import numpy as np
import pytest

import oracle
import synthgen
from support_band import support_mismatches

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COEF_TOL = 1e-5
KKT_TOL = 1e-6


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


def _stop_residual(d, tol, beta):
    """The KKT residual the stopping rule bounds (d times its step bound)."""
    return max(KKT_TOL, 10.0 * d * tol * max(1.0, float(np.abs(beta).max())))


def _coef_err(b, ref):
    """max |b - ref| over the path, in units of max(1, ||ref||_inf)."""
    return float(np.abs(b - ref).max()) / max(1.0, float(np.abs(ref).max()))


def _check_support(G, c, d, pen, lams, beta_gpu, beta_ref, what):
    n_in = 0
    for l, lam in enumerate(lams):
        out, inside = support_mismatches(G, c, d, pen, lam, beta_gpu[l], beta_ref[l])
        assert not out, (what, pen.kind, l, out[:5])
        n_in += len(inside)
        if inside:
            print(f"  {what} {pen.kind} lambda {l}: support differs inside the band at {inside[:5]}")
    return n_in


def _kkt(G, c, beta, lams, pen, d, tol, what):
    """Largest KKT violation along the path; asserts the raw 1e-6 bar, or
    the stopping rule's residual where that is larger (printed)."""
    worst, over = 0.0, 0
    for l, lam in enumerate(lams):
        v = oracle.kkt_violation(G, c, beta[l], lam, pen)
        worst = max(worst, v)
        if v > KKT_TOL:
            over += 1
            assert v <= _stop_residual(d, tol, beta[l]), (what, pen.kind, l, v)
    print(f"  {what} {pen.kind}: max KKT violation {worst:.2e}"
          + (f" (above 1e-6 at {over} lambdas, within the stopping rule's residual)" if over else ""))
    return worst


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
    gerr = _rel_fro(Gg, G)
    print(f"\n  Gram rel. Frobenius {gerr:.2e}, c rel. {np.linalg.norm(cg - c) / np.linalg.norm(c):.2e}")
    assert gerr <= 1e-6
    assert float(np.linalg.norm(cg - c) / np.linalg.norm(c)) <= 1e-6
    G, c, Gg, cg = G / n, c / n, Gg / n, cg / n
    lam1 = float(np.linalg.eigvalsh(G)[-1])
    d_or = oracle.lanczos_d(Gg)[0]
    d_ex = oracle.lanczos_d(G)[0]
    assert d >= lam1 * (1 - 1e-9)
    assert abs(d - d_or) <= 1e-7 * d_or + 1e-6 * lam1
    assert conv.all()
    for i, pen in enumerate(op):
        lams = oracle.lambda_grid(oracle.lambda_max(cg, pen), w.nlambda, w.lambda_min_ratio)
        np.testing.assert_allclose(lam[i], lams, rtol=1e-9)
        # the iteration: the oracle on the GPU's own Gram and d
        ref = oracle.oem_path(Gg, cg, d, pen, lams, tol=w.tol, max_iter=10000)
        e_it = _coef_err(beta[i], ref.beta)
        # end to end: the oracle on the exact Gram, its own d and grid
        lams_e = oracle.lambda_grid(oracle.lambda_max(c, pen), w.nlambda, w.lambda_min_ratio)
        ref_e = oracle.oem_path(G, c, d_ex, pen, lams_e, tol=w.tol, max_iter=10000)
        e_e2e = _coef_err(beta[i], ref_e.beta)
        print(f"  {pen.kind}: coefficient error {e_it:.2e} on the GPU Gram, {e_e2e:.2e} end to end")
        assert e_it <= COEF_TOL, pen.kind
        assert e_e2e <= COEF_TOL, pen.kind
        _check_support(Gg, cg, d, pen, lams, beta[i], ref.beta, "GPU Gram")
        _check_support(G, c, d_ex, pen, lams_e, beta[i], ref_e.beta, "exact Gram")
        _kkt(G, c, beta[i], lam[i], pen, d, w.tol, "exact Gram")


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
    beta_g = out["beta"].cpu().numpy()
    cvm_g, cvsd_g = out["cvm"].cpu().numpy(), out["cvsd"].cpu().numpy()
    imin_g = out["idx_min"].cpu().numpy()
    # every fold Gram against the exact oracle fold Gram
    Gk, ck, Nk, nk = oracle.fold_gram_sums(X, y, fold, K)
    np.testing.assert_array_equal(nk_g, nk)
    worst = max(_rel_fro(Gk_g[k], Gk[k]) for k in range(K))
    print(f"\n  fold Grams: worst rel. Frobenius {worst:.2e}")
    assert worst <= 1e-6
    L = w.nlambda
    # the oracle's CV (Section 3) on the GPU's fold statistics (two-stage),
    # then on the exact ones (end to end)
    for what, stats in (("GPU fold Grams", (Gk_g, ck_g, Nk_g, nk_g)), ("exact fold Grams", (Gk, ck, Nk, nk))):
        G, c, N, cnt = oracle.assemble_fold_grams(*stats)
        d = np.array([oracle.lanczos_d(G[b])[0] for b in range(K + 1)])
        lams = np.array([oracle.lambda_grid(oracle.lambda_max(c[0], pen), L, w.lambda_min_ratio)
                         for pen in op])
        np.testing.assert_allclose(out["lambdas"].cpu().numpy(), lams,
                                   rtol=1e-9 if what.startswith("GPU") else 1e-6)
        mse = np.zeros((len(op), K, L))
        for i, pen in enumerate(op):
            full = oracle.oem_path(G[0], c[0], d[0], pen, lams[i], tol=w.tol)
            e = _coef_err(beta_g[i], full.beta)
            print(f"  {what} {pen.kind}: full-data coefficient error {e:.2e}")
            assert e <= COEF_TOL, (what, pen.kind)
            _check_support(G[0], c[0], d[0], pen, lams[i], beta_g[i], full.beta, what)
            if not what.startswith("GPU"):
                _kkt(G[0], c[0], beta_g[i], lams[i], pen, d[0], w.tol, what)
            for k in range(K):
                fk = oracle.oem_path(G[k + 1], c[k + 1], d[k + 1], pen, lams[i], tol=w.tol)
                mse[i, k] = oracle.cv_mse(stats[0][k], stats[1][k], stats[2][k], stats[3][k], fk.beta)
        for i in range(len(op)):
            cvm, cvsd, imin, i1se = oracle.cv_select(mse[i])
            rel = float(np.abs(cvm_g[i] - cvm).max() / cvm.min())
            print(f"  {what} {op[i].kind}: cvm rel. error {rel:.2e}")
            assert rel <= 1e-6, (what, op[i].kind)
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
    del Xd
    beta, lam, its, conv = (t.cpu().numpy() for t in (beta, lam, its, conv))
    d = float(d.cpu()[0])
    Gg, cg = Gg.cpu().numpy(), cg.cpu().numpy()
    assert conv.all() and its.max() < 10000
    # the exact float64 Gram of all rows (oracle.gram_sums over row blocks)
    t0 = time.time()
    n, p = w.n, w.p
    G = np.zeros((p, p))
    c = np.zeros(p)
    blk = 50_000
    for r0 in range(0, n, blk):
        Gb, cb, _, _ = oracle.gram_sums(synthgen.bf16_bits_to_f64(X[r0:r0 + blk]), y[r0:r0 + blk])
        G += Gb
        c += cb
    gerr = _rel_fro(Gg, G)
    cerr = float(np.linalg.norm(cg - c) / np.linalg.norm(c))
    print(f"\n  exact Gram in {time.time() - t0:.1f} s; Gram rel. Frobenius {gerr:.2e}, c rel. {cerr:.2e}")
    assert gerr <= 1e-6 and cerr <= 1e-6
    G, c, Gg, cg = G / n, c / n, Gg / n, cg / n
    lam1 = float(np.linalg.eigvalsh(Gg)[-1])
    assert lam1 <= d <= lam1 * (1 + 1e-6)
    d_ex = oracle.lanczos_d(G)[0]
    assert d >= float(np.linalg.eigvalsh(G)[-1]) * (1 - 1e-6)
    pen = op[0]
    lams = oracle.lambda_grid(oracle.lambda_max(cg, pen), w.nlambda, w.lambda_min_ratio)
    np.testing.assert_allclose(lam[0], lams, rtol=1e-9)
    # KKT of the GPU path on the GPU's Gram at every lambda, and on the exact
    # Gram
    _kkt(Gg, cg, beta[0], lam[0], pen, d, w.tol, "GPU Gram")
    _kkt(G, c, beta[0], lam[0], pen, d, w.tol, "exact Gram")
    # the oracle's path for the first 30 lambdas on the GPU's Gram and on the
    # exact one (the oracle's group threshold is a plain loop: ~1 ms per
    # iteration at p = 2000)
    L30 = 30
    t0 = time.time()
    ref = oracle.oem_path(Gg, cg, d, pen, lams[:L30], tol=w.tol, max_iter=10000)
    lams_e = oracle.lambda_grid(oracle.lambda_max(c, pen), w.nlambda, w.lambda_min_ratio)
    ref_e = oracle.oem_path(G, c, d_ex, pen, lams_e[:L30], tol=w.tol, max_iter=10000)
    # On this design (d / lambda_min of the active block up to ~1,350) the
    # stopping rule leaves the oracle itself short of the minimiser by more
    # than 1e-5 || beta ||_inf at the later lambdas: its band per lambda is the
    # distance between the oracle at tol 1e-7 and at tol 1e-10. Two correct
    # iterations that stop by the same rule may differ by up to twice it.
    ref_t = oracle.oem_path(Gg, cg, d, pen, lams[:L30], tol=1e-10, max_iter=200000)
    scale = max(1.0, float(np.abs(ref_t.beta).max()))
    band = np.abs(ref.beta - ref_t.beta).max(axis=1) / scale
    bar = np.maximum(COEF_TOL, 2.0 * band)
    e_it = np.abs(beta[0, :L30] - ref.beta).max(axis=1) / scale
    e_e2e = np.abs(beta[0, :L30] - ref_e.beta).max(axis=1) / scale
    print(f"  oracle paths ({int(ref.iters.sum())} + {int(ref_e.iters.sum())} + {int(ref_t.iters.sum())} "
          f"iterations) in {time.time() - t0:.1f} s")
    print(f"  coefficient error: max {e_it.max():.2e} on the GPU Gram, {e_e2e.max():.2e} end to end; "
          f"oracle's own stopping band up to {band.max():.2e}; "
          f"lambdas above 1e-5: {int((e_it > COEF_TOL).sum())} (GPU Gram), {int((e_e2e > COEF_TOL).sum())} (end to end)")
    assert (e_it <= bar).all(), list(zip(e_it, bar))
    assert (e_e2e <= bar).all(), list(zip(e_e2e, bar))
    _check_support(Gg, cg, d, pen, lams[:L30], beta[0, :L30], ref.beta, "GPU Gram")
    _check_support(G, c, d_ex, pen, lams_e[:L30], beta[0, :L30], ref_e.beta, "exact Gram")
