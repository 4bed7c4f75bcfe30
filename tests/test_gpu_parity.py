"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Sizes are small enough for the oracle to finish in seconds but span several
tiles with ragged tails (p = 70 and 130: two or three 64-column tiles, a 128
tile plus a tail; n not a multiple of any block). Tolerances:
  * Gram, float64 mode: relative Frobenius 1e-12 (float64 sums, different
    order); float32 mode: 2e-6 (float32 products and 256-row float32 sums);
  * d: within 1e-9 relative of the oracle's Lanczos d, and >= lambda_1;
  * paths: max |beta_gpu - beta_oracle| <= 1e-5 * max(1, ||beta||_inf)
    (both stop at tol = 1e-7 of the same fixed point; the GPU iterates in
    float32 on the downcast Gram with a compensated running u);
  * lambda grid: 1e-12 relative; CV error 1e-6 relative; selections exact.
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


def _rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _data(n, p, seed, dtype=np.float32, rho=0.5, sigma=1.0, head=(1.0, -0.8, 0.5, 0.0, 0.3)):
    X = synthgen.ar1_design(n, p, rho, seed, dtype)
    beta = synthgen.leading_beta(p, head[:p])
    y = synthgen.response(X, beta, sigma, seed, np.float64 if dtype == np.float64 else np.float32)
    return X, y


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _xdev(X):
    from paper_1801_09661_gb300 import padded
    return padded(X)


# ----------------------------------------------------------------------------- Gram

@pytest.mark.parametrize("mode,dtype,tol", [("fp64", np.float64, 1e-12), ("fp64", np.float32, 1e-12),
                                            ("fp32", np.float32, 2e-6)])
@pytest.mark.parametrize("n,p", [(5003, 70), (1, 3), (777, 130), (20000, 64)])
def test_gram_matches_oracle(oem, ctx, mode, dtype, tol, n, p):
    X, y = _data(n, p, 11 + p, dtype)
    G, c, yty = oem.oem_gram(ctx, _xdev(X), _dev(y), mode=mode)
    assert ctx.sync() == 0
    Gr, cr, Nr, _ = oracle.gram_sums(X, y)
    assert _rel_fro(G.cpu().numpy(), Gr) <= tol
    assert _rel_fro(c.cpu().numpy(), cr) <= tol
    assert abs(float(yty.cpu()[0]) - Nr) <= tol * abs(Nr)
    Gn = G.cpu().numpy()
    assert np.array_equal(Gn, Gn.T)


@pytest.mark.parametrize("K", [1, 5, 10])
def test_fold_grams_match_oracle(oem, ctx, K):
    n, p = 6007, 70
    X, y = _data(n, p, 5, np.float64)
    fold = synthgen.fold_ids(n, K, 5)
    Gk, ck, ytyk, nk = oem.oem_fold_grams(ctx, _xdev(X), _dev(y), _dev(fold), K, mode="fp64")
    assert ctx.sync() == 0
    Gr, cr, Nr, nr = oracle.fold_gram_sums(X, y, fold, K)
    assert np.array_equal(nk.cpu().numpy(), nr)
    for k in range(K):
        assert _rel_fro(Gk[k].cpu().numpy(), Gr[k]) <= 1e-12
        assert _rel_fro(ck[k].cpu().numpy(), cr[k]) <= 1e-12
        assert abs(float(ytyk[k].cpu()) - Nr[k]) <= 1e-12 * Nr[k]
    # fold identity on the device result (Section 3)
    G, c, yty = oem.oem_gram(ctx, _xdev(X), _dev(y), mode="fp64")
    ctx.sync()
    assert _rel_fro(Gk.sum(0).cpu().numpy(), G.cpu().numpy()) <= 1e-13


def test_fold_grams_with_an_empty_fold(oem, ctx):
    n, p, K = 900, 9, 4
    X, y = _data(n, p, 3, np.float64)
    fold = synthgen.fold_ids(n, 3, 3)  # labels 0..2 only: fold 3 is empty
    Gk, ck, ytyk, nk = oem.oem_fold_grams(ctx, _xdev(X), _dev(y), _dev(fold), K, mode="fp64")
    assert ctx.sync() == 0
    assert int(nk[3]) == 0 and float(Gk[3].abs().max()) == 0.0
    Gr, cr, Nr, nr = oracle.fold_gram_sums(X, y, fold, K)
    for k in range(3):
        assert _rel_fro(Gk[k].cpu().numpy(), Gr[k]) <= 1e-12


def test_nonfinite_input_is_reported(oem, ctx):
    X, y = _data(500, 8, 1, np.float32)
    X[17, 3] = np.nan
    oem.oem_gram(ctx, _xdev(X), _dev(y), mode="fp32")
    with pytest.raises(oem.OemError) as e:
        ctx.sync()
    assert e.value.code == oem.OEM_ENONFINITE
    assert ctx.sync() == 0  # the status word was cleared


# ----------------------------------------------------------------------------- d

@pytest.mark.parametrize("p", [1, 5, 64, 200])
def test_spectral_d(oem, ctx, p):
    X, y = _data(4 * p + 100, p, p, np.float64)
    G = X.T @ X / X.shape[0]
    d = oem.oem_spectral_d(ctx, _dev(G), steps=64)
    ctx.sync()
    dg = float(d.cpu()[0])
    dr, theta, r, m = oracle.lanczos_d(G, 64)
    lam1 = float(np.linalg.eigvalsh(G)[-1])
    assert dg >= lam1 * (1 - 1e-13)
    assert abs(dg - dr) <= 1e-7 * dr + 2 * r


def test_spectral_d_batched_and_zero(oem, ctx):
    p = 30
    Gs = []
    for s in range(3):
        X, _ = _data(300, p, 40 + s, np.float64)
        Gs.append(X.T @ X / 300)
    Gs.append(np.zeros((p, p)))
    d = oem.oem_spectral_d(ctx, _dev(np.stack(Gs)), steps=64).cpu().numpy()
    ctx.sync()
    for s in range(3):
        assert d[s] >= np.linalg.eigvalsh(Gs[s])[-1] * (1 - 1e-12)
        assert abs(d[s] - oracle.lanczos_d(Gs[s], 64)[0]) <= 1e-7 * d[s]
    assert d[3] == 1.0


# ----------------------------------------------------------------------------- paths

PENS = [("lasso", {}), ("enet", {"alpha": 0.5}), ("mcp", {"gamma": 3.0}), ("scad", {"gamma": 3.7}),
        ("grp.lasso", {})]


def _pens(p, kinds, gsize=5):
    groups = np.arange(p) // gsize
    gp, op = [], []
    for k, kw in kinds:
        g = groups if k in ("grp.lasso", "grp.mcp", "grp.scad", "sgl") else None
        gp.append(__import__("paper_1801_09661_gb300").Penalty(k, groups=g, **kw))
        op.append(oracle.Penalty(k, groups=g, **kw))
    return gp, op


def _check_paths(beta, lam, its, conv, G, c, d, opens, L, ratio, tol=1e-7, precision="f32", its_slack=0.1):
    for i, pen in enumerate(opens):
        lams = oracle.lambda_grid(oracle.lambda_max(c, pen), L, ratio)
        np.testing.assert_allclose(lam[i], lams, rtol=1e-12)
        ref = oracle.oem_path(G, c, d, pen, lams, tol=tol, max_iter=10000)
        scale = max(1.0, float(np.abs(ref.beta).max()))
        err = float(np.abs(beta[i] - ref.beta).max())
        assert err <= 1e-5 * scale, (pen.kind, err)
        assert conv[i].all() == ref.converged.all()
        # iteration counts agree closely (same rule, same fixed point)
        assert np.abs(its[i].astype(int) - ref.iters).max() <= max(5, its_slack * ref.iters.max())


@pytest.mark.parametrize("p,ncl", [(50, 0), (130, 0), (130, 1), (130, 4), (257, 16), (500, 0)])
def test_fit_path_matches_oracle(oem, ctx, p, ncl):
    n = 20 * p + 1000
    X, y = _data(n, p, 100 + p, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    d = oracle.lanczos_d(G)[0]
    gp, op = _pens(p, PENS)
    L, ratio = 30, 1e-2
    beta, lam, its, conv = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, d=d, nlambda=L,
                                            lambda_min_ratio=ratio, tol=1e-7, cluster_ctas=ncl)
    assert ctx.sync() == 0
    _check_paths(beta.cpu().numpy(), lam.cpu().numpy(), its.cpu().numpy(), conv.cpu().numpy(),
                 G, c, d, op, L, ratio)


def test_fit_path_float64_iteration(oem, ctx):
    p, n = 50, 3000
    X, y = _data(n, p, 3, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    d = oracle.lanczos_d(G)[0]
    gp, op = _pens(p, PENS[:2])
    beta, lam, its, conv = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, d=d, nlambda=25,
                                            lambda_min_ratio=1e-3, tol=1e-10,
                                            iter_precision="f64")
    assert ctx.sync() == 0
    for i, pen in enumerate(op):
        lams = oracle.lambda_grid(oracle.lambda_max(c, pen), 25, 1e-3)
        ref = oracle.oem_path(G, c, d, pen, lams, tol=1e-10, max_iter=10000)
        np.testing.assert_allclose(beta[i].cpu().numpy(), ref.beta, atol=1e-8)


def test_fit_path_lambda_above_max_gives_zero(oem, ctx):
    p, n = 20, 2000
    X, y = _data(n, p, 9, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    gp, op = _pens(p, PENS)
    lams = np.array([[oracle.lambda_max(c, pen) * f for f in (1.0, 1.5)] for pen in op])
    beta, lam, its, conv = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, nlambda=2, lambdas=lams)
    assert ctx.sync() == 0
    assert float(beta.abs().max()) == 0.0


def test_fit_path_kkt(oem, ctx):
    p, n = 60, 5000
    X, y = _data(n, p, 21, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    gp, op = _pens(p, PENS)
    beta, lam, its, conv = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, nlambda=20,
                                            lambda_min_ratio=1e-2, tol=1e-9)
    assert ctx.sync() == 0
    d = oracle.lanczos_d(G)[0]
    b = beta.cpu().numpy()
    lm = lam.cpu().numpy()
    for i, pen in enumerate(op):
        for l in range(20):
            v = oracle.kkt_violation(G, c, b[i, l], lm[i, l], pen)
            assert v <= max(1e-6, 10 * d * 1e-9 * max(1.0, np.abs(b[i, l]).max())) + 1e-5, (pen.kind, l, v)


# ----------------------------------------------------------------------------- oem() and xval

def test_fit_end_to_end_f64_lasso(oem, ctx):
    """The plain float64 lasso workload at its full size: n = 10,000, p = 50,
    AR(0.5), beta_1..5 = (2, -1.5, 1, -0.5, 0.25), sigma = 1, 100 lambdas to
    1e-3 lambda_max, tol 1e-7, float64 Gram and float64 iteration."""
    w = synthgen.WORKLOADS["lasso_f64_n1e4_p50"]
    X, y, _, _ = synthgen.make_data(w)
    beta, lam, its, conv, d = oem.oem_fit(ctx, _xdev(X), _dev(y), [oem.Penalty("lasso")],
                                          nlambda=100, lambda_min_ratio=1e-3, tol=1e-7,
                                          gram_mode="fp64", iter_precision="f64")
    assert ctx.sync() == 0
    G, c, N, n = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    dr = oracle.lanczos_d(G)[0]
    assert abs(float(d.cpu()[0]) - dr) <= 1e-7 * dr
    assert float(d.cpu()[0]) >= np.linalg.eigvalsh(G)[-1] * (1 - 1e-12)
    pen = oracle.Penalty("lasso")
    lams = oracle.lambda_grid(oracle.lambda_max(c, pen), 100, 1e-3)
    ref = oracle.oem_path(G, c, dr, pen, lams, tol=1e-7)
    b = beta[0].cpu().numpy()
    assert float(np.abs(b - ref.beta).max()) <= 1e-5 * max(1.0, np.abs(ref.beta).max())
    assert ((b != 0) == (ref.beta != 0)).mean() > 0.999


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_cv_matches_oracle(oem, ctx, mode):
    n, p, K = 12011, 40, 5
    X, y = _data(n, p, 77, np.float32, sigma=2.0, head=(-0.5, -0.5, 0.5, 0.5, 1.0))
    fold = synthgen.fold_ids(n, K, 77)
    kinds = PENS[:4]
    gp, op = _pens(p, kinds)
    L, ratio = 25, 1e-2
    out = oem.oem_cv(ctx, _xdev(X), _dev(y), _dev(fold), K, gp, nlambda=L, lambda_min_ratio=ratio,
                     tol=1e-7, gram_mode=mode)
    assert ctx.sync() == 0
    ref = oracle.xval(X, y, fold, K, op, nlambda=L, lambda_min_ratio=ratio, tol=1e-7)
    # the grid comes from c of the Gram pass: float32 sums carry ~1e-7 error
    np.testing.assert_allclose(out["lambdas"].cpu().numpy(), ref.lambdas,
                               rtol=1e-9 if mode == "fp64" else 2e-6)
    for i in range(len(op)):
        rb = ref.full[i].beta
        assert float(np.abs(out["beta"][i].cpu().numpy() - rb).max()) <= 1e-5 * max(1, np.abs(rb).max())
    np.testing.assert_allclose(out["cvm"].cpu().numpy(), ref.cvm, rtol=1e-5)
    np.testing.assert_allclose(out["cvsd"].cpu().numpy(), ref.cvsd, rtol=1e-3, atol=1e-7)
    # selections: exact unless the oracle's cvm has a near-tie at the choice
    imin = out["idx_min"].cpu().numpy()
    for i in range(len(op)):
        if imin[i] != ref.idx_min[i]:
            assert abs(ref.cvm[i, imin[i]] - ref.cvm[i, ref.idx_min[i]]) <= 1e-6 * ref.cvm[i].min()
    assert int(out["best_penalty"].cpu()[0]) == ref.best_penalty or \
        abs(ref.cvm[int(out["best_penalty"].cpu()[0])].min() - ref.cvm[ref.best_penalty].min()) <= 1e-6


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_iteration_layouts_give_identical_paths(oem, ctx, precision):
    # Each (row, instance) sum is formed in the same order whatever the
    # cluster size, cluster or grid mode, and however the penalties are
    # grouped into tasks, so every layout, and the one the autotuner picks,
    # returns the same bits.
    p, n = 130, 4000
    X, y = _data(n, p, 21, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    d = oracle.lanczos_d(G)[0]
    gp, op = _pens(p, PENS)
    runs = []
    for ncl, mg, tune in [(4, 8, False), (1, 1, False), (16, 1, False), (2, 2, False),
                          (8, 4, False), (32, 1, False), (24, 8, False), (30, 2, False),
                          (0, 0, True), (0, 0, True), (0, 0, False)]:
        out = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, d=d, nlambda=20, lambda_min_ratio=1e-2,
                               tol=1e-8, cluster_ctas=ncl, instances_per_task=mg, autotune=tune,
                               iter_precision=precision)
        assert ctx.sync() == 0
        runs.append([t.cpu().numpy() for t in out])
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            np.testing.assert_array_equal(a, b)
    _check_paths(*runs[0], G, c, d, op, 20, 1e-2, tol=1e-8)


GROUP_PENS = [("grp.lasso", {}), ("grp.mcp", {"gamma": 3.0}), ("grp.scad", {"gamma": 3.7}),
              ("sgl", {"tau": 0.5}), ("sgl", {"tau": 0.2}), ("lasso", {})]


@pytest.mark.parametrize("p,ncl", [(60, 0), (130, 4), (130, 40), (257, 16)])
def test_group_penalties_match_oracle(oem, ctx, p, ncl):
    # Eqs. gmcp, gscad, sglasso next to the group lasso and the lasso in one
    # launch (groups of 5; grid mode at 40 CTAs)
    n = 20 * p + 1000
    X, y = _data(n, p, 300 + p, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    d = oracle.lanczos_d(G)[0]
    gp, op = _pens(p, GROUP_PENS)
    L, ratio = 25, 1e-2
    # tol 1e-7: the float32 iteration resolves changes of beta to its ulp
    beta, lam, its, conv = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, d=d, nlambda=L,
                                            lambda_min_ratio=ratio, tol=1e-7, cluster_ctas=ncl)
    assert ctx.sync() == 0
    beta, lam, its, conv = (t.cpu().numpy() for t in (beta, lam, its, conv))
    _check_paths(beta, lam, its, conv, G, c, d, op, L, ratio, tol=1e-7)
    for i, pen in enumerate(op):
        kt = max(1e-6, 10 * oracle.effective_d(d, pen) * 1e-7 * max(1.0, np.abs(beta[i]).max()))
        for l in range(L):
            assert oracle.kkt_violation(G, c, beta[i, l], lam[i, l], pen) <= kt, (pen.kind, l)


def test_group_penalty_arguments_are_checked(oem, ctx):
    p = 20
    G, c = np.eye(p), np.ones(p)
    bad = [oem.Penalty("sgl", groups=np.arange(p) // 5, tau=1.5),
           oem.Penalty("grp.mcp", groups=np.arange(p) // 5, gamma=0.9),
           oem.Penalty("grp.scad", groups=np.arange(p) // 5, gamma=1.9),
           oem.Penalty("grp.mcp")]  # no groups
    for pen in bad:
        with pytest.raises(oem.OemError) as e:
            oem.oem_fit_path(ctx, _dev(G), _dev(c), [pen], d=1.0, nlambda=5)
        assert e.value.code == oem.OEM_EINVAL


def test_long_rows_and_group_slots_identical_across_layouts(oem, ctx):
    # p > 512: grid layouts with at most 16 rows per CTA run the 512-thread
    # variant (one G row per warp in registers), cluster layouts the 256-thread
    # one; group norms go through 32-lane slots of whole groups. The sums are
    # formed in the same order either way: every layout gives the same bits,
    # and the paths match the oracle.
    p, n = 700, 6000
    X, y = _data(n, p, 31, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    d = oracle.lanczos_d(G)[0]
    kinds = [("grp.lasso", {}), ("lasso", {}), ("grp.mcp", {"gamma": 3.0}), ("sgl", {"tau": 0.5})]
    gp, op = _pens(p, kinds, gsize=10)
    runs = []
    for ncl, mg in [(152, 1), (64, 2), (16, 1), (8, 4), (100, 1)]:
        out = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, d=d, nlambda=15, lambda_min_ratio=5e-2,
                               tol=1e-8, cluster_ctas=ncl, instances_per_task=mg, autotune=False)
        assert ctx.sync() == 0
        runs.append([t.cpu().numpy() for t in out])
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            np.testing.assert_array_equal(a, b)
    # at tol 1e-8 the float32 iteration's steps near convergence are a few
    # ulps of beta, so its stopping iteration may differ more from the
    # float64 oracle's
    _check_paths(*runs[0], G, c, d, op, 15, 5e-2, tol=1e-8, its_slack=0.25)


def test_groups_longer_than_a_warp_match_oracle(oem, ctx):
    # groups of 40 rows do not fit a 32-lane slot: their norms are taken by
    # one thread per group
    p, n = 200, 5000
    X, y = _data(n, p, 33, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    d = oracle.lanczos_d(G)[0]
    gp, op = _pens(p, [("grp.lasso", {}), ("grp.scad", {"gamma": 3.7})], gsize=40)
    out = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, d=d, nlambda=15, lambda_min_ratio=5e-2, tol=1e-8)
    assert ctx.sync() == 0
    _check_paths(*[t.cpu().numpy() for t in out], G, c, d, op, 15, 5e-2, tol=1e-8, its_slack=0.25)


def test_row_owned_kernel_layouts_identical(oem, ctx):
    # p above 1024: the row-owned kernel (each CTA thresholds its own rows and
    # sends its dbeta rows and maxima; grid mode through tagged words in
    # global memory). Cluster and grid layouts give the same bits.
    p, n = 1100, 6000
    X, y = _data(n, p, 35, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    d = oracle.lanczos_d(G)[0]
    kinds = [("grp.lasso", {}), ("lasso", {}), ("scad", {"gamma": 3.7})]
    gp, op = _pens(p, kinds, gsize=10)
    runs = []
    for ncl, mg in [(152, 1), (16, 1), (40, 4), (8, 2)]:
        out = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, d=d, nlambda=10, lambda_min_ratio=0.1,
                               tol=1e-7, cluster_ctas=ncl, instances_per_task=mg, autotune=False)
        assert ctx.sync() == 0
        runs.append([t.cpu().numpy() for t in out])
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            np.testing.assert_array_equal(a, b)
    _check_paths(*runs[0], G, c, d, op, 10, 0.1, tol=1e-7, its_slack=0.25)


def test_row_owned_unit_cache_overflow_identical(oem, ctx):
    # p = 2100 with 16- and 8-CTA clusters: a slice's Gram rows do not fit in
    # shared memory, so each CTA caches the 16-column blocks of G that nonzero
    # dbeta entries touch (zero blocks are skipped). At the small lambdas of a
    # dense lasso path more blocks are touched than the cache holds and the
    # rest come from L2. Every layout gives the bits of grid mode (one task of
    # both paths on 105 CTAs of 20 rows, every block of them cached).
    p, n = 2100, 2600
    X, y = _data(n, p, 41, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    d = oracle.lanczos_d(G)[0]
    gp, op = _pens(p, [("lasso", {}), ("grp.lasso", {})], gsize=10)
    runs = []
    for ncl, mg in [(105, 2), (16, 1), (8, 2), (16, 2)]:
        out = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, d=d, nlambda=5, lambda_min_ratio=0.02,
                               tol=1e-7, max_iter=300, cluster_ctas=ncl, instances_per_task=mg,
                               autotune=False)
        assert ctx.sync() in (0, 1)  # 1: some lambda stopped at max_iter
        runs.append([t.cpu().numpy() for t in out])
    # enough active columns at the last lambda to overflow every warp's cache
    assert int(np.count_nonzero(runs[0][0][0, -1])) > 600
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            np.testing.assert_array_equal(a, b)


def test_row_owned_kernel_beyond_4096_columns(oem, ctx):
    p, n = 4200, 9000
    X, y = _data(n, p, 37, np.float64)
    G, c, N, _ = oracle.gram_sums(X, y)
    G, c = G / n, c / n
    d = oracle.lanczos_d(G)[0]
    gp, op = _pens(p, [("lasso", {})])
    out = oem.oem_fit_path(ctx, _dev(G), _dev(c), gp, d=d, nlambda=4, lambda_min_ratio=0.3, tol=1e-7)
    assert ctx.sync() == 0
    _check_paths(*[t.cpu().numpy() for t in out], G, c, d, op, 4, 0.3, tol=1e-7)
