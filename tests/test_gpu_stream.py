"""GPU parity with X in host memory: the Gram pass streams X in row blocks
(pinned or pageable memory) through two device staging buffers and adds the
blocks' fold sums up (the paper's out-of-memory big.oem, Section 5.7, done as
a stream of row blocks; a memory-mapped file is one more kind of pageable
host memory).

Block sizes are forced small (OEM_STREAM_ROWS) so that every case runs
several blocks with a ragged last one. Tolerances are those of the
device-resident path for the same Gram mode (the sums are regrouped by block,
which changes only their rounding order): relative Frobenius 1e-12 in float64
mode, 1e-6 split-bfloat16 and bfloat16, 2e-6 float32; paths and CV as in the
device-resident parity tests.
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _data(n, p, seed, dtype=np.float32, mean_scale=0.0):
    X = synthgen.ar1_design(n, p, 0.5, seed, np.float64)
    if mean_scale:
        X = X * np.linspace(0.3, 4.0, p) + mean_scale * np.sin(np.arange(p) + 0.5)
    beta = synthgen.leading_beta(p, [1.0, -0.8, 0.5, 0.0, 0.3])
    y = synthgen.response(X, beta, 1.0, seed, np.float64) + (7.0 if mean_scale else 0.0)
    return X.astype(dtype), y.astype(np.float64 if dtype == np.float64 else np.float32)


def _host(a, pinned):
    """Host copy; 2-D arrays get a row stride that is a multiple of 16 bytes."""
    t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
    if t.dim() == 1:
        return t.pin_memory() if pinned else t.clone()
    n, p = t.shape
    per = 16 // t.element_size()
    ld = (p + per - 1) // per * per
    buf = torch.zeros((n, ld), dtype=t.dtype, pin_memory=pinned)
    buf[:, :p] = t
    return buf[:, :p]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _xdev(X):
    from paper_1801_09661_gb300 import padded
    return padded(X)


GRAM_CASES = [("fp64", np.float64, 1e-12), ("fp32", np.float32, 2e-6), ("split_bf16", np.float32, 1e-6)]


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("mode,dtype,tol", GRAM_CASES)
def test_streamed_gram_matches_oracle(oem, ctx, monkeypatch, pinned, mode, dtype, tol):
    monkeypatch.setenv("OEM_STREAM_ROWS", "4096")
    n, p = 20011, 70  # five blocks, the last of 3627 rows
    X, y = _data(n, p, 3, dtype)
    G, c, yty = oem.oem_gram(ctx, _host(X, pinned), _host(y, pinned), mode=mode)
    assert ctx.sync() == 0
    assert G.is_cuda
    Gr, cr, Nr, _ = oracle.gram_sums(X, y)
    assert _rel(G.cpu().numpy(), Gr) <= tol
    assert _rel(c.cpu().numpy(), cr) <= tol
    assert abs(float(yty.cpu()[0]) - Nr) <= tol * Nr
    Gn = G.cpu().numpy()
    assert np.array_equal(Gn, Gn.T)
    # y on the device with X on the host is allowed too, and gives the same sums
    G2, c2, _ = oem.oem_gram(ctx, _host(X, pinned), _dev(y), mode=mode)
    assert ctx.sync() == 0
    assert torch.equal(G, G2) and torch.equal(c, c2)


def test_streamed_gram_bfloat16_and_a_tiny_last_block(oem, ctx, monkeypatch):
    monkeypatch.setenv("OEM_STREAM_ROWS", "2048")
    n, p = 2 * 2048 + 5, 130  # the last block holds 5 rows
    X, y = _data(n, p, 8)
    Xb = torch.from_numpy(X).to(torch.bfloat16)
    Xr = Xb.float().numpy()
    G, c, yty = oem.oem_gram(ctx, _host(Xb, True), _host(y, True), mode="bf16")
    assert ctx.sync() == 0
    Gr, cr, Nr, _ = oracle.gram_sums(Xr, y)
    assert _rel(G.cpu().numpy(), Gr) <= 1e-6
    assert _rel(c.cpu().numpy(), cr) <= 1e-6


def test_streamed_single_block(oem, ctx, monkeypatch):
    monkeypatch.delenv("OEM_STREAM_ROWS", raising=False)
    n, p = 9001, 40  # below the default block size: one block
    X, y = _data(n, p, 4, np.float64)
    G, c, yty = oem.oem_gram(ctx, _host(X, True), _host(y, True), mode="fp64")
    assert ctx.sync() == 0
    Gr, cr, Nr, _ = oracle.gram_sums(X, y)
    assert _rel(G.cpu().numpy(), Gr) <= 1e-12


@pytest.mark.parametrize("pinned", [True, False])
def test_streamed_fold_grams(oem, ctx, monkeypatch, pinned):
    monkeypatch.setenv("OEM_STREAM_ROWS", "1024")
    n, p, K = 6007, 70, 5
    X, y = _data(n, p, 5, np.float64)
    fold = synthgen.fold_ids(n, K, 5)
    Gk, ck, ytyk, nk = oem.oem_fold_grams(ctx, _host(X, pinned), _dev(y), _host(fold, pinned), K,
                                          mode="fp64")
    assert ctx.sync() == 0
    Gr, cr, Nr, nr = oracle.fold_gram_sums(X, y, fold, K)
    assert np.array_equal(nk.cpu().numpy(), nr)
    for k in range(K):
        assert _rel(Gk[k].cpu().numpy(), Gr[k]) <= 1e-12
        assert _rel(ck[k].cpu().numpy(), cr[k]) <= 1e-12
        assert abs(float(ytyk[k].cpu()) - Nr[k]) <= 1e-12 * Nr[k]


def test_streamed_fit_with_intercept(oem, ctx, monkeypatch):
    # the column shifts come from the first block's rows; later blocks reuse them
    monkeypatch.setenv("OEM_STREAM_ROWS", "2048")
    n, p, L = 6007, 70, 20
    X, y = _data(n, p, 31, mean_scale=40.0)
    kinds = [("lasso", {}), ("enet", {"alpha": 0.5}), ("mcp", {"gamma": 3.0})]
    gp = [oem.Penalty(k, **kw) for k, kw in kinds]
    op = [oracle.Penalty(k, **kw) for k, kw in kinds]
    beta, lam, its, conv, d, beta0 = oem.oem_fit(ctx, _host(X, True), _host(y, True), gp, nlambda=L,
                                                 lambda_min_ratio=1e-2, tol=1e-7, intercept=True,
                                                 standardize=True)
    assert ctx.sync() == 0
    ref = oracle.fit(X, y, op, True, True, nlambda=L, lambda_min_ratio=1e-2, tol=1e-7)
    np.testing.assert_allclose(lam.cpu().numpy(), ref.lambdas, rtol=2e-6)
    assert abs(float(d.cpu()[0]) - ref.d) <= 1e-6 * ref.d
    b, b0 = beta.cpu().numpy(), beta0.cpu().numpy()
    for i in range(len(kinds)):
        assert float(np.abs(b[i] - ref.beta[i]).max()) <= 1e-5 * max(1.0, np.abs(ref.beta[i]).max())
        assert float(np.abs(b0[i] - ref.beta0[i]).max()) <= 1e-5 * max(1.0, np.abs(ref.beta0[i]).max())


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_streamed_cv_matches_oracle(oem, ctx, monkeypatch, mode):
    monkeypatch.setenv("OEM_STREAM_ROWS", "4096")
    n, p, K, L = 12011, 40, 5, 25
    X, y = _data(n, p, 77)
    fold = synthgen.fold_ids(n, K, 77)
    kinds = [("lasso", {}), ("mcp", {"gamma": 3.0}), ("scad", {"gamma": 3.7})]
    gp = [oem.Penalty(k, **kw) for k, kw in kinds]
    op = [oracle.Penalty(k, **kw) for k, kw in kinds]
    out = oem.oem_cv(ctx, _host(X, False), _host(y, False), _host(fold, False), K, gp, nlambda=L,
                     lambda_min_ratio=1e-2, tol=1e-7, gram_mode=mode)
    assert ctx.sync() == 0
    ref = oracle.xval(X, y, fold, K, op, nlambda=L, lambda_min_ratio=1e-2, tol=1e-7)
    np.testing.assert_allclose(out["lambdas"].cpu().numpy(), ref.lambdas,
                               rtol=1e-9 if mode == "fp64" else 2e-6)
    for i in range(len(op)):
        rb = ref.full[i].beta
        assert float(np.abs(out["beta"][i].cpu().numpy() - rb).max()) <= 1e-5 * max(1, np.abs(rb).max())
    np.testing.assert_allclose(out["cvm"].cpu().numpy(), ref.cvm, rtol=1e-5)
    imin = out["idx_min"].cpu().numpy()
    for i in range(len(op)):
        if imin[i] != ref.idx_min[i]:
            assert abs(ref.cvm[i, imin[i]] - ref.cvm[i, ref.idx_min[i]]) <= 1e-6 * ref.cvm[i].min()


def test_streamed_from_a_memory_mapped_file(oem, ctx, monkeypatch, tmp_path):
    # the paper's big.oem keeps X in a file-backed matrix: a memory-mapped
    # file is pageable host memory to the library
    monkeypatch.setenv("OEM_STREAM_ROWS", "2048")
    n, p, L = 7001, 36, 15
    X, y = _data(n, p, 17)
    mm = np.lib.format.open_memmap(str(tmp_path / "X.npy"), mode="w+", dtype=np.float32, shape=(n, p))
    mm[:] = X
    mm.flush()
    Xm = np.load(str(tmp_path / "X.npy"), mmap_mode="r+")
    Xt = torch.from_numpy(Xm)
    assert not Xt.is_pinned()
    pens = [oem.Penalty("lasso"), oem.Penalty("scad", gamma=3.7)]
    beta, lam, its, conv, d = oem.oem_fit(ctx, Xt, _host(y, False), pens, nlambda=L,
                                          lambda_min_ratio=1e-2, tol=1e-7)
    assert ctx.sync() == 0
    for i, pen in enumerate([oracle.Penalty("lasso"), oracle.Penalty("scad", gamma=3.7)]):
        ref = oracle.fit(X, y, [pen], False, False, nlambda=L, lambda_min_ratio=1e-2, tol=1e-7)
        rb = ref.beta[0]
        assert float(np.abs(beta[i].cpu().numpy() - rb).max()) <= 1e-5 * max(1.0, np.abs(rb).max())
    del Xt, Xm


def test_streamed_matches_device_resident_at_full_size(oem, ctx, monkeypatch):
    # n = 10^6, p = 500 float32 (2 GB pinned): eight default-size blocks.
    # Same kernels as the device-resident pass on a different row grouping;
    # sampled entries are checked against float64 dot products.
    monkeypatch.delenv("OEM_STREAM_ROWS", raising=False)
    n, p = 1_000_000, 500
    X, y = _data(n, p, 1)
    Xh = _host(X, True)
    Gs, cs, ys = oem.oem_gram(ctx, Xh, _host(y, True))
    Gd, cd, yd = oem.oem_gram(ctx, _xdev(X), _dev(y))
    assert ctx.sync() == 0
    Gs, Gd = Gs.cpu().numpy(), Gd.cpu().numpy()
    assert _rel(Gs, Gd) <= 2e-6
    rng = np.random.default_rng(0)
    for j, k in rng.integers(0, p, size=(16, 2)):
        ref = float(X[:, j].astype(np.float64) @ X[:, k].astype(np.float64))
        scale = float(np.sqrt(Gd[j, j] * Gd[k, k]))
        assert abs(Gs[j, k] - ref) <= 1e-6 * scale, (j, k)
    for j in rng.integers(0, p, size=8):
        ref = float(X[:, j].astype(np.float64) @ y.astype(np.float64))
        assert abs(float(cs.cpu()[j]) - ref) <= 1e-6 * float(np.sqrt(Gd[j, j] * float(yd.cpu()[0])))


def test_residence_rules(oem, ctx):
    X, y = _data(500, 10, 1)
    with pytest.raises(oem.OemError):
        oem.oem_gram(ctx, _xdev(X), _host(y, True))  # X on the device needs y there too
    fold = synthgen.fold_ids(500, 3, 1)
    with pytest.raises(oem.OemError):
        oem.oem_fold_grams(ctx, _xdev(X), _dev(y), _host(fold, False), 3)
    with pytest.raises(oem.OemError):
        oem.oem_fit_logistic(ctx, _host(X, True), _dev((y > 0).astype(np.float32)),
                             [oem.Penalty("lasso")])
