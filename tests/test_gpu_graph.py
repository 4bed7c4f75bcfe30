"""CUDA graph capture of the fit entry points: a call made once outside the
capture sizes the workspace and fixes the iteration layout; the same call
captured into a graph then replays the whole path (Gram pass, d, lambda grids,
the OEM launch, CV scoring) on whatever the input buffers hold, and gives the
same bits as a direct call on the same data. Host data the calls upload
(penalty tables, task tables, user lambdas, d) travel inside the captured
launches.
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


def _data(n, p, seed):
    X = synthgen.ar1_design(n, p, 0.5, seed, np.float32)
    beta = synthgen.leading_beta(p, [1.0, -0.8, 0.5, 0.0, 0.3])
    y = synthgen.response(X, beta, 1.0, seed, np.float32)
    return X, y


def _xdev(X):
    from paper_1801_09661_gb300 import padded
    return padded(X)


def _capture(fn):
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    return g


def _same(a, b):
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_fit_replays_on_new_data(oem, ctx):
    n, p, L = 20011, 70, 20
    X, y = _data(n, p, 3)
    Xd, yd = _xdev(X), torch.from_numpy(y).cuda()
    pens = [oem.Penalty("lasso"), oem.Penalty("mcp", gamma=3.0), oem.Penalty("scad", gamma=3.7)]
    kw = dict(nlambda=L, lambda_min_ratio=1e-2, tol=1e-7)
    ref = [t.clone() for t in oem.oem_fit(ctx, Xd, yd, pens, **kw)]
    assert ctx.sync() == 0
    out = tuple(torch.empty_like(t) for t in ref)
    g = _capture(lambda: oem.oem_fit(ctx, Xd, yd, pens, out=out, **kw))
    g.replay()
    torch.cuda.synchronize()
    assert ctx.sync() == 0
    _same(out, ref)
    # new data in the same buffers: the replay fits the new problem
    X2, y2 = _data(n, p, 4)
    Xd.copy_(torch.from_numpy(X2).cuda())
    yd.copy_(torch.from_numpy(y2).cuda())
    g.replay()
    torch.cuda.synchronize()
    assert ctx.sync() == 0
    direct = oem.oem_fit(ctx, Xd, yd, pens, **kw)
    assert ctx.sync() == 0
    _same(out, direct)
    r = oracle.fit(X2, y2, [oracle.Penalty("lasso")], False, False, **kw)
    b = out[0].cpu().numpy()[0]
    assert float(np.abs(b - r.beta[0]).max()) <= 1e-5 * max(1.0, np.abs(r.beta[0]).max())


def test_cv_replays(oem, ctx):
    n, p, K, L = 12011, 40, 5, 15
    X, y = _data(n, p, 7)
    fold = torch.from_numpy(synthgen.fold_ids(n, K, 7)).cuda()
    Xd, yd = _xdev(X), torch.from_numpy(y).cuda()
    pens = [oem.Penalty("lasso"), oem.Penalty("enet", alpha=0.5)]
    kw = dict(nlambda=L, lambda_min_ratio=1e-2, tol=1e-7, intercept=True, standardize=True)
    ref = oem.oem_cv(ctx, Xd, yd, fold, K, pens, **kw)
    assert ctx.sync() == 0
    ref = {k: v.clone() for k, v in ref.items()}
    holder = {}

    def call():
        holder["out"] = oem.oem_cv(ctx, Xd, yd, fold, K, pens, **kw)

    g = _capture(call)
    g.replay()
    torch.cuda.synchronize()
    assert ctx.sync() == 0
    for k in ref:
        assert torch.equal(holder["out"][k], ref[k]), k


def test_fit_path_with_groups_and_user_lambdas_replays(oem, ctx):
    n, p = 8009, 60
    X, y = _data(n, p, 11)
    G, c, N, _ = oracle.gram_sums(X.astype(np.float64), y.astype(np.float64))
    G, c = torch.from_numpy(G / n).cuda(), torch.from_numpy(c / n).cuda()
    groups = np.repeat(np.arange(12), 5)
    pens = [oem.Penalty("grp.lasso", groups=groups), oem.Penalty("lasso")]
    lams = np.geomspace(0.5, 0.01, 12)
    user = np.stack([lams, lams])
    kw = dict(nlambda=12, lambdas=user, tol=1e-7)
    ref = [t.clone() for t in oem.oem_fit_path(ctx, G, c, pens, **kw)]
    assert ctx.sync() == 0
    holder = {}

    def call():
        holder["out"] = oem.oem_fit_path(ctx, G, c, pens, **kw)

    g = _capture(call)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert ctx.sync() == 0
    _same(holder["out"], ref)


def test_capture_refuses_what_it_cannot_record(oem, ctx):
    # the workspace cannot grow inside a capture: a first call of a larger
    # shape is refused with an error, and the context stays usable
    X, y = _data(30011, 90, 5)
    Xd, yd = _xdev(X), torch.from_numpy(y).cuda()
    err = {}
    big = oem.Context(0)
    try:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.graph(g, stream=s):
            try:
                oem.oem_fit(big, Xd, yd, [oem.Penalty("lasso")], nlambda=5, lambda_min_ratio=0.1)
            except oem.OemError as e:
                err["e"] = e
        assert "e" in err and err["e"].code == oem.OEM_EINVAL
        beta = oem.oem_fit(big, Xd, yd, [oem.Penalty("lasso")], nlambda=5, lambda_min_ratio=0.1)[0]
        assert big.sync() == 0 and torch.isfinite(beta).all()
    finally:
        big.close()
