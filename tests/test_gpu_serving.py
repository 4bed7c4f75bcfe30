"""Serving (continuous batching) through the C ABI.

* A job's result is the same alone and in a mix of jobs of other n, p, K and
  penalty submitted at the same time (the batch only changes which clusters
  share a launch; each job's arithmetic is its own): compared to 1e-12.
* Served results agree with oem_fit / oem_cv on the same data (same kernels)
  and with the FP64 oracle (max |dbeta| <= 1e-5 max(1, ||beta||_inf)).
* Admission: a job larger than the budget is refused at submission; jobs that
  fit one at a time but not together all complete (they wait for memory).
* The plain form (float32 CUDA-core Gram, one launch per iteration) reaches
  the same paths (tolerance 1e-5 relative: different Gram arithmetic).
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
    assert torch.cuda.is_available()
    return m


def _job_data(n, p, seed, K):
    X = synthgen.ar1_design(n, p, 0.5, seed, np.float32)
    y = synthgen.response(X, synthgen.leading_beta(p, [-0.5, -0.5, 0.5, 0.5, 1.0]), 2.0, seed,
                          np.float32)
    fold = synthgen.fold_ids(n, K, seed) if K else None
    return X, y, fold


JOBS = [  # (n, p, K, penalty)
    (20000, 37, 0, ("lasso", {})),
    (30011, 120, 5, ("mcp", {"gamma": 3.0})),
    (15000, 260, 0, ("mcp", {"gamma": 3.0})),
    (40000, 64, 5, ("lasso", {})),
    (12000, 501, 0, ("lasso", {})),
]


def _submit(oem, srv, spec, data, L=30):
    n, p, K, (kind, kw) = spec
    X, y, fold = data
    Xd = oem.padded(X)
    yd = torch.from_numpy(y).cuda()
    fd = torch.from_numpy(fold).cuda() if K else None
    return srv.submit(Xd, yd, oem.Penalty(kind, **kw), fold=fd, K=K, nlambda=L,
                      lambda_min_ratio=1e-2, tol=1e-7)


@pytest.fixture(scope="module")
def data():
    return [_job_data(n, p, 100 + i, K) for i, (n, p, K, _) in enumerate(JOBS)]


@pytest.fixture(scope="module")
def mixed(oem, data):
    srv = oem.Server(0, budget_bytes=8 << 30, form="batched", iters_per_round=300)
    ids = [_submit(oem, srv, spec, d) for spec, d in zip(JOBS, data)]
    out = []
    for i in ids:
        st, lat, rc = srv.wait(i, 300)
        assert st == "done", (st, rc)
        out.append(srv.result(i))
    stats = srv.stats()
    srv.close()
    assert stats["jobs_done"] == len(JOBS)
    assert stats["paths_done"] == sum((K + 1) if K else 1 for _, _, K, _ in JOBS)
    assert stats["rounds"] >= 2  # the paths spanned several batched rounds
    return out


@pytest.mark.parametrize("j", [0, 1, 4])
def test_same_result_alone_and_in_the_mix(oem, data, mixed, j):
    srv = oem.Server(0, budget_bytes=8 << 30, form="batched", iters_per_round=300)
    i = _submit(oem, srv, JOBS[j], data[j])
    st, lat, rc = srv.wait(i, 300)
    assert st == "done"
    alone = srv.result(i)
    srv.close()
    np.testing.assert_allclose(alone["beta"], mixed[j]["beta"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(alone["lambdas"], mixed[j]["lambdas"], rtol=1e-15)
    if JOBS[j][2]:
        np.testing.assert_allclose(alone["cvm"], mixed[j]["cvm"], rtol=1e-12)


@pytest.mark.parametrize("j", [0, 1, 2, 3, 4])
def test_served_matches_direct_calls_and_oracle(oem, data, mixed, j):
    n, p, K, (kind, kw) = JOBS[j]
    X, y, fold = data[j]
    res = mixed[j]
    ctx = oem.Context(0)
    pen = oem.Penalty(kind, **kw)
    if K:
        out = oem.oem_cv(ctx, oem.padded(X), torch.from_numpy(y).cuda(),
                         torch.from_numpy(fold).cuda(), K, [pen], nlambda=30,
                         lambda_min_ratio=1e-2, tol=1e-7)
        ctx.sync()
        np.testing.assert_allclose(res["beta"], out["beta"][0].cpu().numpy(), atol=1e-12)
        np.testing.assert_allclose(res["cvm"], out["cvm"][0].cpu().numpy(), rtol=1e-10)
        assert res["idx_min"] == int(out["idx_min"][0])
    else:
        beta, lam, its, conv, d = oem.oem_fit(ctx, oem.padded(X), torch.from_numpy(y).cuda(), [pen],
                                              nlambda=30, lambda_min_ratio=1e-2, tol=1e-7)
        ctx.sync()
        np.testing.assert_allclose(res["beta"], beta[0].cpu().numpy(), atol=1e-12)
    ctx.close()
    # against the FP64 oracle on the full-data path
    G, c, N, nn = oracle.gram_sums(X, y)
    G, c = G / nn, c / nn
    opn = oracle.Penalty(kind, **kw)
    lams = oracle.lambda_grid(oracle.lambda_max(c, opn), 30, 1e-2)
    ref = oracle.oem_path(G, c, oracle.lanczos_d(G)[0], opn, lams, tol=1e-7)
    assert np.abs(res["beta"] - ref.beta).max() <= 1e-5 * max(1.0, np.abs(ref.beta).max())


def test_budget_admission(oem, data):
    # a job larger than the whole budget is refused at submission
    srv = oem.Server(0, budget_bytes=64 << 20, form="batched")
    X = torch.zeros((200000, 256), dtype=torch.float32, device="cuda")
    y = torch.zeros(200000, dtype=torch.float32, device="cuda")
    with pytest.raises(oem.OemError) as e:
        srv.submit(X, y, oem.Penalty("lasso"))
    assert e.value.code == oem.OEM_EBUDGET
    srv.close()
    # jobs that fit one at a time but not two at once (the p = 501 job needs
    # about 22 MB of tile partials and Grams) all complete, one after another
    budget = 40 << 20
    srv = oem.Server(0, budget_bytes=budget, form="batched", iters_per_round=200)
    ids = [_submit(oem, srv, JOBS[4], data[4]) for _ in range(3)]
    for i in ids:
        st, lat, rc = srv.wait(i, 300)
        assert st == "done"
    res = [srv.result(i) for i in ids]
    stats = srv.stats()
    srv.close()
    assert 0 < stats["peak_bytes"] <= budget
    for r in res[1:]:
        np.testing.assert_array_equal(r["beta"], res[0]["beta"])


def test_plain_form_reaches_the_same_paths(oem, data, mixed):
    srv = oem.Server(0, budget_bytes=8 << 30, form="plain")
    ids = [_submit(oem, srv, JOBS[j], data[j]) for j in (0, 1)]
    for j, i in zip((0, 1), ids):
        st, lat, rc = srv.wait(i, 600)
        assert st == "done"
        r = srv.result(i)
        ref = mixed[j]["beta"]
        assert np.abs(r["beta"] - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
        if JOBS[j][2]:
            assert r["idx_min"] == mixed[j]["idx_min"] or \
                abs(r["cvm"][r["idx_min"]] - mixed[j]["cvm"][mixed[j]["idx_min"]]) < 1e-6
    srv.close()
