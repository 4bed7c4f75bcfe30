"""The allocation-free Gram entry point, oem_gram_noalloc, against oem_gram.

oem_gram_noalloc serves callers that cannot allocate device memory when they
call: code under a framework that owns the whole device memory pool, loops
that must not allocate once started, or callers without an oem_ctx. It keeps
its working memory in one array the library declares in device memory, so it
must give the same G, c, y^T y as oem_gram. Each test makes two calls in a row
with different shapes: the array keeps the first call's contents, and those
must not leak into the second result. This file is named to be collected last.
"""
import numpy as np
import pytest

import synthgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# tolerance of the Gram parity tests for each mode (relative Frobenius)
TOL = {"fp64": 1e-12, "fp32": 2e-6, "split_bf16": 1e-6}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("mode,dtype", [("fp64", np.float64), ("fp32", np.float32),
                                        ("split_bf16", np.float32)])
def test_noalloc_matches_oem_gram_twice(mode, dtype):
    import paper_1801_09661_gb300 as oem
    assert torch.cuda.is_available()
    ctx = oem.Context(0)
    for n, p, seed in ((20011, 300, 1), (5003, 70, 2)):
        X = synthgen.ar1_design(n, p, 0.5, seed, dtype)
        y = synthgen.response(X, synthgen.leading_beta(p, [1.0, -0.5]), 1.0, seed,
                              np.float64 if dtype == np.float64 else np.float32)
        Xd = oem.padded(X)
        yd = torch.from_numpy(y).cuda()
        G1, c1, n1 = oem.oem_gram_noalloc(Xd, yd, mode=mode)
        torch.cuda.synchronize()
        G2, c2, n2 = oem.oem_gram(ctx, Xd, yd, mode=mode)
        assert ctx.sync() == 0
        tol = TOL[mode]
        assert _rel(G1.cpu().numpy(), G2.cpu().numpy()) <= tol
        assert _rel(c1.cpu().numpy(), c2.cpu().numpy()) <= tol
        assert abs(float(n1.cpu()[0]) - float(n2.cpu()[0])) <= tol * abs(float(n2.cpu()[0]))
    ctx.close()
