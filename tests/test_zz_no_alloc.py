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
TOL = {"fp64": 1e-12, "fp32": 2e-6, "split_bf16": 1e-6, "bf16": 1e-6, "tf32": 2e-5}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("mode,dtype", [("fp64", np.float64), ("fp32", np.float32),
                                        ("split_bf16", np.float32), ("tf32", np.float32),
                                        ("bf16", "bf16")])
def test_noalloc_matches_oem_gram_twice(mode, dtype):
    import paper_1801_09661_gb300 as oem
    assert torch.cuda.is_available()
    ctx = oem.Context(0)
    for n, p, seed in ((20011, 300, 1), (5003, 70, 2)):
        X = synthgen.ar1_design(n, p, 0.5, seed, dtype)
        y = synthgen.response(X, synthgen.leading_beta(p, [1.0, -0.5]), 1.0, seed,
                              np.float64 if dtype == np.float64 else np.float32)
        if dtype == "bf16":  # bfloat16 X: y travels as three bfloat16 columns
            Xd = oem.padded(torch.from_numpy(X.view(np.int16)).view(torch.bfloat16))
        else:
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


def test_noalloc_refuses_host_memory():
    """The entry point has no host path: X in host memory is refused before
    any launch (the binding refuses a CPU tensor; the C entry point itself
    refuses a pinned host pointer)."""
    import paper_1801_09661_gb300 as oem
    from paper_1801_09661_gb300 import _binding as b
    X = torch.randn(300, 16, dtype=torch.float32)
    y = torch.randn(300, dtype=torch.float32)
    with pytest.raises(TypeError):
        oem.oem_gram_noalloc(X, y)
    Xh, yh = X.pin_memory(), y.pin_memory()
    G = torch.empty((16, 16), dtype=torch.float64, device="cuda")
    c = torch.empty(16, dtype=torch.float64, device="cuda")
    n1 = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = b.lib.oem_gram_noalloc(Xh.data_ptr(), b.OEM_F32, 300, 16, 16, yh.data_ptr(), b.OEM_GRAM_AUTO,
                                G.data_ptr(), c.data_ptr(), n1.data_ptr(), None)
    assert rc == b.OEM_EINVAL
