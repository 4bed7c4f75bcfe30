"""The bounded-wait failure path of the OEM iteration kernel, made to run out
on purpose without faulting the GPU.

Every wait of the iteration kernel (the cluster-mode mbarrier wait for the
peers' G dbeta words, the grid-mode poll of the tagged words in global
memory) gives up after a clock budget, sets the timeout bit of the status
word and leaves the loop; the kernel then returns normally. The budget is
about 2 s; OEM_DEVICE_WAIT_CYCLES, read at each launch, shortens it, and
OEM_DEVICE_WAIT_TEST=1 makes the first exchange of a launch wait for data
that nobody sends (four bytes more than the peers store, or a tag nobody
writes), so the wait must run out. A fit with several CTAs per task must then
report OEM_ETIMEOUT from oem_sync, and the same context must fit the same
problem normally, bit for bit as before.
"""
import os

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


def _problem(p=300, n=6000, seed=4):
    X = synthgen.ar1_design(n, p, 0.5, seed, np.float64)
    y = synthgen.response(X, synthgen.leading_beta(p, [1.0, -0.8, 0.5]), 1.0, seed, np.float64)
    G, c, _, _ = oracle.gram_sums(X, y)
    return torch.from_numpy(G / n).cuda(), torch.from_numpy(c / n).cuda()


# p = 300: the replicated-update kernel; p = 1100: the row-owned kernel (every
# warp of a CTA waits on the cluster barrier, or polls the tagged words)
@pytest.mark.parametrize("p,layout", [(300, {"cluster_ctas": 8}), (300, {"cluster_ctas": 40}),
                                      (1100, {"cluster_ctas": 16}), (1100, {"cluster_ctas": 60})])
def test_expired_wait_reports_timeout_and_context_stays_usable(oem, p, layout):
    G, c = _problem(p=p)
    pens = [oem.Penalty("lasso"), oem.Penalty("mcp", gamma=3.0)]
    kw = dict(nlambda=30, lambda_min_ratio=1e-2, tol=1e-7, autotune=False, **layout)
    ctx = oem.Context(0)
    try:
        ref = [t.clone() for t in oem.oem_fit_path(ctx, G, c, pens, **kw)]
        assert ctx.sync() == 0
        os.environ["OEM_DEVICE_WAIT_CYCLES"] = "2000000"  # about 1 ms
        os.environ["OEM_DEVICE_WAIT_TEST"] = "1"
        try:
            oem.oem_fit_path(ctx, G, c, pens, **kw)
            with pytest.raises(oem.OemError) as ei:
                ctx.sync()
            assert ei.value.code == oem.OEM_ETIMEOUT
        finally:
            del os.environ["OEM_DEVICE_WAIT_CYCLES"]
            del os.environ["OEM_DEVICE_WAIT_TEST"]
        # the kernel returned and the context is usable: the same fit again
        again = oem.oem_fit_path(ctx, G, c, pens, **kw)
        assert ctx.sync() == 0
        for a, b in zip(again, ref):
            assert torch.equal(a, b)
    finally:
        ctx.close()
