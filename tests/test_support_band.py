"""The support-band helper of the full-size parity tests, on CPU: it must
flag a support difference far from the threshold and excuse one inside the
band (planted in the oracle's output)."""
import numpy as np

import oracle
from support_band import support_mismatches


def _problem(p=12, seed=3):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((200, p))
    G = A.T @ A / 200
    c = G @ np.r_[1.5, -1.0, 0.5, np.zeros(p - 3)] + 0.05 * rng.standard_normal(p)
    return G, c


def test_identical_supports_have_no_mismatch():
    G, c = _problem()
    pen = oracle.Penalty("lasso")
    d = oracle.lanczos_d(G)[0]
    lam = 0.1 * oracle.lambda_max(c, pen)
    ref = oracle.oem_path(G, c, d, pen, [lam], tol=1e-12, max_iter=100000).beta[0]
    assert support_mismatches(G, c, d, pen, lam, ref.copy(), ref) == ([], [])


def test_far_mismatch_is_flagged_and_near_one_excused():
    G, c = _problem()
    d = oracle.lanczos_d(G)[0]
    for kind in ("lasso", "enet", "mcp", "scad"):
        pen = oracle.Penalty(kind, alpha=0.5)
        lam = 0.1 * oracle.lambda_max(c, pen)
        ref = oracle.oem_path(G, c, d, pen, [lam], tol=1e-12, max_iter=100000).beta[0]
        de = oracle.effective_d(d, pen)
        u = c + de * ref - G @ ref
        thr = lam * (0.5 if kind == "enet" else 1.0)
        # a zero coordinate far below the threshold switched on: flagged
        j = int(np.argmin(np.where(ref == 0, np.abs(u), np.inf)))
        bad = ref.copy()
        bad[j] = 1e-3
        out, inside = support_mismatches(G, c, d, pen, lam, bad, ref)
        assert [k for k, _ in out] == [j] and not inside, kind
        # the same switch is excused when |u_j| sits at the threshold
        c2 = c.copy()
        c2[j] += np.sign(u[j] if u[j] != 0 else 1.0) * (thr - abs(u[j]))
        out, inside = support_mismatches(G, c2, d, pen, lam, bad, ref)
        assert not out and [k for k, _ in inside] == [j], kind


def test_group_mismatch():
    G, c = _problem(p=12)
    groups = np.arange(12) // 3
    pen = oracle.Penalty("grp.lasso", groups=groups)
    d = oracle.lanczos_d(G)[0]
    lam = 0.3 * oracle.lambda_max(c, pen)
    ref = oracle.oem_path(G, c, d, pen, [lam], tol=1e-12, max_iter=100000).beta[0]
    members, _ = pen.group_list(12)
    zero = [k for k, m in enumerate(members) if not np.any(ref[m])]
    assert zero
    bad = ref.copy()
    bad[members[zero[0]][0]] = 1e-3
    out, inside = support_mismatches(G, c, d, pen, lam, bad, ref)
    assert [k for k, _ in out] == [zero[0]]
