"""FP64 oracle: Gram sums, fold statistics, Lanczos d, lambda grid, penalty
thresholds, warm-started OEM paths and cross-validation scoring.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
calls this module.

Notation (paper, Sections 2-3): X is n x p, y has length n. The scaled
sufficient statistics are G = X^T X / n, c = X^T y / n and N = y^T y / n.
Reading of the scaling (the paper writes ||y - X beta||^2 in Eq. (2) and a
factor 1/2 in the M-step, Eq. (3); the oem.xtx example of Section 5.6 divides
both X^T X and X^T y by n): the problem solved is

    minimise  f(beta) = 1/(2n) ||y - X beta||^2 + P_lambda(beta)
            = N/2 - c^T beta + beta^T G beta / 2 + P_lambda(beta).

With scalar d >= lambda_1(G) and S = I (Section 2.1), A = d I - G and the OEM
update is beta <- threshold(u), u = c + A beta = c + d beta - G beta.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import scipy.linalg

__all__ = [
    "Penalty", "PathResult", "CVResult",
    "gram_sums", "fold_gram_sums", "assemble_fold_grams",
    "lanczos_d", "effective_d", "lambda_max", "lambda_grid",
    "threshold", "threshold_lasso", "threshold_enet", "threshold_mcp",
    "threshold_scad", "threshold_group_lasso", "threshold_group_mcp",
    "threshold_group_scad", "threshold_sparse_group_lasso",
    "oem_path", "penalty_value", "objective", "kkt_violation",
    "cv_mse", "cv_select", "xval", "group_weights_default",
    "FitResult", "augmented_sums", "centered_stats", "back_transform", "cv_mse_intercept",
    "fit", "xval_intercept",
    "LogisticResult", "sigmoid", "logistic_loss", "logistic_path",
]

KINDS = ("lasso", "enet", "mcp", "scad", "grp.lasso", "grp.mcp", "grp.scad", "sgl")
GROUP_KINDS = ("grp.lasso", "grp.mcp", "grp.scad", "sgl")


@dataclass
class Penalty:
    """One penalty of Table 1: lasso, elastic net, MCP, SCAD, group lasso,
    group MCP ("grp.mcp"), group SCAD ("grp.scad"), sparse group lasso ("sgl").

    w: variable weights w_j (default 1). groups: group id per variable
    (0..G-1) for the group penalties. cg: group weights c_k (default
    sqrt|g_k|, the Yuan-Lin convention; the paper states no default). alpha:
    elastic-net mixing; gamma: MCP / SCAD (and their group forms); tau: the
    sparse group lasso's split between the l1 and the group terms.
    """
    kind: str
    alpha: float = 1.0
    gamma: float = 3.0
    w: Optional[np.ndarray] = None
    groups: Optional[np.ndarray] = None
    cg: Optional[np.ndarray] = None
    tau: float = 0.5

    def weights(self, p: int) -> np.ndarray:
        return np.ones(p) if self.w is None else np.asarray(self.w, dtype=np.float64)

    def group_list(self, p: int):
        g = np.asarray(self.groups, dtype=np.int64)
        assert g.shape == (p,)
        ng = int(g.max()) + 1
        members = [np.flatnonzero(g == k) for k in range(ng)]
        cg = group_weights_default(members) if self.cg is None else np.asarray(self.cg, float)
        return members, cg


def group_weights_default(members) -> np.ndarray:
    return np.array([math.sqrt(len(m)) for m in members], dtype=np.float64)


# ---------------------------------------------------------------------------
# Sufficient statistics (Section 3)
# ---------------------------------------------------------------------------

def gram_sums(X: np.ndarray, y: np.ndarray):
    """Raw sums X^T X, X^T y, y^T y and n in float64 (Section 3: A = dI - X^T X).

    Inputs are widened to float64 exactly (float32 and bfloat16 values are
    representable), so products are exact and only the summation rounds.
    """
    Xd = np.asarray(X, dtype=np.float64)
    yd = np.asarray(y, dtype=np.float64)
    return Xd.T @ Xd, Xd.T @ yd, float(yd @ yd), Xd.shape[0]


def fold_gram_sums(X: np.ndarray, y: np.ndarray, fold: np.ndarray, K: int):
    """Per-fold raw sums X_k^T X_k, X_k^T y_k, y_k^T y_k, n_k (Section 3).

    The rows of fold k are those with fold[i] == k, k = 0..K-1.
    """
    p = X.shape[1]
    Gk = np.zeros((K, p, p))
    ck = np.zeros((K, p))
    Nk = np.zeros(K)
    nk = np.zeros(K, dtype=np.int64)
    for k in range(K):
        rows = np.flatnonzero(fold == k)
        Gk[k], ck[k], Nk[k], nk[k] = gram_sums(X[rows], y[rows])
    return Gk, ck, Nk, nk


def assemble_fold_grams(Gk, ck, Nk, nk):
    """Full-data and leave-fold-out statistics from fold sums (Section 3).

    The paper's identities: X^T X = sum_k X_k^T X_k and
    X_{-k}^T X_{-k} = sum_{c != k} X_c^T X_c (likewise X^T y). Index 0 of the
    result is the full data (scaled by 1/n); index k+1 leaves fold k out
    (scaled by 1/n_{-k}). Returns (G, c, N, counts) with shapes (K+1, p, p),
    (K+1, p), (K+1,), (K+1,).
    """
    K = Gk.shape[0]
    Gsum, csum, Nsum, n = Gk.sum(0), ck.sum(0), Nk.sum(), int(nk.sum())
    p = Gk.shape[1]
    G = np.empty((K + 1, p, p))
    c = np.empty((K + 1, p))
    N = np.empty(K + 1)
    cnt = np.empty(K + 1, dtype=np.int64)
    G[0], c[0], N[0], cnt[0] = Gsum / n, csum / n, Nsum / n, n
    for k in range(K):
        m = n - int(nk[k])
        cnt[k + 1] = m
        G[k + 1] = (Gsum - Gk[k]) / m
        c[k + 1] = (csum - ck[k]) / m
        N[k + 1] = (Nsum - Nk[k]) / m
    return G, c, N, cnt


# ---------------------------------------------------------------------------
# d >= lambda_1(G) by Lanczos (Section 2.1)
# ---------------------------------------------------------------------------

def lanczos_d(G: np.ndarray, steps: int = 64):
    """Upper bound d of the largest eigenvalue of symmetric PSD G, by Lanczos.

    Section 2.1: OEM converges for every d >= lambda_1(X^T X) and fastest at
    d = lambda_1, which Lanczos computes efficiently. Reading: run
    min(steps, p) Lanczos steps from v_1 = 1/sqrt(p) (full reorthogonalisation),
    take the largest Ritz value theta of the tridiagonal T and its residual
    norm r = beta_m |s_m| (s the unit eigenvector of T), and return
    d = theta + r: some eigenvalue of G lies within r of theta, and theta <=
    lambda_1 by interlacing. An all-zero G returns d = 1 (any d >= 0 = lambda_1
    is valid). Returns (d, theta, r, m).
    """
    G = np.asarray(G, dtype=np.float64)
    p = G.shape[0]
    m_max = max(1, min(int(steps), p))
    scale = float(np.linalg.norm(G))
    if scale == 0.0:
        return 1.0, 0.0, 0.0, 0
    V = np.zeros((m_max + 1, p))
    V[0] = 1.0 / math.sqrt(p)
    alpha, beta = [], []
    for j in range(m_max):
        w = G @ V[j]
        a = float(V[j] @ w)
        w = w - a * V[j]
        if j > 0:
            w = w - beta[-1] * V[j - 1]
        for _ in range(2):  # full reorthogonalisation against V[0..j]
            w = w - V[:j + 1].T @ (V[:j + 1] @ w)
        b = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(b)
        if b <= 1e-13 * scale:  # invariant subspace: theta is exact
            break
        V[j + 1] = w / b
    m = len(alpha)
    if m == 1:
        theta, s_last = alpha[0], 1.0
    else:
        ev, evec = scipy.linalg.eigh_tridiagonal(np.array(alpha), np.array(beta[:-1]))
        theta, s_last = float(ev[-1]), float(evec[-1, -1])
    r = beta[-1] * abs(s_last)
    return theta + r, theta, r, m


def effective_d(d: float, pen: Penalty) -> float:
    """d used by the threshold of pen. Reading: the MCP and SCAD updates
    (Eqs. for M and C in Section 2.2) divide by gamma d - 1 and
    (gamma - 1) d - 1, so d is raised to 1.01/gamma (MCP) or 1.01/(gamma - 1)
    (SCAD) when smaller; any d >= lambda_1 is valid (Section 2.1)."""
    if pen.kind in ("mcp", "grp.mcp"):
        return max(d, 1.01 / pen.gamma)
    if pen.kind in ("scad", "grp.scad"):
        return max(d, 1.01 / (pen.gamma - 1.0))
    return d


# ---------------------------------------------------------------------------
# lambda grid (Section 5.1: lambda.min.ratio)
# ---------------------------------------------------------------------------

def lambda_max(c: np.ndarray, pen: Penalty) -> float:
    """Smallest lambda at which beta = 0 is the fixed point of the update.

    With beta = 0, u = c. The lasso/MCP/SCAD updates give 0 iff |c_j| <= w_j
    lambda; the elastic net iff |c_j| <= alpha w_j lambda; the group lasso iff
    ||c_g|| <= c_k lambda. Variables (groups) with zero weight are not
    penalised and do not enter. Reading for alpha = 0 (ridge): alpha is taken
    as max(alpha, 1e-3) here, as glmnet does.
    """
    c = np.asarray(c, dtype=np.float64)
    p = c.size
    if pen.kind in ("grp.lasso", "grp.mcp", "grp.scad"):
        # group MCP / SCAD update the norm with M / C, which vanish iff
        # ||u_g|| <= c_k lambda, like the group lasso
        members, cg = pen.group_list(p)
        vals = [np.linalg.norm(c[m]) / cg[k] for k, m in enumerate(members) if cg[k] > 0]
        return float(max(vals)) if vals else 0.0
    if pen.kind == "sgl":
        members, cg = pen.group_list(p)
        w = pen.weights(p)
        return float(max([_sgl_group_lambda(c[m], w[m], cg[k], pen.tau)
                          for k, m in enumerate(members)] + [0.0]))
    w = pen.weights(p)
    pos = w > 0
    if not pos.any():
        return 0.0
    lm = float(np.max(np.abs(c[pos]) / w[pos]))
    if pen.kind == "enet":
        lm /= max(pen.alpha, 1e-3)
    return lm


def _sgl_group_lambda(cgrp, wgrp, ck, tau):
    """Smallest lambda with a zero sparse-group-lasso update for one group at
    beta = 0: ||S(c_g, lambda tau w_g)|| <= lambda (1 - tau) c_k, where S is
    the soft threshold. The left side falls and the right side grows with
    lambda, so the crossing is found by bisection (to float64 resolution)."""
    a = np.abs(cgrp)
    if tau > 0.0:
        pos = wgrp > 0
        if (~pos).any() and np.linalg.norm(a[~pos]) > 0 and (1.0 - tau) * ck <= 0:
            return math.inf  # an unpenalised nonzero coordinate
        hi = float(np.max(a[pos] / (tau * wgrp[pos]))) if pos.any() else 0.0
    else:
        hi = float(np.linalg.norm(a) / ck) if ck > 0 else math.inf
    if not math.isfinite(hi):
        return hi

    def f(lam):
        return float(np.linalg.norm(np.maximum(a - lam * tau * wgrp, 0.0))) - lam * (1.0 - tau) * ck

    lo = 0.0
    hi = max(hi, 1e-300)
    for _ in range(2100):  # unpenalised coordinates can push the crossing up
        if f(hi) <= 0.0:
            break
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if f(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    return hi


def lambda_grid(lmax: float, nlambda: int, ratio: float) -> np.ndarray:
    """lambda_l = lmax * ratio^((l-1)/(L-1)), l = 1..L (log-spaced, decreasing)."""
    if nlambda == 1:
        return np.array([lmax])
    t = np.arange(nlambda) / (nlambda - 1)
    return lmax * np.power(ratio, t)


# ---------------------------------------------------------------------------
# Thresholding operators (Section 2.2, Eqs. lasso, net, mcp, scad, glasso)
# ---------------------------------------------------------------------------

def threshold_lasso(u, wl, d):
    """Eq. (lasso): sign(u) (|u| - w lambda)_+ / d."""
    return np.sign(u) * np.maximum(np.abs(u) - wl, 0.0) / d


def threshold_enet(u, wl, alpha, d):
    """Eq. (net): sign(u) (|u| - w alpha lambda)_+ / (d + w (1 - alpha) lambda)."""
    return np.sign(u) * np.maximum(np.abs(u) - wl * alpha, 0.0) / (d + wl * (1.0 - alpha))


def threshold_mcp(u, wl, gamma, d):
    """Eq. (mcp): sign(u) gamma (|u| - w lambda)_+ / (gamma d - 1) if
    |u| <= w gamma lambda d, else u / d."""
    au = np.abs(u)
    inner = np.sign(u) * gamma * np.maximum(au - wl, 0.0) / (gamma * d - 1.0)
    return np.where(au <= wl * gamma * d, inner, u / d)


def threshold_scad(u, wl, gamma, d):
    """Eq. (scad): soft threshold / d if |u| <= (d + 1) w lambda;
    sign(u) ((gamma - 1)|u| - w gamma lambda) / ((gamma - 1) d - 1) if
    (d + 1) w lambda < |u| <= w gamma lambda d; u / d beyond."""
    au = np.abs(u)
    r1 = np.sign(u) * np.maximum(au - wl, 0.0) / d
    r2 = np.sign(u) * ((gamma - 1.0) * au - wl * gamma) / ((gamma - 1.0) * d - 1.0)
    return np.where(au <= (d + 1.0) * wl, r1, np.where(au <= wl * gamma * d, r2, u / d))


def threshold_group_lasso(u, members, cl, d):
    """Eq. (glasso): beta_g = (u_g / d) (1 - c_k lambda / ||u_g||)_+ per group;
    ||u_g|| = 0 gives beta_g = 0."""
    out = np.zeros_like(u)
    for k, m in enumerate(members):
        nrm = float(np.linalg.norm(u[m]))
        if nrm > 0.0:
            out[m] = u[m] / d * max(1.0 - cl[k] / nrm, 0.0)
    return out


def threshold_group_mcp(u, members, cl, gamma, d):
    """Eq. (gmcp): beta_g = M(||u_g||, c_k lambda, gamma, d) u_g / ||u_g||;
    ||u_g|| = 0 gives beta_g = 0."""
    out = np.zeros_like(u)
    for k, m in enumerate(members):
        nrm = float(np.linalg.norm(u[m]))
        if nrm > 0.0:
            out[m] = float(threshold_mcp(np.array(nrm), cl[k], gamma, d)) * u[m] / nrm
    return out


def threshold_group_scad(u, members, cl, gamma, d):
    """Eq. (gscad): beta_g = C(||u_g||, c_k lambda, gamma, d) u_g / ||u_g||."""
    out = np.zeros_like(u)
    for k, m in enumerate(members):
        nrm = float(np.linalg.norm(u[m]))
        if nrm > 0.0:
            out[m] = float(threshold_scad(np.array(nrm), cl[k], gamma, d)) * u[m] / nrm
    return out


def threshold_sparse_group_lasso(u, members, wl_tau, cl_1mtau, d):
    """Eq. (sglasso), reading: v = S(u, w lambda tau, d) (the lasso update),
    then the group step of the prox of d/2 ||beta - u/d||^2 + P, which
    shrinks v_g by c_k lambda (1 - tau) / d:
    beta_g = v_g (1 - c_k lambda (1 - tau) / (d ||v_g||))_+.
    (The paper writes G(v_g, c_k lambda (1 - tau), 1), which is this at d = 1.)"""
    v = threshold_lasso(u, wl_tau, d)
    out = np.zeros_like(u)
    for k, m in enumerate(members):
        nrm = float(np.linalg.norm(v[m]))
        if nrm > 0.0:
            out[m] = v[m] * max(1.0 - cl_1mtau[k] / (d * nrm), 0.0)
    return out


def threshold(u: np.ndarray, lam: float, d: float, pen: Penalty) -> np.ndarray:
    """Apply pen's update to u at tuning parameter lam (Section 2.2)."""
    p = u.size
    de = effective_d(d, pen)
    if pen.kind in GROUP_KINDS:
        members, cg = pen.group_list(p)
        if pen.kind == "grp.lasso":
            return threshold_group_lasso(u, members, cg * lam, de)
        if pen.kind == "grp.mcp":
            return threshold_group_mcp(u, members, cg * lam, pen.gamma, de)
        if pen.kind == "grp.scad":
            return threshold_group_scad(u, members, cg * lam, pen.gamma, de)
        return threshold_sparse_group_lasso(u, members, pen.weights(p) * lam * pen.tau,
                                            cg * lam * (1.0 - pen.tau), de)
    wl = pen.weights(p) * lam
    if pen.kind == "lasso":
        return threshold_lasso(u, wl, de)
    if pen.kind == "enet":
        return threshold_enet(u, wl, pen.alpha, de)
    if pen.kind == "mcp":
        return threshold_mcp(u, wl, pen.gamma, de)
    if pen.kind == "scad":
        return threshold_scad(u, wl, pen.gamma, de)
    raise ValueError(pen.kind)


# ---------------------------------------------------------------------------
# Warm-started OEM path (Section 2.1 Steps 1-2; Section 5.2)
# ---------------------------------------------------------------------------

@dataclass
class PathResult:
    beta: np.ndarray        # (L, p)
    lambdas: np.ndarray     # (L,)
    iters: np.ndarray       # (L,) iterations taken at each lambda
    converged: np.ndarray   # (L,) bool
    d: float


def oem_path(G, c, d, pen: Penalty, lambdas: Sequence[float], tol: float = 1e-7,
             max_iter: int = 10_000, beta0: Optional[np.ndarray] = None,
             trace: Optional[list] = None) -> PathResult:
    """OEM iterations along a decreasing lambda grid, warm-started.

    Each iteration is u = c + d beta - G beta (Section 2.1, u = X^T y + A beta
    with A = d I - X^T X) followed by beta <- threshold(u). The first lambda
    starts from beta = 0 (or beta0); each later lambda starts from the
    previous solution. Reading of the stopping rule (the paper leaves it
    unstated): stop at the first iteration t with
    max_j |beta_j^(t) - beta_j^(t-1)| <= tol * max(1, max_j |beta_j^(t)|),
    or after max_iter iterations (then converged = False). If trace is a list,
    the objective after every iteration is appended (lambda index, value).
    """
    G = np.asarray(G, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    p = c.size
    # A = d I - G must use the same d as the threshold (effective_d raises it
    # for MCP / SCAD when needed; any d >= lambda_1 is valid)
    d = effective_d(d, pen)
    lambdas = np.asarray(lambdas, dtype=np.float64)
    L = lambdas.size
    beta = np.zeros(p) if beta0 is None else np.array(beta0, dtype=np.float64)
    B = np.zeros((L, p))
    its = np.zeros(L, dtype=np.int64)
    conv = np.zeros(L, dtype=bool)
    for l, lam in enumerate(lambdas):
        for t in range(1, max_iter + 1):
            u = c + d * beta - G @ beta
            new = threshold(u, lam, d, pen)
            delta = float(np.max(np.abs(new - beta))) if p else 0.0
            beta = new
            if trace is not None:
                trace.append((l, objective(G, c, 0.0, beta, lam, pen)))
            if delta <= tol * max(1.0, float(np.max(np.abs(beta))) if p else 0.0):
                conv[l] = True
                its[l] = t
                break
        else:
            its[l] = max_iter
        B[l] = beta
    return PathResult(B, lambdas, its, conv, d)


# ---------------------------------------------------------------------------
# Objective and optimality (Table 1 penalty forms)
# ---------------------------------------------------------------------------

def _scad_value(b, lam, gamma):
    a = np.abs(b)
    return np.where(a <= lam, lam * a,
                    np.where(a <= gamma * lam,
                             -(a * a - 2.0 * gamma * lam * a + lam * lam) / (2.0 * (gamma - 1.0)),
                             (gamma + 1.0) * lam * lam / 2.0))


def _mcp_value(b, lam, gamma):
    a = np.abs(b)
    return np.where(a <= gamma * lam, lam * a - a * a / (2.0 * gamma), gamma * lam * lam / 2.0)


def penalty_value(beta: np.ndarray, lam: float, pen: Penalty) -> float:
    """P_lambda(beta) for the forms of Table 1."""
    p = beta.size
    if pen.kind in GROUP_KINDS:
        members, cg = pen.group_list(p)
        nb = np.array([np.linalg.norm(beta[m]) for m in members])
        if pen.kind == "grp.lasso":
            return float(lam * np.sum(cg * nb))
        if pen.kind == "grp.mcp":  # Table 1 (reading: one lambda, inside P)
            return float(np.sum(_mcp_value(nb, lam * cg, pen.gamma)))
        if pen.kind == "grp.scad":
            return float(np.sum(_scad_value(nb, lam * cg, pen.gamma)))
        return float(lam * (1.0 - pen.tau) * np.sum(cg * nb)
                     + lam * pen.tau * np.sum(pen.weights(p) * np.abs(beta)))
    w = pen.weights(p)
    if pen.kind == "lasso":
        return float(lam * np.sum(w * np.abs(beta)))
    if pen.kind == "enet":
        return float(pen.alpha * lam * np.sum(w * np.abs(beta))
                     + 0.5 * (1.0 - pen.alpha) * lam * np.sum(w * beta * beta))
    if pen.kind == "mcp":
        return float(np.sum(_mcp_value(beta, lam * w, pen.gamma)))
    if pen.kind == "scad":
        return float(np.sum(_scad_value(beta, lam * w, pen.gamma)))
    raise ValueError(pen.kind)


def objective(G, c, N, beta, lam, pen: Penalty) -> float:
    """N/2 - c^T beta + beta^T G beta / 2 + P_lambda(beta) = (1/2n)||y - X beta||^2 + P."""
    beta = np.asarray(beta, dtype=np.float64)
    return float(0.5 * N - c @ beta + 0.5 * beta @ (G @ beta) + penalty_value(beta, lam, pen))


def kkt_violation(G, c, beta, lam, pen: Penalty) -> float:
    """Largest violation of the stationarity / subgradient conditions at beta.

    With g = G beta - c (the gradient of the smooth part): lasso
    g_j + lambda w_j sign(beta_j) = 0 on the support, |g_j| <= lambda w_j off
    it; elastic net adds (1 - alpha) lambda w_j beta_j and uses alpha lambda w_j;
    MCP / SCAD use the derivative of their penalty (Table 1 forms); group lasso
    g_g + lambda c_k beta_g / ||beta_g|| = 0 or ||g_g|| <= lambda c_k.
    """
    beta = np.asarray(beta, dtype=np.float64)
    p = beta.size
    g = G @ beta - c
    if pen.kind in ("grp.lasso", "grp.mcp", "grp.scad"):
        # g_g + P'(||beta_g||) beta_g / ||beta_g|| = 0 on nonzero groups,
        # ||g_g|| <= P'(0) = lambda c_k on zero groups
        members, cg = pen.group_list(p)
        v = 0.0
        for k, m in enumerate(members):
            nb = float(np.linalg.norm(beta[m]))
            lk = lam * cg[k]
            if nb > 0:
                if pen.kind == "grp.lasso":
                    dp = lk
                elif pen.kind == "grp.mcp":
                    dp = max(lk - nb / pen.gamma, 0.0)
                else:
                    dp = lk if nb <= lk else max(pen.gamma * lk - nb, 0.0) / (pen.gamma - 1.0)
                v = max(v, float(np.linalg.norm(g[m] + dp * beta[m] / nb)))
            else:
                v = max(v, float(np.linalg.norm(g[m])) - lk)
        return max(v, 0.0)
    if pen.kind == "sgl":
        # nonzero group: g_j + lambda tau w_j sign(beta_j) + lambda (1 - tau)
        # c_k beta_j / ||beta_g|| = 0 where beta_j != 0, |g_j| <= lambda tau
        # w_j where beta_j = 0; zero group: ||S(g_g, lambda tau w_g)|| <=
        # lambda (1 - tau) c_k
        members, cg = pen.group_list(p)
        wt = pen.weights(p) * lam * pen.tau
        v = 0.0
        for k, m in enumerate(members):
            b = beta[m]
            nb = float(np.linalg.norm(b))
            lk = lam * (1.0 - pen.tau) * cg[k]
            if nb > 0:
                on = b != 0
                r = g[m] + wt[m] * np.sign(b) + lk * b / nb
                if on.any():
                    v = max(v, float(np.max(np.abs(r[on]))))
                if (~on).any():
                    v = max(v, float(np.max(np.abs(g[m][~on]) - wt[m][~on])))
            else:
                v = max(v, float(np.linalg.norm(np.maximum(np.abs(g[m]) - wt[m], 0.0))) - lk)
        return max(v, 0.0)
    wl = pen.weights(p) * lam
    a = np.abs(beta)
    s = np.sign(beta)
    on = a > 0
    if pen.kind == "lasso":
        on_v = np.abs(g + wl * s)
        off_t = wl
    elif pen.kind == "enet":
        on_v = np.abs(g + (1.0 - pen.alpha) * wl * beta + pen.alpha * wl * s)
        off_t = pen.alpha * wl
    elif pen.kind == "mcp":
        on_v = np.abs(g + s * np.maximum(wl - a / pen.gamma, 0.0))
        off_t = wl
    elif pen.kind == "scad":
        dp = np.where(a <= wl, wl, np.maximum(pen.gamma * wl - a, 0.0) / (pen.gamma - 1.0))
        on_v = np.abs(g + s * dp)
        off_t = wl
    else:
        raise ValueError(pen.kind)
    v_on = float(np.max(on_v[on])) if on.any() else 0.0
    v_off = float(np.max(np.abs(g[~on]) - off_t[~on])) if (~on).any() else 0.0
    return max(v_on, v_off, 0.0)


# ---------------------------------------------------------------------------
# Cross validation by fold statistics (Sections 3, 5.4-5.5)
# ---------------------------------------------------------------------------

def cv_mse(Gk_raw, ck_raw, Nk_raw, nk, beta):
    """Held-out mean squared error of fold k for coefficients beta (any shape
    (..., p)): ||y_k - X_k beta||^2 / n_k = (N_k - 2 beta^T c_k + beta^T G_k beta) / n_k,
    with the raw fold sums. Reading: the paper plots and summarises a CV mean
    squared error without defining it; this is the usual held-out MSE."""
    b = np.asarray(beta, dtype=np.float64)
    quad = np.einsum("...i,ij,...j->...", b, Gk_raw, b)
    return (Nk_raw - 2.0 * b @ ck_raw + quad) / nk


def cv_select(mse: np.ndarray):
    """From mse (K, L) return cvm, cvsd, idx_min, idx_1se (Section 5.4).

    cvm = mean over folds, cvsd = sample sd over folds / sqrt(K) (glmnet's
    convention). lambda.min = argmin cvm (ties -> larger lambda, i.e. the
    smaller index). lambda.1se = the largest lambda (smallest index) with
    cvm <= cvm[min] + cvsd[min].
    """
    K = mse.shape[0]
    cvm = mse.mean(0)
    cvsd = mse.std(0, ddof=1) / math.sqrt(K) if K > 1 else np.zeros_like(cvm)
    i_min = int(np.argmin(cvm))
    lim = cvm[i_min] + cvsd[i_min]
    i_1se = int(np.flatnonzero(cvm <= lim)[0])
    return cvm, cvsd, i_min, i_1se


@dataclass
class CVResult:
    full: list              # PathResult per penalty on the full data
    folds: list             # [k][pen] PathResult leaving fold k out
    lambdas: np.ndarray     # (npen, L)
    mse: np.ndarray         # (npen, K, L)
    cvm: np.ndarray         # (npen, L)
    cvsd: np.ndarray        # (npen, L)
    idx_min: np.ndarray     # (npen,)
    idx_1se: np.ndarray     # (npen,)
    best_penalty: int
    d: np.ndarray           # (K+1,)
    G: np.ndarray           # (K+1, p, p) scaled
    c: np.ndarray           # (K+1, p)


def xval(X, y, fold, K, pens: Sequence[Penalty], nlambda=100, lambda_min_ratio=1e-3,
         tol=1e-7, max_iter=10_000, lanczos_steps=64) -> CVResult:
    """K-fold cross validation by per-fold statistics (Section 3, xval.oem).

    Fold sums once; leave-fold-out statistics by subtraction; d_(k) per
    Gram; one lambda grid per penalty from the full-data statistics (reading:
    folds reuse the full-data grid so the CV error can be averaged per
    lambda); warm-started paths on the full data and on every leave-fold-out
    Gram; held-out MSE per fold; best penalty = lowest cvm at its lambda.min.
    """
    Gk, ck, Nk, nk = fold_gram_sums(X, y, fold, K)
    G, c, N, cnt = assemble_fold_grams(Gk, ck, Nk, nk)
    d = np.array([lanczos_d(G[b], lanczos_steps)[0] for b in range(K + 1)])
    lams = np.array([lambda_grid(lambda_max(c[0], pen), nlambda, lambda_min_ratio)
                     for pen in pens])
    full = [oem_path(G[0], c[0], d[0], pen, lams[i], tol, max_iter)
            for i, pen in enumerate(pens)]
    folds = [[oem_path(G[k + 1], c[k + 1], d[k + 1], pen, lams[i], tol, max_iter)
              for i, pen in enumerate(pens)] for k in range(K)]
    mse = np.zeros((len(pens), K, nlambda))
    for i in range(len(pens)):
        for k in range(K):
            mse[i, k] = cv_mse(Gk[k], ck[k], Nk[k], nk[k], folds[k][i].beta)
    sel = [cv_select(mse[i]) for i in range(len(pens))]
    cvm = np.array([s[0] for s in sel])
    cvsd = np.array([s[1] for s in sel])
    imin = np.array([s[2] for s in sel])
    i1se = np.array([s[3] for s in sel])
    best = int(np.argmin([cvm[i, imin[i]] for i in range(len(pens))]))
    return CVResult(full, folds, lams, mse, cvm, cvsd, imin, i1se, best, d, G, c)


# ---------------------------------------------------------------------------
# Centring, standardisation and the intercept
# ---------------------------------------------------------------------------
# Section 2.1 assumes standardized columns (sum_i x_ij^2 = 1; with the 1/n
# scaling above: unit second moment), and the package's API follows glmnet's
# (Section 5, API comparison with glmnet), where an unpenalised intercept and
# standardisation are options. Reading: with an intercept, X and y are
# centred by their means over the rows of the fit; with standardisation,
# column j is divided by sd_j = sqrt(G_c[j, j]) (the population sd of the
# centred column, or the root second moment without an intercept); penalties
# apply to the standardized coefficients; a column whose variance is zero
# (or below 1e-14 of its second moment) keeps scale 1 and drops out (zero
# coefficient). Coefficients are reported on the original scale:
# beta_j = beta_std_j / sd_j and beta_0 = ybar - mu^T beta.

def augmented_sums(X: np.ndarray, y: np.ndarray):
    """Raw sums of Z = [X | y | 1]: X^T X, X^T y, y^T y, X^T 1, y^T 1, n."""
    Xd = np.asarray(X, dtype=np.float64)
    yd = np.asarray(y, dtype=np.float64)
    return Xd.T @ Xd, Xd.T @ yd, float(yd @ yd), Xd.sum(0), float(yd.sum()), Xd.shape[0]


def centered_stats(Gr, cr, Nr, s, t, n, intercept: bool = True, standardize: bool = True):
    """Statistics (G, c, N) of the centred / scaled problem from the raw sums
    of one row set, and the maps back: (G, c, N, mu, sd, ybar, const).

    G = D (X^T X / n - mu mu^T) D, c = D (X^T y / n - mu ybar),
    N = y^T y / n - ybar^2, D = diag(1 / sd); mu, ybar = 0 without an intercept.
    """
    Gr = np.asarray(Gr, dtype=np.float64)
    cr = np.asarray(cr, dtype=np.float64)
    p = cr.size
    mu = np.asarray(s, dtype=np.float64) / n if intercept else np.zeros(p)
    ybar = float(t) / n if intercept else 0.0
    Gc = Gr / n - np.outer(mu, mu)
    cc = cr / n - mu * ybar
    Nc = float(Nr) / n - ybar * ybar
    raw2 = np.diag(Gr) / n
    var = np.diag(Gc).copy()
    const = ~(var > 1e-14 * raw2)
    if standardize:
        sd = np.where(const, 1.0, np.sqrt(np.where(const, 1.0, var)))
    else:
        sd = np.ones(p)
    keep = (~const).astype(np.float64)
    G = Gc / np.outer(sd, sd) * np.outer(keep, keep)
    c = cc / sd * keep
    return G, c, Nc, mu, sd, ybar, const


def back_transform(beta_std, mu, sd, ybar, intercept: bool = True):
    """Original-scale coefficients (beta, beta_0) of standardized beta_std
    (any leading shape (..., p))."""
    b = np.asarray(beta_std, dtype=np.float64) / sd
    b0 = (ybar - b @ mu) if intercept else np.zeros(b.shape[:-1])
    return b, b0


def cv_mse_intercept(Gk_raw, ck_raw, Nk_raw, sk, tk, nk, beta, beta0):
    """Held-out MSE of fold k for the model beta_0 + x^T beta from the raw
    sums of [X_k | y_k | 1]: ||y_k - beta_0 - X_k beta||^2 / n_k
    = (N_k - 2 beta_0 t_k - 2 beta^T c_k + n_k beta_0^2 + 2 beta_0 beta^T s_k
       + beta^T G_k beta) / n_k."""
    b = np.asarray(beta, dtype=np.float64)
    b0 = np.asarray(beta0, dtype=np.float64)
    quad = np.einsum("...i,ij,...j->...", b, Gk_raw, b)
    return (Nk_raw - 2.0 * b0 * tk - 2.0 * b @ ck_raw + nk * b0 * b0
            + 2.0 * b0 * (b @ sk) + quad) / nk


@dataclass
class FitResult:
    beta: np.ndarray        # (npen, L, p) original scale
    beta0: np.ndarray       # (npen, L)
    lambdas: np.ndarray     # (npen, L)
    paths: list             # PathResult per penalty (standardized problem)
    d: float
    G: np.ndarray           # the standardized G the paths ran on
    c: np.ndarray


def fit(X, y, pens: Sequence[Penalty], intercept: bool = True, standardize: bool = True,
        nlambda=100, lambda_min_ratio=1e-3, tol=1e-7, max_iter=10_000,
        lanczos_steps=64) -> FitResult:
    """oem() with the intercept / standardisation options: raw sums of
    [X | y | 1], the centred and scaled statistics, d, one lambda grid per
    penalty from the scaled c, warm-started paths, back to the original
    scale."""
    Gr, cr, Nr, s, t, n = augmented_sums(X, y)
    G, c, N, mu, sd, ybar, const = centered_stats(Gr, cr, Nr, s, t, n, intercept, standardize)
    d = lanczos_d(G, lanczos_steps)[0]
    lams = np.array([lambda_grid(lambda_max(c, pen), nlambda, lambda_min_ratio) for pen in pens])
    paths = [oem_path(G, c, d, pen, lams[i], tol, max_iter) for i, pen in enumerate(pens)]
    bs = np.stack([pr.beta for pr in paths])
    beta, beta0 = back_transform(bs, mu, sd, ybar, intercept)
    return FitResult(beta, beta0, lams, paths, d, G, c)


def xval_intercept(X, y, fold, K, pens: Sequence[Penalty], intercept: bool = True,
                   standardize: bool = True, nlambda=100, lambda_min_ratio=1e-3, tol=1e-7,
                   max_iter=10_000, lanczos_steps=64):
    """xval.oem with the intercept / standardisation options: every fit
    (full data and each leave-fold-out set) centres and scales by its own
    rows' statistics; held-out MSE by cv_mse_intercept on the raw fold sums.
    Returns (FitResult of the full data, mse (npen, K, L), cvm, cvsd,
    idx_min, idx_1se, best_penalty)."""
    X = np.asarray(X)
    y = np.asarray(y)
    sums = [augmented_sums(X[fold == k], y[fold == k]) for k in range(K)]
    tot = [sum(v[i] for v in sums) for i in range(6)]
    sets = [tot] + [[tot[i] - sums[k][i] for i in range(6)] for k in range(K)]
    stats = [centered_stats(*st, intercept, standardize) for st in sets]
    d = [lanczos_d(sb[0], lanczos_steps)[0] for sb in stats]
    lams = np.array([lambda_grid(lambda_max(stats[0][1], pen), nlambda, lambda_min_ratio)
                     for pen in pens])
    res = []
    for b in range(K + 1):
        G, c, N, mu, sd, ybar, const = stats[b]
        paths = [oem_path(G, c, d[b], pen, lams[i], tol, max_iter) for i, pen in enumerate(pens)]
        beta, beta0 = back_transform(np.stack([pr.beta for pr in paths]), mu, sd, ybar, intercept)
        res.append(FitResult(beta, beta0, lams, paths, d[b], G, c))
    mse = np.zeros((len(pens), K, nlambda))
    for i in range(len(pens)):
        for k in range(K):
            Gk, ck, Nk, sk, tk, nk = sums[k]
            mse[i, k] = cv_mse_intercept(Gk, ck, Nk, sk, tk, nk, res[k + 1].beta[i], res[k + 1].beta0[i])
    sel = [cv_select(mse[i]) for i in range(len(pens))]
    cvm = np.array([s_[0] for s_ in sel])
    cvsd = np.array([s_[1] for s_ in sel])
    imin = np.array([s_[2] for s_ in sel])
    i1se = np.array([s_[3] for s_ in sel])
    best = int(np.argmin([cvm[i, imin[i]] for i in range(len(pens))]))
    return res[0], mse, cvm, cvsd, imin, i1se, best


# ---------------------------------------------------------------------------
# Logistic regression (Section 4)
# ---------------------------------------------------------------------------
# Section 4: maximise the penalised log-likelihood by the proximal Newton
# algorithm of glmnet, with OEM as the inner solver of each weighted
# penalised least squares; the Hessian weights w_i = mu_i (1 - mu_i) may be
# replaced by their upper bound 1/4, which this build uses. Readings (the
# printed formulas are garbled: a '+' where the log-likelihood has '-', and
# the square missing from the weighted least squares): minimise
#   l(beta) = -(1/n) sum_i { y_i x_i^T beta - log(1 + exp(x_i^T beta)) } + P_lambda(beta);
# with w_i = 1/4 the surrogate at beta_t is
#   (1/2) beta^T G beta - c^T beta + P_lambda(beta),
#   G = Z^T Z / (4n), c = G beta_t + Z^T (y - mu(beta_t)) / n,
# (Z = [X | 1] with an unpenalised intercept), which majorises l up to a
# constant (the logistic loss has Hessian <= Z^T Z / (4n)): every outer step
# decreases the objective. Each surrogate is solved by OEM iterations warm
# started at beta_t (d >= lambda_1(G) by Lanczos); the outer loop stops with
# the inner stopping rule applied to successive outer iterates. lambda_max
# and the first warm start come from the null model (beta = 0, intercept
# logit(mean y)).

def sigmoid(t):
    t = np.asarray(t, dtype=np.float64)
    return np.where(t >= 0, 1.0 / (1.0 + np.exp(-np.abs(t))), np.exp(-np.abs(t)) / (1.0 + np.exp(-np.abs(t))))


def logistic_loss(Z, y, beta) -> float:
    """-(1/n) sum_i { y_i eta_i - log(1 + exp(eta_i)) }, eta = Z beta."""
    eta = np.asarray(Z, np.float64) @ beta
    return float(np.mean(np.logaddexp(0.0, eta) - np.asarray(y, np.float64) * eta))


@dataclass
class LogisticResult:
    beta: np.ndarray        # (L, p)
    beta0: np.ndarray       # (L,)
    lambdas: np.ndarray     # (L,)
    outer: np.ndarray       # (L,) outer (proximal Newton) steps
    iters: np.ndarray       # (L,) inner OEM iterations, summed over the outer steps
    converged: np.ndarray   # (L,)
    d: float
    trace: list             # (lambda index, objective after each outer step)


def logistic_path(X, y, pen: Penalty, nlambda=100, lambda_min_ratio=1e-3, lambdas=None,
                  intercept: bool = True, tol: float = 1e-7, max_iter: int = 10_000,
                  max_outer: int = 100, lanczos_steps: int = 64) -> LogisticResult:
    """Penalised logistic regression path (Section 4, Hessian bound 1/4)."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, p = X.shape
    Z = np.column_stack([X, np.ones(n)]) if intercept else X
    q = Z.shape[1]
    G = Z.T @ Z / (4.0 * n)
    d = lanczos_d(G, lanczos_steps)[0]
    w = np.concatenate([pen.weights(p), [0.0]]) if intercept else pen.weights(p)
    pe = Penalty(pen.kind, pen.alpha, pen.gamma, w)
    beta = np.zeros(q)
    if intercept:
        ybar = float(np.clip(y.mean(), 1e-12, 1 - 1e-12))
        beta[p] = math.log(ybar / (1.0 - ybar))
    g0 = Z.T @ (y - sigmoid(Z @ beta)) / n
    if lambdas is None:
        lambdas = lambda_grid(lambda_max(g0[:p], Penalty(pen.kind, pen.alpha, pen.gamma, pen.w)),
                              nlambda, lambda_min_ratio)
    lambdas = np.asarray(lambdas, dtype=np.float64)
    L = lambdas.size
    B = np.zeros((L, p))
    B0 = np.zeros(L)
    outer = np.zeros(L, dtype=np.int64)
    its = np.zeros(L, dtype=np.int64)
    conv = np.zeros(L, dtype=bool)
    trace = []
    for l, lam in enumerate(lambdas):
        for t in range(1, max_outer + 1):
            g = Z.T @ (y - sigmoid(Z @ beta)) / n
            c = G @ beta + g
            pr = oem_path(G, c, d, pe, [lam], tol, max_iter, beta0=beta)
            new = pr.beta[0]
            its[l] += int(pr.iters[0])
            delta = float(np.max(np.abs(new - beta)))
            beta = new
            trace.append((l, logistic_loss(Z, y, beta) + penalty_value(beta, lam, pe)))
            if delta <= tol * max(1.0, float(np.max(np.abs(beta)))):
                conv[l] = True
                break
        outer[l] = t
        B[l] = beta[:p]
        B0[l] = beta[p] if intercept else 0.0
    return LogisticResult(B, B0, lambdas, outer, its, conv, d, trace)
