"""Seeded synthetic inputs for the OEM penalized-regression path.

This module is the only code shared by the CUDA path's tests/benchmarks and the
FP64 oracle. It draws random designs, responses, true coefficients and fold
labels; it holds none of the method's arithmetic (no Gram, no eigenvalue, no
threshold, no iteration).

Designs follow the simulation settings of the paper:
  * AR(rho) rows, Sigma_ij = rho^|i-j| (Section "Timings / Cross validation":
    rho = 0.5, true beta_1..5 = (-0.5, -0.5, 0.5, 0.5, 1), noise sd 2);
  * exchangeable rows, Sigma_ij = rho for i != j (Section 5 examples);
  * block-correlated rows (groups of contiguous columns, rho_in within a
    group, rho_out across groups), generated by a factor model.

Every generator is deterministic given its seed and independent of the number
of worker threads: rows are drawn in fixed-size blocks, each block from its own
``numpy.random.SeedSequence`` child.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

ROW_BLOCK = 1 << 15  # rows per independently seeded block


def _block_seeds(seed: int, n: int, tag: int):
    nblk = (n + ROW_BLOCK - 1) // ROW_BLOCK
    ss = np.random.SeedSequence([int(seed), int(tag)])
    return ss.spawn(nblk)


def _fill_blocks(n: int, seed: int, tag: int, fn, threads: int | None = None):
    """Run fn(rng, r0, r1) over all row blocks (threaded, deterministic)."""
    seeds = _block_seeds(seed, n, tag)
    jobs = [(np.random.Generator(np.random.PCG64(s)), b * ROW_BLOCK,
             min(n, (b + 1) * ROW_BLOCK)) for b, s in enumerate(seeds)]
    if threads is None:
        threads = min(16, os.cpu_count() or 1)
    if threads <= 1 or len(jobs) == 1:
        for j in jobs:
            fn(*j)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda j: fn(*j), jobs))


def f32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even); return uint16 bits."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def bf16_bits_to_f64(b: np.ndarray) -> np.ndarray:
    """Exact widening of bfloat16 bit patterns to float64."""
    b = np.ascontiguousarray(b, dtype=np.uint16)
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def ar1_design(n: int, p: int, rho: float, seed: int, dtype=np.float32,
               threads: int | None = None) -> np.ndarray:
    """Rows iid N(0, Sigma), Sigma_ij = rho^|i-j| (the paper's CV design).

    x_1 = e_1, x_j = rho x_{j-1} + sqrt(1 - rho^2) e_j gives exactly that
    covariance. Returns an (n, p) C-contiguous array of ``dtype``
    (float32 / float64), or uint16 bfloat16 bits when dtype == "bf16".
    """
    out_dtype = np.float32 if dtype == "bf16" else dtype
    X = np.empty((n, p), dtype=out_dtype)
    s = math.sqrt(1.0 - rho * rho)

    def fn(rng, r0, r1):
        e = rng.standard_normal((p, r1 - r0), dtype=np.float64)
        for j in range(1, p):
            e[j] = rho * e[j - 1] + s * e[j]
        X[r0:r1] = e.T
    _fill_blocks(n, seed, 1, fn, threads)
    if dtype == "bf16":
        return f32_to_bf16_bits(X)
    return X


def exchangeable_design(n: int, p: int, rho: float, seed: int, dtype=np.float32,
                        threads: int | None = None) -> np.ndarray:
    """Rows iid N(0, Sigma), Sigma_ii = 1, Sigma_ij = rho (Section 5 examples)."""
    out_dtype = np.float32 if dtype == "bf16" else dtype
    X = np.empty((n, p), dtype=out_dtype)
    a, b = math.sqrt(rho), math.sqrt(1.0 - rho)

    def fn(rng, r0, r1):
        z0 = rng.standard_normal((r1 - r0, 1))
        e = rng.standard_normal((r1 - r0, p))
        X[r0:r1] = a * z0 + b * e
    _fill_blocks(n, seed, 2, fn, threads)
    if dtype == "bf16":
        return f32_to_bf16_bits(X)
    return X


def block_design(n: int, p: int, group_size: int, rho_in: float, rho_out: float,
                 seed: int, dtype="bf16", threads: int | None = None) -> np.ndarray:
    """Block-correlated rows: corr rho_in inside a group of contiguous columns,
    rho_out across groups. x_j = sqrt(rho_out) z0 + sqrt(rho_in - rho_out) z_g(j)
    + sqrt(1 - rho_in) e_j (a PSD factor model with exactly these correlations).
    """
    assert p % group_size == 0 and 0 <= rho_out <= rho_in < 1
    G = p // group_size
    out_dtype = np.float32 if dtype == "bf16" else dtype
    X = np.empty((n, p), dtype=out_dtype)
    a, b, c = math.sqrt(rho_out), math.sqrt(rho_in - rho_out), math.sqrt(1.0 - rho_in)

    def fn(rng, r0, r1):
        m = r1 - r0
        z0 = rng.standard_normal((m, 1))
        zg = rng.standard_normal((m, G))
        e = rng.standard_normal((m, p))
        X[r0:r1] = a * z0 + b * np.repeat(zg, group_size, axis=1) + c * e
    _fill_blocks(n, seed, 3, fn, threads)
    if dtype == "bf16":
        return f32_to_bf16_bits(X)
    return X


def as_f64(X: np.ndarray) -> np.ndarray:
    """Exact float64 view of a design stored as float32/float64/bf16 bits."""
    if X.dtype == np.uint16:
        return bf16_bits_to_f64(X)
    return X.astype(np.float64)


def response(X: np.ndarray, beta: np.ndarray, sigma: float, seed: int,
             dtype=np.float32, threads: int | None = None) -> np.ndarray:
    """y = X beta + sigma * eps, eps iid N(0,1); formed in float64, stored as dtype."""
    n = X.shape[0]
    y = np.empty(n, dtype=dtype)
    nz = np.flatnonzero(beta)
    bnz = np.asarray(beta, dtype=np.float64)[nz]

    def fn(rng, r0, r1):
        xb = as_f64(X[r0:r1][:, nz]) @ bnz if nz.size else np.zeros(r1 - r0)
        y[r0:r1] = xb + sigma * rng.standard_normal(r1 - r0)
    _fill_blocks(n, seed, 4, fn, threads)
    return y


def fold_ids(n: int, K: int, seed: int) -> np.ndarray:
    """Fold label floor(K * U) per row, U ~ Uniform(0,1); uint8."""
    assert 1 <= K <= 255
    out = np.empty(n, dtype=np.uint8)

    def fn(rng, r0, r1):
        out[r0:r1] = np.minimum((K * rng.random(r1 - r0)).astype(np.int64), K - 1)
    _fill_blocks(n, seed, 5, fn, 1)
    return out


def sparse_beta(p: int, nnz: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """nnz nonzeros at random positions, |beta_j| ~ U[lo, hi], random sign."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 6])))
    beta = np.zeros(p)
    pos = rng.choice(p, size=nnz, replace=False)
    beta[pos] = rng.uniform(lo, hi, nnz) * rng.choice([-1.0, 1.0], nnz)
    return beta


def group_beta(p: int, group_size: int, n_active: int, seed: int) -> np.ndarray:
    """n_active randomly chosen groups of contiguous columns with N(0,1) coefficients."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 7])))
    G = p // group_size
    beta = np.zeros(p)
    for g in rng.choice(G, size=n_active, replace=False):
        beta[g * group_size:(g + 1) * group_size] = rng.standard_normal(group_size)
    return beta


def leading_beta(p: int, head) -> np.ndarray:
    beta = np.zeros(p)
    beta[:len(head)] = head
    return beta


# ---------------------------------------------------------------------------
# Named workloads (sizes, distributions, penalties). Each is named by what it is.
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n: int
    p: int
    dtype: str              # "f64" | "f32" | "bf16"
    design: str             # "ar1" | "block" | "exch"
    rho: float = 0.5
    sigma: float = 1.0
    beta: str = "lead"      # "lead" | "sparse25" | "groups10"
    beta_head: tuple = ()
    K: int = 0              # folds (0 = no cross validation)
    penalties: tuple = ("lasso",)
    nlambda: int = 100
    lambda_min_ratio: float = 1e-3
    tol: float = 1e-7
    group_size: int = 0
    seed: int = 0
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "lasso_f64_n1e4_p50": Workload(
        "lasso_f64_n1e4_p50", 10_000, 50, "f64", "ar1", rho=0.5, sigma=1.0,
        beta="lead", beta_head=(2.0, -1.5, 1.0, -0.5, 0.25), seed=0),
    "four_penalties_f32_n1e6_p500": Workload(
        "four_penalties_f32_n1e6_p500", 1_000_000, 500, "f32", "ar1", rho=0.5,
        sigma=1.0, beta="sparse25",
        penalties=("lasso", "enet", "mcp", "scad"), seed=1,
        extra={"alpha": 0.5, "gamma_mcp": 3.0, "gamma_scad": 3.7}),
    # the same problem at n = 200,000 (X = 400 MB, above L2): profiler captures
    "four_penalties_f32_n2e5_p500": Workload(
        "four_penalties_f32_n2e5_p500", 200_000, 500, "f32", "ar1", rho=0.5,
        sigma=1.0, beta="sparse25",
        penalties=("lasso", "enet", "mcp", "scad"), seed=1,
        extra={"alpha": 0.5, "gamma_mcp": 3.0, "gamma_scad": 3.7}),
    "cv10_f32_n4e6_p200": Workload(
        "cv10_f32_n4e6_p200", 4_000_000, 200, "f32", "ar1", rho=0.5, sigma=2.0,
        beta="lead", beta_head=(-0.5, -0.5, 0.5, 0.5, 1.0), K=10,
        penalties=("lasso", "enet", "mcp", "scad"), seed=2,
        extra={"alpha": 0.5, "gamma_mcp": 3.0, "gamma_scad": 3.7}),
    "group_lasso_bf16_n2e6_p2000": Workload(
        "group_lasso_bf16_n2e6_p2000", 2_000_000, 2000, "bf16", "block",
        sigma=2.0, beta="groups10", penalties=("grp.lasso",), group_size=10,
        seed=3, extra={"rho_in": 0.7, "rho_out": 0.2, "n_active_groups": 10}),
    # the same problem at n = 200,000 (X = 800 MB, above L2) over a 20-lambda
    # grid of the same range: profiler captures
    "group_lasso_bf16_n2e5_p2000": Workload(
        "group_lasso_bf16_n2e5_p2000", 200_000, 2000, "bf16", "block",
        sigma=2.0, beta="groups10", penalties=("grp.lasso",), group_size=10, nlambda=20,
        seed=3, extra={"rho_in": 0.7, "rho_out": 0.2, "n_active_groups": 10}),
}


def make_beta(w: Workload) -> np.ndarray:
    if w.beta == "lead":
        return leading_beta(w.p, w.beta_head)
    if w.beta == "sparse25":
        return sparse_beta(w.p, 25, 0.5, 2.0, w.seed)
    if w.beta == "groups10":
        return group_beta(w.p, w.group_size, w.extra.get("n_active_groups", 10), w.seed)
    raise ValueError(w.beta)


def make_data(w: Workload, n: int | None = None, p: int | None = None,
              threads: int | None = None):
    """Return (X, y, fold or None, beta_true) for a workload (optionally resized).

    X is float64/float32 or uint16 bf16 bits; y is float64 for an f64 design,
    float32 otherwise.
    """
    n = w.n if n is None else n
    p = w.p if p is None else p
    ww = Workload(**{**w.__dict__, "n": n, "p": p})
    dt = {"f64": np.float64, "f32": np.float32, "bf16": "bf16"}[w.dtype]
    if w.design == "ar1":
        X = ar1_design(n, p, w.rho, w.seed, dt, threads)
    elif w.design == "exch":
        X = exchangeable_design(n, p, w.rho, w.seed, dt, threads)
    elif w.design == "block":
        X = block_design(n, p, w.group_size, w.extra["rho_in"], w.extra["rho_out"],
                         w.seed, dt, threads)
    else:
        raise ValueError(w.design)
    beta = make_beta(ww)
    ydt = np.float64 if w.dtype == "f64" else np.float32
    y = response(X, beta, w.sigma, w.seed, ydt, threads)
    fold = fold_ids(n, w.K, w.seed) if w.K else None
    return X, y, fold, beta


def random_orthonormal_design(n: int, p: int, seed: int) -> np.ndarray:
    """X with X^T X = n I exactly up to rounding (QR of a Gaussian matrix, times sqrt(n))."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 8])))
    Q, _ = np.linalg.qr(rng.standard_normal((n, p)))
    return Q * math.sqrt(n)


def serving_requests(num: int, seed: int, rate_per_s: float = 50.0,
                     n_range=(10_000, 2_000_000), p_range=(20, 1000),
                     cv_frac: float = 0.3, K: int = 5, nlambda: int = 50):
    """Poisson arrivals of mixed fit / CV jobs (log-uniform n, uniform p)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 9])))
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, num))
    reqs = []
    for i in range(num):
        n = int(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]))))
        p = int(rng.integers(p_range[0], p_range[1] + 1))
        reqs.append({
            "id": i, "arrival_s": float(t[i]), "n": n, "p": p,
            "K": K if rng.random() < cv_frac else 0,
            "penalty": "lasso" if rng.random() < 0.5 else "mcp",
            "gamma": 3.0, "nlambda": nlambda, "seed": int(seed * 100003 + i),
        })
    return reqs


def ar1_coefficients(p: int, rho: float) -> np.ndarray:
    """The p x p lower-triangular C with x = C e for the AR(rho) recurrence
    x_1 = e_1, x_j = rho x_{j-1} + sqrt(1 - rho^2) e_j."""
    s = math.sqrt(1.0 - rho * rho)
    j = np.arange(p)
    C = np.power(rho, np.maximum(j[:, None] - j[None, :], 0).astype(np.float64))
    C = np.tril(C)
    C[:, 1:] *= s
    return C


def device_ar1_base(n: int, p: int, rho: float, seed: int, device="cuda", chunk: int = 1 << 18):
    """n x p float32 AR(rho) rows drawn on the GPU (torch), X = E C^T block by
    block. Any row window and column prefix of it is again an AR(rho) sample."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    Ct = torch.from_numpy(ar1_coefficients(p, rho).T.copy()).to(device=device, dtype=torch.float32)
    X = torch.empty((n, p), dtype=torch.float32, device=device)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        E = torch.randn((r1 - r0, p), generator=g, device=device, dtype=torch.float32)
        X[r0:r1] = E @ Ct
    return X


def device_request_data(base, req: dict, beta_head=(-0.5, -0.5, 0.5, 0.5, 1.0), sigma=2.0):
    """X (a row window / column prefix view of a base matrix), y = X beta +
    sigma eps and fold labels on the device for one serving request."""
    import torch
    n, p, K, seed = req["n"], req["p"], req["K"], req["seed"]
    N = base.shape[0]
    r0 = (seed * 7919) % max(1, N - n + 1)
    X = base[r0:r0 + n, :p]
    g = torch.Generator(device=base.device)
    g.manual_seed(int(seed))
    beta = torch.zeros(p, dtype=torch.float32, device=base.device)
    h = torch.tensor(beta_head[:p], dtype=torch.float32, device=base.device)
    beta[:h.numel()] = h
    y = X @ beta + sigma * torch.randn(n, generator=g, device=base.device, dtype=torch.float32)
    fold = torch.randint(0, K, (n,), generator=g, device=base.device, dtype=torch.uint8) if K else None
    return X, y.contiguous(), fold
