"""ctypes binding of liboem.so (include/oem.h). Argument marshalling only.

Every function here has the name of the C entry point it calls and takes the
same arguments, with device arrays given as torch CUDA tensors (their
data_ptr() is passed) and host arrays as numpy arrays or Python sequences.
There is no fallback: if the library is missing, importing this module
raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("OEM_LIB", os.path.join(_HERE, "_build", "liboem.so"))

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"liboem.so not found at {LIB_PATH}; build it first "
        "(python -c 'import __graft_entry__ as g; g.build()')")
lib = C.CDLL(LIB_PATH)

# status codes and enums (include/oem.h)
OEM_OK, OEM_WARN_NOTCONV = 0, 1
OEM_EINVAL, OEM_ENOMEM, OEM_EBUDGET, OEM_ECUDA = -1, -2, -3, -4
OEM_ENONFINITE, OEM_ETIMEOUT, OEM_EUNSUPPORTED = -5, -6, -7
OEM_F64, OEM_F32, OEM_BF16 = 0, 1, 2
OEM_GRAM_FP64, OEM_GRAM_FP32, OEM_GRAM_TF32 = 0, 1, 2
OEM_GRAM_BF16, OEM_GRAM_SPLIT_BF16, OEM_GRAM_AUTO = 3, 4, 5
OEM_LASSO, OEM_ENET, OEM_MCP, OEM_SCAD, OEM_GROUP_LASSO = 0, 1, 2, 3, 4
OEM_GROUP_MCP, OEM_GROUP_SCAD, OEM_SPARSE_GROUP_LASSO = 5, 6, 7
OEM_ITER_F32, OEM_ITER_F64 = 0, 1

KIND = {"lasso": OEM_LASSO, "enet": OEM_ENET, "mcp": OEM_MCP, "scad": OEM_SCAD,
        "grp.lasso": OEM_GROUP_LASSO, "grp.mcp": OEM_GROUP_MCP, "grp.scad": OEM_GROUP_SCAD,
        "sgl": OEM_SPARSE_GROUP_LASSO}
MODE = {"fp64": OEM_GRAM_FP64, "fp32": OEM_GRAM_FP32, "tf32": OEM_GRAM_TF32,
        "bf16": OEM_GRAM_BF16, "split_bf16": OEM_GRAM_SPLIT_BF16, "auto": OEM_GRAM_AUTO}

EXPORTED = ["oem_options_default", "oem_create", "oem_destroy", "oem_last_error", "oem_sync",
            "oem_kernel_launches", "oem_iter_stats", "oem_profile_enable", "oem_profile_get", "oem_profile_name",
            "oem_gram", "oem_gram_noalloc", "oem_fold_grams", "oem_spectral_d", "oem_fit_path",
            "oem_fit", "oem_cv", "oem_fit_logistic", "oem_server_create", "oem_server_submit", "oem_server_poll",
            "oem_server_result", "oem_server_stats", "oem_server_destroy"]
OEM_PROF_NKERNELS = 12


class oem_penalty(C.Structure):
    _fields_ = [("kind", C.c_int32), ("alpha", C.c_double), ("gamma", C.c_double),
                ("w", C.POINTER(C.c_double)), ("group", C.POINTER(C.c_int32)),
                ("cg", C.POINTER(C.c_double)), ("ngroups", C.c_int32)]


class oem_options(C.Structure):
    _fields_ = [("nlambda", C.c_int32), ("lambda_min_ratio", C.c_double),
                ("lambdas", C.POINTER(C.c_double)), ("tol", C.c_double),
                ("max_iter", C.c_int64), ("lanczos_steps", C.c_int32),
                ("gram_mode", C.c_int32), ("iter_precision", C.c_int32),
                ("cluster_ctas", C.c_int32), ("instances_per_task", C.c_int32),
                ("autotune", C.c_int32), ("intercept", C.c_int32), ("standardize", C.c_int32)]


class oem_job(C.Structure):
    _fields_ = [("X", C.c_void_p), ("xtype", C.c_int32), ("n", C.c_int64), ("p", C.c_int64),
                ("ldx", C.c_int64), ("y", C.c_void_p), ("fold", C.c_void_p), ("K", C.c_int32),
                ("pen", oem_penalty), ("nlambda", C.c_int32), ("lambda_min_ratio", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int64), ("gram_mode", C.c_int32)]


OEM_SERVE_BATCHED, OEM_SERVE_PLAIN = 0, 1
JOB_STATES = {0: "queued", 1: "prep", 2: "iter", 3: "finish", 4: "done", 5: "failed"}

_vp, _i32, _i64, _d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_sigs = {
    "oem_options_default": (None, [C.POINTER(oem_options)]),
    "oem_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_size_t]),
    "oem_destroy": (C.c_int, [_vp]),
    "oem_last_error": (C.c_char_p, [_vp]),
    "oem_sync": (C.c_int, [_vp, _vp]),
    "oem_kernel_launches": (C.c_int64, [_vp]),
    "oem_iter_stats": (C.c_int, [_vp, _vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "oem_profile_enable": (C.c_int, [_vp, C.c_int]),
    "oem_profile_get": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "oem_profile_name": (C.c_char_p, [C.c_int]),
    "oem_gram": (C.c_int, [_vp, _vp, _i32, _i64, _i64, _i64, _vp, _i32, _vp, _vp, _vp, _vp]),
    "oem_gram_noalloc": (C.c_int, [_vp, _i32, _i64, _i64, _i64, _vp, _i32, _vp, _vp, _vp, _vp]),
    "oem_fold_grams": (C.c_int, [_vp, _vp, _i32, _i64, _i64, _i64, _vp, _vp, _i32, _i32,
                                 _vp, _vp, _vp, _vp, _vp]),
    "oem_spectral_d": (C.c_int, [_vp, _vp, _i64, _i64, _i32, _i64, _i32, _vp, _vp]),
    "oem_fit_path": (C.c_int, [_vp, _vp, _vp, _i64, _d, C.POINTER(oem_penalty), _i32,
                               C.POINTER(oem_options), _vp, _vp, _vp, _vp, _vp]),
    "oem_fit": (C.c_int, [_vp, _vp, _i32, _i64, _i64, _i64, _vp, C.POINTER(oem_penalty), _i32,
                          C.POINTER(oem_options), _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "oem_cv": (C.c_int, [_vp, _vp, _i32, _i64, _i64, _i64, _vp, _vp, _i32,
                         C.POINTER(oem_penalty), _i32, C.POINTER(oem_options), _vp, _vp, _vp,
                         _vp, _vp, _vp, _vp, _vp, _vp]),
    "oem_fit_logistic": (C.c_int, [_vp, _vp, _i32, _i64, _i64, _i64, _vp, C.POINTER(oem_penalty), _i32,
                                   C.POINTER(oem_options), _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "oem_server_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_size_t, _i32, _i64]),
    "oem_server_submit": (C.c_int, [_vp, C.POINTER(oem_job), C.POINTER(C.c_int64)]),
    "oem_server_poll": (C.c_int, [_vp, _i64, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "oem_server_result": (C.c_int, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "oem_server_stats": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "oem_server_destroy": (C.c_int, [_vp]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class OemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"oem error {code}: {msg}")
        self.code = code


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return int(t.data_ptr())


def _out_device(ctx, X):
    """Outputs live on the context's device, also when X is in host memory."""
    import torch
    return X.device if X.is_cuda else torch.device("cuda", ctx.device)


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    return int(stream)


@dataclass
class Penalty:
    """A penalty of Table 1 for the C call (host data). tau is the sparse
    group lasso's split (passed in the ABI's alpha field)."""
    kind: str
    alpha: float = 1.0
    gamma: float = 3.0
    w: Optional[Sequence[float]] = None
    groups: Optional[Sequence[int]] = None
    cg: Optional[Sequence[float]] = None
    tau: float = 0.5


class _PenArray:
    """Keeps the host arrays of an oem_penalty[] alive during a call."""

    def __init__(self, pens: Sequence[Penalty]):
        self.keep = []
        arr = (oem_penalty * len(pens))()
        for i, p in enumerate(pens):
            arr[i].kind = KIND[p.kind]
            arr[i].alpha = float(p.tau if p.kind == "sgl" else p.alpha)
            arr[i].gamma = float(p.gamma)
            if p.w is not None:
                w = np.ascontiguousarray(p.w, dtype=np.float64)
                self.keep.append(w)
                arr[i].w = w.ctypes.data_as(C.POINTER(C.c_double))
            if p.groups is not None:
                g = np.ascontiguousarray(p.groups, dtype=np.int32)
                self.keep.append(g)
                arr[i].group = g.ctypes.data_as(C.POINTER(C.c_int32))
                arr[i].ngroups = int(g.max()) + 1 if g.size else 0
            if p.cg is not None:
                cgv = np.ascontiguousarray(p.cg, dtype=np.float64)
                self.keep.append(cgv)
                arr[i].cg = cgv.ctypes.data_as(C.POINTER(C.c_double))
        self.arr = arr
        self.n = len(pens)


def make_options(nlambda=100, lambda_min_ratio=1e-3, lambdas=None, tol=1e-7, max_iter=10000,
                 lanczos_steps=64, gram_mode="auto", iter_precision="f32", cluster_ctas=0,
                 instances_per_task=0, autotune=True, intercept=False, standardize=False):
    o = oem_options()
    lib.oem_options_default(C.byref(o))
    o.nlambda = int(nlambda)
    o.lambda_min_ratio = float(lambda_min_ratio)
    keep = None
    if lambdas is not None:
        keep = np.ascontiguousarray(lambdas, dtype=np.float64)
        o.lambdas = keep.ctypes.data_as(C.POINTER(C.c_double))
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.lanczos_steps = int(lanczos_steps)
    o.gram_mode = MODE[gram_mode] if isinstance(gram_mode, str) else int(gram_mode)
    o.iter_precision = OEM_ITER_F64 if iter_precision == "f64" else OEM_ITER_F32
    o.cluster_ctas = int(cluster_ctas)
    o.instances_per_task = int(instances_per_task)
    o.autotune = 1 if autotune else 0
    o.intercept = 1 if intercept else 0
    o.standardize = 1 if standardize else 0
    o._keep = keep
    return o


class Context:
    """Owns one oem_ctx (device, workspace budget)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        h = C.c_void_p()
        rc = lib.oem_create(C.byref(h), int(device), C.c_size_t(int(budget_bytes)))
        if rc != OEM_OK:
            raise OemError(rc, "oem_create failed")
        self.h = h
        self.device = int(device)

    def close(self):
        if self.h:
            lib.oem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self) -> str:
        return lib.oem_last_error(self.h).decode()

    def check(self, rc: int) -> int:
        if rc < 0:
            raise OemError(rc, self.error())
        return rc

    def sync(self, stream=None) -> int:
        return self.check(lib.oem_sync(self.h, _stream(stream)))

    def launches(self) -> int:
        return int(lib.oem_kernel_launches(self.h))

    def iter_stats(self, stream=None):
        """(iterations, loop trips) of the last fit / cross validation."""
        it, tr = C.c_int64(), C.c_int64()
        self.check(lib.oem_iter_stats(self.h, _stream(stream), C.byref(it), C.byref(tr)))
        return int(it.value), int(tr.value)

    def profile(self, enable: bool = True):
        self.check(lib.oem_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kernel name: (device ms, launches)} accumulated since profile()."""
        out = {}
        for k in range(OEM_PROF_NKERNELS):
            ms, n = C.c_double(), C.c_int64()
            self.check(lib.oem_profile_get(self.h, k, C.byref(ms), C.byref(n)))
            if n.value:
                out[lib.oem_profile_name(k).decode()] = (ms.value, n.value)
        return out


def padded(X, device="cuda"):
    """Device copy of a 2-D array whose row stride is a multiple of 16 bytes
    (the ABI's rule for X), returned as the n x p view of that buffer."""
    import torch
    t = X if isinstance(X, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(X))
    if t.dim() != 2:
        return t.to(device)
    n, p = t.shape
    per = 16 // t.element_size()
    ld = (p + per - 1) // per * per
    buf = torch.zeros((n, ld), dtype=t.dtype, device=device)
    buf[:, :p] = t.to(device)
    return buf[:, :p]


def _xtype(X) -> int:
    import torch
    if X.dtype == torch.float64:
        return OEM_F64
    if X.dtype == torch.float32:
        return OEM_F32
    if X.dtype == torch.bfloat16:
        return OEM_BF16
    raise TypeError(f"unsupported X dtype {X.dtype}")


def oem_gram(ctx: Context, X, y, mode="auto", G=None, c=None, yty=None, stream=None):
    import torch
    n, p = X.shape
    dev = _out_device(ctx, X)
    G = torch.empty((p, p), dtype=torch.float64, device=dev) if G is None else G
    c = torch.empty(p, dtype=torch.float64, device=dev) if c is None else c
    yty = torch.empty(1, dtype=torch.float64, device=dev) if yty is None else yty
    ctx.check(lib.oem_gram(ctx.h, _ptr(X), _xtype(X), n, p, X.stride(0), _ptr(y),
                           MODE[mode] if isinstance(mode, str) else int(mode),
                           _ptr(G), _ptr(c), _ptr(yty), _stream(stream)))
    return G, c, yty


def oem_gram_noalloc(X, y, mode="auto", G=None, c=None, yty=None, stream=None):
    """oem_gram without device allocation or context (see include/oem.h).
    X, y and the outputs must be CUDA tensors of one device; the call runs
    with that device current."""
    import torch
    if not (X.is_cuda and y.is_cuda):
        raise TypeError("oem_gram_noalloc takes X and y in device memory (CUDA tensors)")
    n, p = X.shape
    dev = X.device
    G = torch.empty((p, p), dtype=torch.float64, device=dev) if G is None else G
    c = torch.empty(p, dtype=torch.float64, device=dev) if c is None else c
    yty = torch.empty(1, dtype=torch.float64, device=dev) if yty is None else yty
    if any(t.device != dev for t in (y, G, c, yty)):
        raise ValueError("oem_gram_noalloc: X, y, G, c, yty must be on one device")
    with torch.cuda.device(dev):
        rc = lib.oem_gram_noalloc(_ptr(X), _xtype(X), n, p, X.stride(0), _ptr(y),
                                  MODE[mode] if isinstance(mode, str) else int(mode),
                                  _ptr(G), _ptr(c), _ptr(yty), _stream(stream))
    if rc < 0:
        raise OemError(rc, "oem_gram_noalloc rejected the call")
    return G, c, yty


def oem_fold_grams(ctx: Context, X, y, fold, K, mode="auto", stream=None):
    import torch
    n, p = X.shape
    dev = _out_device(ctx, X)
    Gk = torch.empty((K, p, p), dtype=torch.float64, device=dev)
    ck = torch.empty((K, p), dtype=torch.float64, device=dev)
    ytyk = torch.empty(K, dtype=torch.float64, device=dev)
    nk = torch.empty(K, dtype=torch.int64, device=dev)
    ctx.check(lib.oem_fold_grams(ctx.h, _ptr(X), _xtype(X), n, p, X.stride(0), _ptr(y), _ptr(fold),
                                 int(K), MODE[mode] if isinstance(mode, str) else int(mode),
                                 _ptr(Gk), _ptr(ck), _ptr(ytyk), _ptr(nk), _stream(stream)))
    return Gk, ck, ytyk, nk


def oem_spectral_d(ctx: Context, G, steps=64, stream=None):
    import torch
    if G.dim() == 2:
        G = G.unsqueeze(0)
    B, p, _ = G.shape
    d = torch.empty(B, dtype=torch.float64, device=G.device)
    ctx.check(lib.oem_spectral_d(ctx.h, _ptr(G), p, G.stride(1), B, G.stride(0), int(steps),
                                 _ptr(d), _stream(stream)))
    return d


def _path_outputs(npen, L, p, dev):
    import torch
    return (torch.empty((npen, L, p), dtype=torch.float64, device=dev),
            torch.empty((npen, L), dtype=torch.float64, device=dev),
            torch.empty((npen, L), dtype=torch.int32, device=dev),
            torch.empty((npen, L), dtype=torch.uint8, device=dev))


def oem_fit_path(ctx: Context, G, c, pens: Sequence[Penalty], d: float = 0.0, stream=None, **opts):
    p = c.shape[0]
    o = make_options(**opts)
    P = _PenArray(pens)
    beta, lam, its, conv = _path_outputs(P.n, o.nlambda, p, c.device)
    ctx.check(lib.oem_fit_path(ctx.h, _ptr(G), _ptr(c), p, float(d), P.arr, P.n, C.byref(o),
                               _ptr(beta), _ptr(lam), _ptr(its), _ptr(conv), _stream(stream)))
    return beta, lam, its, conv


def oem_fit(ctx: Context, X, y, pens: Sequence[Penalty], stream=None, out=None, **opts):
    """oem_fit; returns (beta, lambdas, iters, converged, d), and the
    intercepts beta0 as a sixth element when intercept or standardize is set."""
    import torch
    n, p = X.shape
    o = make_options(**opts)
    P = _PenArray(pens)
    dev = _out_device(ctx, X)
    if out is None:
        beta, lam, its, conv = _path_outputs(P.n, o.nlambda, p, dev)
        d = torch.empty(1, dtype=torch.float64, device=dev)
    else:
        beta, lam, its, conv, d = out
    centred = bool(o.intercept or o.standardize)
    beta0 = torch.empty((P.n, o.nlambda), dtype=torch.float64, device=dev) if centred else None
    ctx.check(lib.oem_fit(ctx.h, _ptr(X), _xtype(X), n, p, X.stride(0), _ptr(y), P.arr, P.n,
                          C.byref(o), _ptr(beta), _ptr(lam), _ptr(its), _ptr(conv), _ptr(d),
                          _ptr(beta0), _stream(stream)))
    if centred:
        return beta, lam, its, conv, d, beta0
    return beta, lam, its, conv, d


def cv_outputs(npen, L, p, dev):
    """Output buffers of oem_cv (a dict of device tensors)."""
    import torch
    return {"beta": torch.empty((npen, L, p), dtype=torch.float64, device=dev),
            "beta0": torch.empty((npen, L), dtype=torch.float64, device=dev),
            "lambdas": torch.empty((npen, L), dtype=torch.float64, device=dev),
            "cvm": torch.empty((npen, L), dtype=torch.float64, device=dev),
            "cvsd": torch.empty((npen, L), dtype=torch.float64, device=dev),
            "idx_min": torch.empty(npen, dtype=torch.int32, device=dev),
            "idx_1se": torch.empty(npen, dtype=torch.int32, device=dev),
            "best_penalty": torch.empty(1, dtype=torch.int32, device=dev)}


def oem_cv(ctx: Context, X, y, fold, K, pens: Sequence[Penalty], stream=None, out=None, **opts):
    n, p = X.shape
    o = make_options(**opts)
    P = _PenArray(pens)
    L = o.nlambda
    dev = _out_device(ctx, X)
    r = cv_outputs(P.n, L, p, dev) if out is None else out
    beta, lam, cvm, cvsd = r["beta"], r["lambdas"], r["cvm"], r["cvsd"]
    imin, i1se, best, beta0 = r["idx_min"], r["idx_1se"], r["best_penalty"], r["beta0"]
    ctx.check(lib.oem_cv(ctx.h, _ptr(X), _xtype(X), n, p, X.stride(0), _ptr(y), _ptr(fold), int(K),
                         P.arr, P.n, C.byref(o), _ptr(beta), _ptr(lam), _ptr(cvm), _ptr(cvsd),
                         _ptr(imin), _ptr(i1se), _ptr(best), _ptr(beta0), _stream(stream)))
    return r


def oem_fit_logistic(ctx: Context, X, y, pens: Sequence[Penalty], stream=None, **opts):
    """Penalised logistic regression path; returns (beta, beta0, lambdas,
    iters, converged, d)."""
    import torch
    n, p = X.shape
    o = make_options(**opts)
    P = _PenArray(pens)
    beta, lam, its, conv = _path_outputs(P.n, o.nlambda, p, X.device)
    beta0 = torch.empty((P.n, o.nlambda), dtype=torch.float64, device=X.device)
    d = torch.empty(1, dtype=torch.float64, device=X.device)
    ctx.check(lib.oem_fit_logistic(ctx.h, _ptr(X), _xtype(X), n, p, X.stride(0), _ptr(y), P.arr, P.n,
                                   C.byref(o), _ptr(beta), _ptr(beta0), _ptr(lam), _ptr(its), _ptr(conv),
                                   _ptr(d), _stream(stream)))
    return beta, beta0, lam, its, conv, d


class Server:
    """A serving loop (oem_server_*): submit fit / CV jobs on device-resident
    data as they arrive; the library admits them under the memory budget and
    batches their OEM iterations (form "batched") or runs them one by one
    with per-iteration launches (form "plain")."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, form: str = "batched",
                 iters_per_round: int = 2000):
        h = C.c_void_p()
        f = OEM_SERVE_PLAIN if form == "plain" else OEM_SERVE_BATCHED
        rc = lib.oem_server_create(C.byref(h), int(device), C.c_size_t(int(budget_bytes)), f,
                                   int(iters_per_round))
        if rc != OEM_OK:
            raise OemError(rc, "oem_server_create failed")
        self.h = h
        self._keep = {}
        self._shape = {}

    def submit(self, X, y, pen: Penalty, fold=None, K: int = 0, nlambda: int = 50,
               lambda_min_ratio: float = 1e-3, tol: float = 1e-7, max_iter: int = 10000,
               gram_mode="auto") -> int:
        n, p = X.shape
        P = _PenArray([pen])
        j = oem_job()
        j.X, j.xtype, j.n, j.p, j.ldx = _ptr(X), _xtype(X), n, p, X.stride(0)
        j.y = _ptr(y)
        j.fold = _ptr(fold) if fold is not None else None
        j.K = int(K)
        j.pen = P.arr[0]
        j.nlambda, j.lambda_min_ratio, j.tol, j.max_iter = int(nlambda), float(lambda_min_ratio), \
            float(tol), int(max_iter)
        j.gram_mode = MODE[gram_mode] if isinstance(gram_mode, str) else int(gram_mode)
        jid = C.c_int64()
        rc = lib.oem_server_submit(self.h, C.byref(j), C.byref(jid))
        if rc != OEM_OK:
            raise OemError(rc, "oem_server_submit rejected the job")
        self._keep[jid.value] = (X, y, fold, P)
        self._shape[jid.value] = (p, int(nlambda), int(K))
        return jid.value

    def poll(self, jid: int):
        st, lat = C.c_int32(), C.c_double()
        rc = lib.oem_server_poll(self.h, int(jid), C.byref(st), C.byref(lat))
        return JOB_STATES.get(st.value, "?"), lat.value, rc

    def wait(self, jid: int, timeout_s: float = 600.0):
        import time
        t0 = time.time()
        while True:
            st, lat, rc = self.poll(jid)
            if st in ("done", "failed"):
                return st, lat, rc
            if time.time() - t0 > timeout_s:
                raise TimeoutError(f"job {jid} still {st}")
            time.sleep(0.0005)

    def result(self, jid: int) -> dict:
        p, L, K = self._shape[jid]
        beta = np.empty((L, p))
        lam = np.empty(L)
        cvm = np.empty(L)
        cvsd = np.empty(L)
        imin, i1se, its = C.c_int32(-1), C.c_int32(-1), C.c_int64()
        rc = lib.oem_server_result(self.h, int(jid), beta.ctypes.data, lam.ctypes.data,
                                   cvm.ctypes.data, cvsd.ctypes.data, C.addressof(imin),
                                   C.addressof(i1se), C.addressof(its))
        if rc != OEM_OK:
            raise OemError(rc, f"job {jid} has no result")
        self._keep.pop(jid, None)
        out = {"beta": beta, "lambdas": lam, "iters": its.value}
        if K:
            out.update(cvm=cvm, cvsd=cvsd, idx_min=imin.value, idx_1se=i1se.value)
        return out

    def stats(self) -> dict:
        v = [C.c_int64() for _ in range(5)]
        lib.oem_server_stats(self.h, *[C.addressof(x) for x in v])
        return dict(zip(("jobs_done", "paths_done", "launches", "rounds", "peak_bytes"),
                        [x.value for x in v]))

    def close(self):
        if self.h:
            lib.oem_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
