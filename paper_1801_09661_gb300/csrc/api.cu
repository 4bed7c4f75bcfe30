// C-ABI entry points (include/oem.h): argument validation, the per-context
// workspace arena, and the order of kernels for each call.
#include "oem_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

using namespace oem;

struct oem_ctx {
  int device = 0;
  int num_sms = kNumSMsHint;
  size_t budget = 0;
  void* arena = nullptr;
  size_t arena_cap = 0;
  cudaStream_t arena_stream = nullptr;
  unsigned* dstatus = nullptr;
  int64_t launches = 0;
  char err[512] = {0};
  // per-kernel profiling (events around launches while enabled)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Pending { int cls; cudaEvent_t e0, e1; int64_t n; };
  std::vector<Pending> pending;
  double prof_ms[OEM_PROF_NKERNELS] = {0};
  int64_t prof_n[OEM_PROF_NKERNELS] = {0};
};

namespace {

int fail(oem_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CU(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, OEM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

cudaEvent_t prof_event(oem_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

// Bracket a launch (or a launch sequence of `n` kernels) with events.
struct ProfScope {
  oem_ctx* ctx;
  cudaStream_t s;
  int cls;
  int64_t n;
  cudaEvent_t e0 = nullptr;
  ProfScope(oem_ctx* c, cudaStream_t st, int k, int64_t cnt) : ctx(c), s(st), cls(k), n(cnt) {
    if (ctx->prof && (e0 = prof_event(ctx))) cudaEventRecord(e0, s);
  }
  ~ProfScope() {
    if (!e0) return;
    cudaEvent_t e1 = prof_event(ctx);
    if (!e1) { ctx->ev_pool.push_back(e0); return; }
    cudaEventRecord(e1, s);
    ctx->pending.push_back({cls, e0, e1, n});
  }
};

#define LAUNCH(cls, call)                                                                \
  do {                                                                                   \
    cudaError_t e_;                                                                      \
    {                                                                                    \
      ProfScope ps_(ctx, s, (cls), 1);                                                   \
      e_ = (call);                                                                       \
    }                                                                                    \
    ++ctx->launches;                                                                     \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, OEM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

cudaError_t lanczos_prof(oem_ctx* ctx, cudaStream_t s, const double* G, int64_t p, int64_t ldg,
                         int batch, int64_t strideG, int steps, LanczosWork w, double* d,
                         cudaStream_t s2, int64_t* launches) {
  const int64_t before = *launches;
  cudaEvent_t e0 = ctx->prof ? prof_event(ctx) : nullptr;
  if (e0) cudaEventRecord(e0, s);
  cudaError_t e = launch_lanczos(G, p, ldg, batch, strideG, steps, w, d, s2, launches);
  if (e0) {
    cudaEvent_t e1 = prof_event(ctx);
    if (e1) {
      cudaEventRecord(e1, s);
      ctx->pending.push_back({OEM_PROF_LANCZOS, e0, e1, *launches - before});
    } else {
      ctx->ev_pool.push_back(e0);
    }
  }
  return e;
}

// Bump allocator over one stream-ordered block per call.
struct Arena {
  std::vector<std::pair<void**, size_t>> req;
  template <typename P>
  void add(P** ptr, size_t count) { req.push_back({(void**)ptr, sizeof(P) * count}); }
  size_t total() const {
    size_t t = 0;
    for (auto& r : req) t += (r.second + 255) & ~(size_t)255;
    return t;
  }
};

int arena_commit(oem_ctx* ctx, Arena& A, cudaStream_t s) {
  const size_t need = A.total();
  if (need > ctx->budget)
    return fail(ctx, OEM_EBUDGET, "workspace of %zu bytes exceeds the budget of %zu bytes", need,
                ctx->budget);
  if (need > ctx->arena_cap) {
    if (ctx->arena) CU(cudaFreeAsync(ctx->arena, ctx->arena_stream ? ctx->arena_stream : s));
    ctx->arena = nullptr;
    ctx->arena_cap = 0;
    cudaError_t e = cudaMallocAsync(&ctx->arena, need, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, OEM_ENOMEM, "workspace allocation of %zu bytes failed", need);
    }
    ctx->arena_cap = need;
  }
  ctx->arena_stream = s;
  char* p = (char*)ctx->arena;
  for (auto& r : A.req) {
    *r.first = r.second ? p : nullptr;
    p += (r.second + 255) & ~(size_t)255;
  }
  return OEM_OK;
}

size_t elem_size(int32_t xtype) { return xtype == OEM_F64 ? 8 : xtype == OEM_F32 ? 4 : 2; }

int check_x(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
            const void* y) {
  if (xtype != OEM_F64 && xtype != OEM_F32 && xtype != OEM_BF16)
    return fail(ctx, OEM_EINVAL, "xtype %d is not OEM_F64/OEM_F32/OEM_BF16", xtype);
  if (n < 1 || p < 1) return fail(ctx, OEM_EINVAL, "n=%lld, p=%lld must be >= 1", (long long)n, (long long)p);
  if (n > INT32_MAX) return fail(ctx, OEM_EINVAL, "n=%lld exceeds 2^31-1", (long long)n);
  if (p > 8192) return fail(ctx, OEM_EUNSUPPORTED, "p=%lld exceeds 8192", (long long)p);
  if (ldx < p) return fail(ctx, OEM_EINVAL, "ldx=%lld < p=%lld", (long long)ldx, (long long)p);
  if ((ldx * (int64_t)elem_size(xtype)) % 16 != 0)
    return fail(ctx, OEM_EINVAL, "ldx*sizeof(element) = %lld is not a multiple of 16",
                (long long)(ldx * (int64_t)elem_size(xtype)));
  if (!X || !y) return fail(ctx, OEM_EINVAL, "X or y is NULL");
  if (((uintptr_t)X & 15) || ((uintptr_t)y & 15))
    return fail(ctx, OEM_EINVAL, "X and y must be 16-byte aligned");
  return OEM_OK;
}

int resolve_mode(oem_ctx* ctx, int32_t mode, int32_t xtype, int32_t* out) {
  if (mode == OEM_GRAM_AUTO)
    mode = xtype == OEM_F64 ? OEM_GRAM_FP64 : xtype == OEM_BF16 ? OEM_GRAM_BF16 : OEM_GRAM_SPLIT_BF16;
  switch (mode) {
    case OEM_GRAM_FP64: break;
    case OEM_GRAM_FP32:
      if (xtype == OEM_F64) return fail(ctx, OEM_EINVAL, "OEM_GRAM_FP32 needs float32 or bfloat16 X");
      break;
    case OEM_GRAM_TF32:
    case OEM_GRAM_SPLIT_BF16:
      if (xtype != OEM_F32) return fail(ctx, OEM_EINVAL, "TF32 / SPLIT_BF16 modes need float32 X");
      break;
    case OEM_GRAM_BF16:
      if (xtype != OEM_BF16) return fail(ctx, OEM_EINVAL, "OEM_GRAM_BF16 needs bfloat16 X");
      break;
    default: return fail(ctx, OEM_EINVAL, "unknown gram mode %d", mode);
  }
  *out = mode;
  return OEM_OK;
}

bool tc_mode(int32_t mode) {
  return mode == OEM_GRAM_TF32 || mode == OEM_GRAM_BF16 || mode == OEM_GRAM_SPLIT_BF16;
}

// Everything the Gram pass needs in the workspace.
struct GramPlan {
  int32_t mode, q, ycols, T, nt, ntiles;
  int64_t chunk_rows, nblk;
  int max_chunks;
  int K;
  bool sorted;
};

GramPlan plan_gram(oem_ctx* ctx, int64_t n, int64_t p, int K, int32_t mode, bool sorted) {
  GramPlan g;
  g.mode = mode;
  // bfloat16 mode carries the float32 y as three bfloat16 pieces (exact)
  g.ycols = (mode == OEM_GRAM_BF16) ? 3 : 1;
  g.q = (int32_t)p + g.ycols;
  g.T = tc_mode(mode) ? 128 : 64;
  g.nt = (g.q + g.T - 1) / g.T;
  g.ntiles = g.nt * (g.nt + 1) / 2;
  g.K = K;
  g.sorted = sorted;
  const int64_t target_items = (int64_t)(tc_mode(mode) ? 4 : 4) * ctx->num_sms;
  int64_t chunks = std::max<int64_t>(K, (target_items + g.ntiles - 1) / g.ntiles);
  int64_t cr = (n + chunks - 1) / chunks;
  const int64_t align = tc_mode(mode) ? 128 : 16;
  cr = std::max<int64_t>(tc_mode(mode) ? 1024 : 256, (cr + align - 1) / align * align);
  g.chunk_rows = cr;
  g.max_chunks = (int)((n + cr - 1) / cr + K);
  g.nblk = (n + 1023) / 1024;
  return g;
}

struct GramBufs {
  int32_t *blk_counts = nullptr, *blk_offsets = nullptr, *perm = nullptr;
  ChunkTable ct{};
  double* partial = nullptr;
  double* Zg = nullptr;
};

void gram_request(Arena& A, const GramPlan& g, int64_t n, GramBufs& b) {
  if (g.sorted) {
    A.add(&b.blk_counts, (size_t)g.nblk * g.K);
    A.add(&b.blk_offsets, (size_t)g.nblk * g.K);
    A.add(&b.perm, (size_t)n);
  }
  A.add(&b.ct.row0, (size_t)g.max_chunks);
  A.add(&b.ct.row1, (size_t)g.max_chunks);
  A.add(&b.ct.fold, (size_t)g.max_chunks);
  A.add(&b.ct.count, 1);
  A.add(&b.ct.fold_c0, (size_t)g.K + 1);
  A.add(&b.ct.fold_off, (size_t)g.K + 1);
  A.add(&b.partial, (size_t)g.max_chunks * g.ntiles * g.T * g.T);
  A.add(&b.Zg, (size_t)g.K * g.q * g.q);
}

// fold sort (if any) -> chunk table -> Gram partials -> per-fold Z Grams.
int run_gram(oem_ctx* ctx, const GramPlan& g, GramBufs& b, const void* X, int32_t xtype,
             int64_t n, int64_t p, int64_t ldx, const void* y, const uint8_t* fold,
             bool require_nonempty, cudaStream_t s) {
  if (g.sorted) {
    LAUNCH(OEM_PROF_FOLD_SORT, launch_fold_count(fold, n, g.K, b.blk_counts, g.nblk, s));
    LAUNCH(OEM_PROF_FOLD_SORT, launch_fold_scan(b.blk_counts, g.nblk, g.K, g.chunk_rows, b.blk_offsets, b.ct,
                            g.max_chunks, ctx->dstatus, require_nonempty ? 1 : 0, s));
    LAUNCH(OEM_PROF_FOLD_SORT, launch_fold_scatter(fold, n, g.K, b.blk_offsets, b.perm, s));
  } else {
    LAUNCH(OEM_PROF_CHUNKS, launch_identity_chunks(n, g.chunk_rows, b.ct, g.max_chunks, s));
  }
  GramArgs a{};
  a.X = X; a.xtype = xtype; a.n = n; a.p = p; a.ldx = ldx; a.y = y;
  a.perm = g.sorted ? b.perm : nullptr;
  a.mode = g.mode; a.q = g.q; a.ycols = g.ycols; a.T = g.T; a.ntile1 = g.nt; a.ntiles = g.ntiles;
  a.ct = b.ct; a.max_chunks = g.max_chunks; a.partial = b.partial; a.dstatus = ctx->dstatus;
  if (tc_mode(g.mode)) {
    // Rows summed in float32 tensor memory before the compensated flush. The
    // tensor cores' float32 accumulation rounds toward zero, so the error
    // grows with the number of MMAs per window (measured at n = 2e6, p = 100,
    // split mode: 32 rows 3.2e-7, 64 rows 5.2e-7, 256 rows 1.6e-6 relative
    // Frobenius): split mode (4 products) uses 32-row windows, bfloat16 / tf32
    // 256 / 128. OEM_GRAM_FLUSH_ROWS overrides.
    int flush = g.mode == OEM_GRAM_SPLIT_BF16 ? 32 : g.mode == OEM_GRAM_TF32 ? 128 : 256;
    if (const char* ev = getenv("OEM_GRAM_FLUSH_ROWS")) {
      const int v = atoi(ev);
      if (v >= 32 && v <= 65536) flush = v;
    }
    LAUNCH(OEM_PROF_GRAM_TC, launch_gram_tc(a, flush, s));
  } else {
    LAUNCH(OEM_PROF_GRAM_SIMT, launch_gram_simt(a, s));
  }
  LAUNCH(OEM_PROF_GRAM_REDUCE, launch_gram_reduce(a, g.K, b.Zg, s));
  return OEM_OK;
}

// Penalties on the device.
struct PenPlan {
  int npen = 0;
  int p = 0;
  std::vector<DevPenalty> host;       // device pointers filled after commit
  std::vector<std::vector<double>> w64;
  std::vector<std::vector<float>> w32;
  std::vector<std::vector<int32_t>> grp;
  std::vector<std::vector<double>> cg;
  DevPenalty* dpens = nullptr;
  std::vector<double*> d_w64;
  std::vector<float*> d_w32;
  std::vector<int32_t*> d_grp;
  std::vector<double*> d_cg;
  std::vector<char> allowed;  // slice boundary allowed at row i (group starts)
};

int prepare_pens(oem_ctx* ctx, const oem_penalty* pens, int npen, int64_t p, PenPlan& P) {
  if (!pens || npen < 1 || npen > 8) return fail(ctx, OEM_EINVAL, "npen=%d must be in [1,8]", npen);
  P.npen = npen;
  P.p = (int)p;
  P.host.resize(npen);
  P.w64.resize(npen); P.w32.resize(npen); P.grp.resize(npen); P.cg.resize(npen);
  P.d_w64.assign(npen, nullptr); P.d_w32.assign(npen, nullptr);
  P.d_grp.assign(npen, nullptr); P.d_cg.assign(npen, nullptr);
  P.allowed.assign((size_t)p + 1, 1);
  for (int i = 0; i < npen; ++i) {
    const oem_penalty& q = pens[i];
    if (q.kind < OEM_LASSO || q.kind > OEM_GROUP_LASSO)
      return fail(ctx, OEM_EINVAL, "penalty %d: unknown kind %d", i, q.kind);
    if (q.kind == OEM_ENET && !(q.alpha >= 0.0 && q.alpha <= 1.0))
      return fail(ctx, OEM_EINVAL, "penalty %d: elastic net alpha=%g not in [0,1]", i, q.alpha);
    if (q.kind == OEM_MCP && !(q.gamma > 1.0))
      return fail(ctx, OEM_EINVAL, "penalty %d: MCP gamma=%g must exceed 1", i, q.gamma);
    if (q.kind == OEM_SCAD && !(q.gamma > 2.0))
      return fail(ctx, OEM_EINVAL, "penalty %d: SCAD gamma=%g must exceed 2", i, q.gamma);
    DevPenalty d{};
    d.kind = q.kind;
    d.alpha64 = q.kind == OEM_ENET ? q.alpha : 1.0;
    d.gamma64 = (q.kind == OEM_MCP || q.kind == OEM_SCAD) ? q.gamma : 3.0;
    d.alpha = (float)d.alpha64;
    d.gamma = (float)d.gamma64;
    if (q.w && q.kind != OEM_GROUP_LASSO) {
      P.w64[i].assign(q.w, q.w + p);
      P.w32[i].resize(p);
      for (int64_t j = 0; j < p; ++j) {
        if (!(q.w[j] >= 0.0) || !std::isfinite(q.w[j]))
          return fail(ctx, OEM_EINVAL, "penalty %d: weight %lld is %g", i, (long long)j, q.w[j]);
        P.w32[i][j] = (float)q.w[j];
      }
    }
    if (q.kind == OEM_GROUP_LASSO) {
      if (!q.group || q.ngroups < 1)
        return fail(ctx, OEM_EINVAL, "penalty %d: group lasso needs group ids and ngroups >= 1", i);
      P.grp[i].assign(q.group, q.group + p);
      std::vector<int> seen(q.ngroups, 0), cnt(q.ngroups, 0);
      for (int64_t j = 0; j < p; ++j) {
        const int g = q.group[j];
        if (g < 0 || g >= q.ngroups)
          return fail(ctx, OEM_EINVAL, "penalty %d: group id %d out of range", i, g);
        if (j > 0 && g != q.group[j - 1]) {
          if (seen[g])
            return fail(ctx, OEM_EUNSUPPORTED,
                        "penalty %d: the variables of group %d are not contiguous", i, g);
        }
        seen[g] = 1;
        ++cnt[g];
        if (j > 0 && g == q.group[j - 1]) P.allowed[j] = 0;
      }
      P.cg[i].resize(q.ngroups);
      for (int g = 0; g < q.ngroups; ++g) {
        const double v = q.cg ? q.cg[g] : std::sqrt((double)cnt[g]);
        if (!(v >= 0.0)) return fail(ctx, OEM_EINVAL, "penalty %d: group weight %d is %g", i, g, v);
        P.cg[i][g] = v;
      }
      d.ngroups = q.ngroups;
    }
    P.host[i] = d;
  }
  return OEM_OK;
}

void pens_request(Arena& A, PenPlan& P) {
  A.add(&P.dpens, (size_t)P.npen);
  for (int i = 0; i < P.npen; ++i) {
    if (!P.w64[i].empty()) { A.add(&P.d_w64[i], P.w64[i].size()); A.add(&P.d_w32[i], P.w32[i].size()); }
    if (!P.grp[i].empty()) { A.add(&P.d_grp[i], P.grp[i].size()); A.add(&P.d_cg[i], P.cg[i].size()); }
  }
}

int pens_upload(oem_ctx* ctx, PenPlan& P, cudaStream_t s) {
  for (int i = 0; i < P.npen; ++i) {
    DevPenalty& d = P.host[i];
    if (!P.w64[i].empty()) {
      CU(cudaMemcpyAsync(P.d_w64[i], P.w64[i].data(), P.w64[i].size() * 8, cudaMemcpyHostToDevice, s));
      CU(cudaMemcpyAsync(P.d_w32[i], P.w32[i].data(), P.w32[i].size() * 4, cudaMemcpyHostToDevice, s));
      d.w64 = P.d_w64[i];
      d.w32 = P.d_w32[i];
    }
    if (!P.grp[i].empty()) {
      CU(cudaMemcpyAsync(P.d_grp[i], P.grp[i].data(), P.grp[i].size() * 4, cudaMemcpyHostToDevice, s));
      CU(cudaMemcpyAsync(P.d_cg[i], P.cg[i].data(), P.cg[i].size() * 8, cudaMemcpyHostToDevice, s));
      d.grp = P.d_grp[i];
      d.cg = P.d_cg[i];
    }
  }
  CU(cudaMemcpyAsync(P.dpens, P.host.data(), sizeof(DevPenalty) * P.npen, cudaMemcpyHostToDevice, s));
  return OEM_OK;
}

int check_opts(oem_ctx* ctx, const oem_options* o) {
  if (!o) return fail(ctx, OEM_EINVAL, "options are NULL");
  if (o->nlambda < 1 || o->nlambda > 100000) return fail(ctx, OEM_EINVAL, "nlambda=%d", o->nlambda);
  if (!o->lambdas && !(o->lambda_min_ratio > 0.0 && o->lambda_min_ratio <= 1.0))
    return fail(ctx, OEM_EINVAL, "lambda_min_ratio=%g not in (0,1]", o->lambda_min_ratio);
  if (!(o->tol > 0.0)) return fail(ctx, OEM_EINVAL, "tol=%g must be > 0", o->tol);
  if (o->max_iter < 1) return fail(ctx, OEM_EINVAL, "max_iter=%lld must be >= 1", (long long)o->max_iter);
  if (o->iter_precision != OEM_ITER_F32 && o->iter_precision != OEM_ITER_F64)
    return fail(ctx, OEM_EINVAL, "iter_precision=%d", o->iter_precision);
  const int c = o->cluster_ctas;
  if (!(c == 0 || c == 1 || c == 2 || c == 4 || c == 8 || c == 16))
    return fail(ctx, OEM_EINVAL, "cluster_ctas=%d not in {0,1,2,4,8,16}", c);
  return OEM_OK;
}

// Iteration launch plan: cluster size, row slices aligned to group starts.
struct IterPlan {
  int C = 1, max_rows = 0, smem_rows = 0;
  size_t smem = 0;
  std::vector<int32_t> slice;
  int32_t* d_slice = nullptr;
};

int plan_iter(oem_ctx* ctx, int64_t p, int B, const PenPlan& P, const oem_options* o, IterPlan& I,
              IterArgs& probe) {
  const int prec = o->iter_precision;
  const size_t cap = 227 * 1024;
  int C;
  if (o->cluster_ctas > 0) {
    C = o->cluster_ctas;
  } else {
    int want = (int)std::min<int64_t>(16, std::max<int64_t>(1, (p + 31) / 32));
    int byB = std::max(1, ctx->num_sms / std::max(1, B));
    C = 1;
    while (C * 2 <= std::min(want, byB) && C < 16) C *= 2;
    // enough CTAs that the Gram rows fit in shared memory
    while (C < 16 && (size_t)((p + C - 1) / C) * oem_iter_smem_per_row((int)p, prec) +
                             oem_iter_smem_fixed((int)p, P.npen, (int)((p + C - 1) / C), C, prec) > cap)
      C *= 2;
  }
  for (;; C /= 2) {
    // slices: ideal boundaries moved forward to the next allowed row
    I.slice.assign(C + 1, 0);
    I.slice[C] = (int32_t)p;
    for (int r = 1; r < C; ++r) {
      int64_t bnd = std::max<int64_t>(I.slice[r - 1], (p * r) / C);
      while (bnd < p && !P.allowed[bnd]) ++bnd;
      I.slice[r] = (int32_t)bnd;
    }
    I.max_rows = 0;
    for (int r = 0; r < C; ++r) I.max_rows = std::max(I.max_rows, I.slice[r + 1] - I.slice[r]);
    I.max_rows = std::max(I.max_rows, 1);
    const size_t fixed = oem_iter_smem_fixed((int)p, P.npen, I.max_rows, C, prec);
    if (fixed + 1024 > cap) {
      if (C == 16) return fail(ctx, OEM_EUNSUPPORTED, "p=%lld too large for the iteration kernel", (long long)p);
      // a bigger cluster does not shrink the per-CTA fixed part much; give up
      return fail(ctx, OEM_EUNSUPPORTED, "p=%lld too large for the iteration kernel", (long long)p);
    }
    const size_t per = oem_iter_smem_per_row((int)p, prec);
    I.smem_rows = (int)std::min<size_t>((size_t)I.max_rows, (cap - fixed) / per);
    I.smem = fixed + (size_t)I.smem_rows * per;
    I.C = C;
    probe.C = C;
    probe.max_rows = I.max_rows;
    probe.smem_rows = I.smem_rows;
    if (oem_iter_max_cluster(probe, I.smem, C) >= 1) return OEM_OK;
    if (C == 1) return fail(ctx, OEM_ECUDA, "no cluster configuration of the iteration kernel fits");
  }
}

int run_iter(oem_ctx* ctx, int64_t p, int B, const float* G32, int ldg, const double* G64,
             const double* c, const double* d, const double* lam, PenPlan& P,
             const oem_options* o, IterPlan& I, double* beta, int32_t* iters, uint8_t* conv,
             cudaStream_t s) {
  CU(cudaMemcpyAsync(I.d_slice, I.slice.data(), sizeof(int32_t) * I.slice.size(),
                     cudaMemcpyHostToDevice, s));
  IterArgs a{};
  a.p = (int)p; a.B = B; a.npen = P.npen; a.nlambda = o->nlambda;
  a.G32 = G32; a.G64 = G64; a.ldg = ldg; a.c = c; a.d = d; a.lam = lam; a.pens = P.dpens;
  a.tol = o->tol; a.max_iter = o->max_iter; a.beta = beta; a.iters = iters; a.conv = conv;
  a.dstatus = ctx->dstatus; a.slice = I.d_slice; a.C = I.C; a.max_rows = I.max_rows;
  a.smem_rows = I.smem_rows; a.precision = o->iter_precision;
  LAUNCH(OEM_PROF_ITER, launch_oem_iter(a, I.smem, s));
  return OEM_OK;
}

}  // namespace

namespace oem {
cudaError_t launch_convert_g(const double* G64, int64_t p, int B, float* G32, int ldg32, cudaStream_t s);
}

extern "C" {

static void prof_collect(oem_ctx* ctx);

void oem_options_default(oem_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->nlambda = 100;
  o->lambda_min_ratio = 1e-3;
  o->lambdas = nullptr;
  o->tol = 1e-7;
  o->max_iter = 10000;
  o->lanczos_steps = 64;
  o->gram_mode = OEM_GRAM_AUTO;
  o->iter_precision = OEM_ITER_F32;
  o->cluster_ctas = 0;
}

int oem_create(oem_ctx** out, int device, size_t budget) {
  if (!out) return OEM_EINVAL;
  *out = nullptr;
  oem_ctx* ctx = new oem_ctx();
  ctx->device = device;
  ctx->budget = budget ? budget : ((size_t)8 << 30);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->dstatus, sizeof(unsigned) * 4);
  if (e == cudaSuccess) e = cudaMemset(ctx->dstatus, 0, sizeof(unsigned) * 4);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return OEM_ECUDA;
  }
  *out = ctx;
  return OEM_OK;
}

int oem_destroy(oem_ctx* ctx) {
  if (!ctx) return OEM_EINVAL;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  prof_collect(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->dstatus) cudaFree(ctx->dstatus);
  delete ctx;
  return OEM_OK;
}

const char* oem_last_error(const oem_ctx* ctx) { return ctx ? ctx->err : "null context"; }

int64_t oem_kernel_launches(const oem_ctx* ctx) { return ctx ? ctx->launches : 0; }

static void prof_collect(oem_ctx* ctx) {
  for (auto& pd : ctx->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(pd.e1) == cudaSuccess && cudaEventElapsedTime(&ms, pd.e0, pd.e1) == cudaSuccess) {
      ctx->prof_ms[pd.cls] += ms;
      ctx->prof_n[pd.cls] += pd.n;
    } else {
      cudaGetLastError();
    }
    ctx->ev_pool.push_back(pd.e0);
    ctx->ev_pool.push_back(pd.e1);
  }
  ctx->pending.clear();
}

int oem_profile_enable(oem_ctx* ctx, int enable) {
  if (!ctx) return OEM_EINVAL;
  prof_collect(ctx);
  ctx->prof = enable != 0;
  for (int k = 0; k < OEM_PROF_NKERNELS; ++k) { ctx->prof_ms[k] = 0.0; ctx->prof_n[k] = 0; }
  return OEM_OK;
}

int oem_profile_get(oem_ctx* ctx, int kernel, double* ms, int64_t* launches) {
  if (!ctx || kernel < 0 || kernel >= OEM_PROF_NKERNELS) return OEM_EINVAL;
  prof_collect(ctx);
  if (ms) *ms = ctx->prof_ms[kernel];
  if (launches) *launches = ctx->prof_n[kernel];
  return OEM_OK;
}

const char* oem_profile_name(int kernel) {
  static const char* names[OEM_PROF_NKERNELS] = {
      "fold_sort", "chunk_table", "gram_simt_kernel", "gram_tc_kernel", "gram_reduce_kernel",
      "assemble", "lanczos", "lambda_grid_kernel", "oem_iter_kernel", "cv_score", "copy_paths"};
  return (kernel >= 0 && kernel < OEM_PROF_NKERNELS) ? names[kernel] : "unknown";
}

int oem_sync(oem_ctx* ctx, void* stream) {
  if (!ctx) return OEM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaStreamSynchronize(s));
  unsigned st = 0;
  CU(cudaMemcpy(&st, ctx->dstatus, sizeof(unsigned), cudaMemcpyDeviceToHost));
  CU(cudaMemset(ctx->dstatus, 0, sizeof(unsigned)));
  if (st & kStatTimeout) return fail(ctx, OEM_ETIMEOUT, "a bounded device wait expired");
  if (st & kStatNonFinite) return fail(ctx, OEM_ENONFINITE, "X or y holds NaN or Inf");
  if (st & kStatEmptyFold) return fail(ctx, OEM_EINVAL, "a cross-validation fold has no rows");
  if (st & kStatNotConv) return OEM_WARN_NOTCONV;
  return OEM_OK;
}

int oem_gram(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
             const void* y, int32_t mode, double* G, double* c, double* yty, void* stream) {
  if (!ctx) return OEM_EINVAL;
  int r = check_x(ctx, X, xtype, n, p, ldx, y);
  if (r) return r;
  if (!G || !c || !yty) return fail(ctx, OEM_EINVAL, "output pointers must not be NULL");
  int32_t m;
  if ((r = resolve_mode(ctx, mode, xtype, &m))) return r;
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  GramPlan g = plan_gram(ctx, n, p, 1, m, false);
  GramBufs b;
  Arena A;
  gram_request(A, g, n, b);
  int64_t* nk = nullptr;
  A.add(&nk, 1);
  if ((r = arena_commit(ctx, A, s))) return r;
  if ((r = run_gram(ctx, g, b, X, xtype, n, p, ldx, y, nullptr, false, s))) return r;
  LAUNCH(OEM_PROF_ASSEMBLE, launch_extract_folds(b.Zg, 1, g.q, (int)p, g.ycols, G, c, yty, nk, b.ct.fold_off, s));
  return OEM_OK;
}

int oem_fold_grams(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
                   const void* y, const uint8_t* fold, int32_t K, int32_t mode, double* Gk,
                   double* ck, double* ytyk, int64_t* nk, void* stream) {
  if (!ctx) return OEM_EINVAL;
  int r = check_x(ctx, X, xtype, n, p, ldx, y);
  if (r) return r;
  if (K < 1 || K > 64) return fail(ctx, OEM_EINVAL, "K=%d not in [1,64]", K);
  if (!fold || !Gk || !ck || !ytyk || !nk) return fail(ctx, OEM_EINVAL, "NULL pointer argument");
  int32_t m;
  if ((r = resolve_mode(ctx, mode, xtype, &m))) return r;
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  GramPlan g = plan_gram(ctx, n, p, K, m, true);
  GramBufs b;
  Arena A;
  gram_request(A, g, n, b);
  if ((r = arena_commit(ctx, A, s))) return r;
  if ((r = run_gram(ctx, g, b, X, xtype, n, p, ldx, y, fold, false, s))) return r;
  LAUNCH(OEM_PROF_ASSEMBLE, launch_extract_folds(b.Zg, K, g.q, (int)p, g.ycols, Gk, ck, ytyk, nk, b.ct.fold_off, s));
  return OEM_OK;
}

int oem_spectral_d(oem_ctx* ctx, const double* G, int64_t p, int64_t ldg, int32_t batch,
                   int64_t strideG, int32_t steps, double* d, void* stream) {
  if (!ctx) return OEM_EINVAL;
  if (!G || !d) return fail(ctx, OEM_EINVAL, "NULL pointer argument");
  if (p < 1 || ldg < p || batch < 1 || (batch > 1 && strideG < p * ldg))
    return fail(ctx, OEM_EINVAL, "bad sizes p=%lld ldg=%lld batch=%d strideG=%lld", (long long)p,
                (long long)ldg, batch, (long long)strideG);
  if (steps > 128) return fail(ctx, OEM_EINVAL, "steps=%d exceeds 128", steps);
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  LanczosWork w{};
  Arena A;
  A.add(&w.V, (size_t)batch * 3 * p);
  A.add(&w.alpha, (size_t)batch * 128);
  A.add(&w.beta, (size_t)batch * 128);
  A.add(&w.fro, (size_t)batch);
  A.add(&w.mlen, (size_t)batch);
  int r;
  if ((r = arena_commit(ctx, A, s))) return r;
  cudaError_t e = lanczos_prof(ctx, s, G, p, ldg, batch, strideG, steps, w, d, s, &ctx->launches);
  if (e != cudaSuccess) return fail(ctx, OEM_ECUDA, "Lanczos launch failed: %s", cudaGetErrorString(e));
  return OEM_OK;
}

// Shared tail of oem_fit_path / oem_fit / oem_cv: lambda grid + iteration.
static int fit_tail(oem_ctx* ctx, int64_t p, int B, const double* G64, const float* G32, int ldg32,
                    const double* c, const double* d, PenPlan& P, IterPlan& I,
                    const oem_options* o, double* lam, double* beta, int32_t* iters,
                    uint8_t* conv, cudaStream_t s) {
  int r;
  if ((r = pens_upload(ctx, P, s))) return r;
  if (o->lambdas) {
    CU(cudaMemcpyAsync(lam, o->lambdas, sizeof(double) * P.npen * o->nlambda, cudaMemcpyHostToDevice, s));
  } else {
    LAUNCH(OEM_PROF_LAMBDA, launch_lambda_grid(c, (int)p, P.dpens, P.npen, o->nlambda, o->lambda_min_ratio, lam, s));
  }
  return run_iter(ctx, p, B, G32, ldg32, G64, c, d, lam, P, o, I, beta, iters, conv, s);
}

static int check_user_lambdas(oem_ctx* ctx, const oem_options* o, int npen) {
  if (!o->lambdas) return OEM_OK;
  for (int i = 0; i < npen; ++i)
    for (int l = 0; l < o->nlambda; ++l) {
      const double v = o->lambdas[(size_t)i * o->nlambda + l];
      if (!(v >= 0.0) || !std::isfinite(v))
        return fail(ctx, OEM_EINVAL, "lambda[%d][%d] = %g", i, l, v);
    }
  return OEM_OK;
}

int oem_fit_path(oem_ctx* ctx, const double* G, const double* c, int64_t p, double d,
                 const oem_penalty* pens, int32_t npen, const oem_options* opt, double* beta,
                 double* lambdas_out, int32_t* iters, uint8_t* converged, void* stream) {
  if (!ctx) return OEM_EINVAL;
  int r;
  if ((r = check_opts(ctx, opt))) return r;
  if (!G || !c || !beta || !lambdas_out || !iters || !converged)
    return fail(ctx, OEM_EINVAL, "NULL pointer argument");
  if (p < 1 || p > 8192) return fail(ctx, OEM_EINVAL, "p=%lld not in [1,8192]", (long long)p);
  if (!(d <= 0.0 || std::isfinite(d))) return fail(ctx, OEM_EINVAL, "d=%g", d);
  PenPlan P;
  if ((r = prepare_pens(ctx, pens, npen, p, P))) return r;
  if ((r = check_user_lambdas(ctx, opt, npen))) return r;
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  const int ldg32 = (int)((p + 3) & ~3LL);
  IterArgs probe{};
  probe.p = (int)p; probe.B = 1; probe.npen = npen; probe.precision = opt->iter_precision;
  IterPlan I;
  if ((r = plan_iter(ctx, p, 1, P, opt, I, probe))) return r;
  float* G32 = nullptr;
  double* dd = nullptr;
  LanczosWork w{};
  Arena A;
  if (opt->iter_precision == OEM_ITER_F32) A.add(&G32, (size_t)p * ldg32);
  A.add(&dd, 1);
  A.add(&w.V, (size_t)3 * p);
  A.add(&w.alpha, 128);
  A.add(&w.beta, 128);
  A.add(&w.fro, 1);
  A.add(&w.mlen, 1);
  pens_request(A, P);
  A.add(&I.d_slice, I.slice.size());
  if ((r = arena_commit(ctx, A, s))) return r;
  if (G32) LAUNCH(OEM_PROF_ASSEMBLE, launch_convert_g(G, p, 1, G32, ldg32, s));
  if (d > 0.0) {
    CU(cudaMemcpyAsync(dd, &d, sizeof(double), cudaMemcpyHostToDevice, s));
  } else {
    cudaError_t e = lanczos_prof(ctx, s, G, p, p, 1, p * p, opt->lanczos_steps, w, dd, s, &ctx->launches);
    if (e != cudaSuccess) return fail(ctx, OEM_ECUDA, "Lanczos launch failed: %s", cudaGetErrorString(e));
  }
  return fit_tail(ctx, p, 1, G, G32, ldg32, c, dd, P, I, opt, lambdas_out, beta, iters, converged, s);
}

int oem_fit(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
            const void* y, const oem_penalty* pens, int32_t npen, const oem_options* opt,
            double* beta, double* lambdas_out, int32_t* iters, uint8_t* converged, double* d_out,
            void* stream) {
  if (!ctx) return OEM_EINVAL;
  int r = check_x(ctx, X, xtype, n, p, ldx, y);
  if (r) return r;
  if ((r = check_opts(ctx, opt))) return r;
  if (!beta || !lambdas_out || !iters || !converged) return fail(ctx, OEM_EINVAL, "NULL pointer argument");
  int32_t m;
  if ((r = resolve_mode(ctx, opt->gram_mode, xtype, &m))) return r;
  PenPlan P;
  if ((r = prepare_pens(ctx, pens, npen, p, P))) return r;
  if ((r = check_user_lambdas(ctx, opt, npen))) return r;
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  const int ldg32 = (int)((p + 3) & ~3LL);
  IterArgs probe{};
  probe.p = (int)p; probe.B = 1; probe.npen = npen; probe.precision = opt->iter_precision;
  IterPlan I;
  if ((r = plan_iter(ctx, p, 1, P, opt, I, probe))) return r;
  GramPlan g = plan_gram(ctx, n, p, 1, m, false);
  GramBufs b;
  double *G64 = nullptr, *c = nullptr, *N = nullptr, *cnt = nullptr, *dd = nullptr;
  float* G32 = nullptr;
  LanczosWork w{};
  Arena A;
  gram_request(A, g, n, b);
  A.add(&G64, (size_t)p * p);
  if (opt->iter_precision == OEM_ITER_F32) A.add(&G32, (size_t)p * ldg32);
  A.add(&c, (size_t)p);
  A.add(&N, 1);
  A.add(&cnt, 1);
  A.add(&dd, 1);
  A.add(&w.V, (size_t)3 * p);
  A.add(&w.alpha, 128);
  A.add(&w.beta, 128);
  A.add(&w.fro, 1);
  A.add(&w.mlen, 1);
  pens_request(A, P);
  A.add(&I.d_slice, I.slice.size());
  if ((r = arena_commit(ctx, A, s))) return r;
  if ((r = run_gram(ctx, g, b, X, xtype, n, p, ldx, y, nullptr, false, s))) return r;
  LAUNCH(OEM_PROF_ASSEMBLE, launch_assemble(b.Zg, 1, g.q, (int)p, g.ycols, b.ct.fold_off, 0, G64, G32, ldg32, c, N,
                         cnt, s));
  cudaError_t e = lanczos_prof(ctx, s, G64, p, p, 1, p * p, opt->lanczos_steps, w, dd, s, &ctx->launches);
  if (e != cudaSuccess) return fail(ctx, OEM_ECUDA, "Lanczos launch failed: %s", cudaGetErrorString(e));
  if (d_out) CU(cudaMemcpyAsync(d_out, dd, sizeof(double), cudaMemcpyDeviceToDevice, s));
  return fit_tail(ctx, p, 1, G64, G32, ldg32, c, dd, P, I, opt, lambdas_out, beta, iters, converged, s);
}

int oem_cv(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
           const void* y, const uint8_t* fold, int32_t K, const oem_penalty* pens, int32_t npen,
           const oem_options* opt, double* beta_full, double* lambdas_out, double* cvm,
           double* cvsd, int32_t* idx_min, int32_t* idx_1se, int32_t* best_penalty, void* stream) {
  if (!ctx) return OEM_EINVAL;
  int r = check_x(ctx, X, xtype, n, p, ldx, y);
  if (r) return r;
  if ((r = check_opts(ctx, opt))) return r;
  if (K < 2 || K > 64) return fail(ctx, OEM_EINVAL, "K=%d not in [2,64]", K);
  if (!fold || !beta_full || !lambdas_out || !cvm || !cvsd || !idx_min || !idx_1se || !best_penalty)
    return fail(ctx, OEM_EINVAL, "NULL pointer argument");
  int32_t m;
  if ((r = resolve_mode(ctx, opt->gram_mode, xtype, &m))) return r;
  PenPlan P;
  if ((r = prepare_pens(ctx, pens, npen, p, P))) return r;
  if ((r = check_user_lambdas(ctx, opt, npen))) return r;
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  const int B = K + 1;
  const int ldg32 = (int)((p + 3) & ~3LL);
  const int L = opt->nlambda;
  IterArgs probe{};
  probe.p = (int)p; probe.B = B; probe.npen = npen; probe.precision = opt->iter_precision;
  IterPlan I;
  if ((r = plan_iter(ctx, p, B, P, opt, I, probe))) return r;
  GramPlan g = plan_gram(ctx, n, p, K, m, true);
  GramBufs b;
  double *G64 = nullptr, *c = nullptr, *N = nullptr, *cnt = nullptr, *dd = nullptr;
  double *beta_all = nullptr, *mse = nullptr;
  int32_t* it_all = nullptr;
  uint8_t* cv_all = nullptr;
  float* G32 = nullptr;
  LanczosWork w{};
  Arena A;
  gram_request(A, g, n, b);
  A.add(&G64, (size_t)B * p * p);
  if (opt->iter_precision == OEM_ITER_F32) A.add(&G32, (size_t)B * p * ldg32);
  A.add(&c, (size_t)B * p);
  A.add(&N, (size_t)B);
  A.add(&cnt, (size_t)B);
  A.add(&dd, (size_t)B);
  A.add(&w.V, (size_t)B * 3 * p);
  A.add(&w.alpha, (size_t)B * 128);
  A.add(&w.beta, (size_t)B * 128);
  A.add(&w.fro, (size_t)B);
  A.add(&w.mlen, (size_t)B);
  A.add(&beta_all, (size_t)B * npen * L * p);
  A.add(&it_all, (size_t)B * npen * L);
  A.add(&cv_all, (size_t)B * npen * L);
  A.add(&mse, (size_t)npen * K * L);
  pens_request(A, P);
  A.add(&I.d_slice, I.slice.size());
  if ((r = arena_commit(ctx, A, s))) return r;
  if ((r = run_gram(ctx, g, b, X, xtype, n, p, ldx, y, fold, true, s))) return r;
  LAUNCH(OEM_PROF_ASSEMBLE, launch_assemble(b.Zg, K, g.q, (int)p, g.ycols, b.ct.fold_off, 1, G64, G32, ldg32, c, N,
                         cnt, s));
  cudaError_t e = lanczos_prof(ctx, s, G64, p, p, B, p * p, opt->lanczos_steps, w, dd, s, &ctx->launches);
  if (e != cudaSuccess) return fail(ctx, OEM_ECUDA, "Lanczos launch failed: %s", cudaGetErrorString(e));
  if ((r = fit_tail(ctx, p, B, G64, G32, ldg32, c, dd, P, I, opt, lambdas_out, beta_all, it_all,
                    cv_all, s)))
    return r;
  LAUNCH(OEM_PROF_CV, launch_cv_score(b.Zg, K, g.q, (int)p, g.ycols, b.ct.fold_off, beta_all, npen, L, mse, cvm,
                         cvsd, idx_min, idx_1se, best_penalty, s));
  LAUNCH(OEM_PROF_COPY, launch_copy_paths(beta_all, it_all, cv_all, npen, L, (int)p, beta_full, nullptr, nullptr,
                           ctx->dstatus, s));
  return OEM_OK;
}

}  // extern "C"
