// C-ABI entry points (include/oem.h): argument validation, the per-context
// workspace arena, and the order of kernels for each call.
#include "host.cuh"

using namespace oem::host;


namespace oem {

constexpr int kUpChunk = 3840;  // bytes per upload kernel (parameters stay under 4 KB)
struct UpChunk {
  unsigned char b[kUpChunk];
};
__global__ void upload_kernel(unsigned char* dst, UpChunk c, int nbytes) {
  for (int i = threadIdx.x; i < nbytes; i += blockDim.x) dst[i] = c.b[i];
}
cudaError_t launch_upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  for (size_t o = 0; o < bytes; o += kUpChunk) {
    UpChunk c;
    const int nb = (int)std::min<size_t>(kUpChunk, bytes - o);
    memcpy(c.b, (const unsigned char*)src + o, (size_t)nb);
    upload_kernel<<<1, 256, 0, s>>>((unsigned char*)dst + o, c, nb);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
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
  o->instances_per_task = 0;
  o->autotune = 1;
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
  // load the upload kernel now: its first use may be inside a stream capture
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, oem::upload_kernel);
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
      "fold_sort", "chunk_table", "gram_simt_kernel", "gram_tc_pass", "gram_reduce_kernel",
      "assemble", "lanczos", "lambda_grid_kernel", "oem_iter_kernel", "cv_score", "copy_paths",
      "logistic_outer_step"};
  return (kernel >= 0 && kernel < OEM_PROF_NKERNELS) ? names[kernel] : "unknown";
}

int oem_iter_stats(oem_ctx* ctx, void* stream, int64_t* iterations, int64_t* loop_trips) {
  if (!ctx) return OEM_EINVAL;
  if (!ctx->last_iters) return fail(ctx, OEM_EINVAL, "no path has been fitted on this context");
  CU(cudaSetDevice(ctx->device));
  CU(cudaStreamSynchronize((cudaStream_t)stream));
  const size_t inst = (size_t)ctx->last_B * ctx->last_npen, L = (size_t)ctx->last_L;
  std::vector<int32_t> h(inst * L);
  CU(cudaMemcpy(h.data(), ctx->last_iters, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost));
  int64_t tot = 0, trips = 0;
  for (size_t i = 0; i < inst; ++i) {
    int64_t s = 0;
    for (size_t l = 0; l < L; ++l) s += h[i * L + l];
    tot += s;
    trips = std::max(trips, s);
  }
  if (iterations) *iterations = tot;
  if (loop_trips) *loop_trips = trips;
  return OEM_OK;
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

// Where X, y and fold live: X in host memory streams through the Gram pass
// (y and fold may then live on either side); with X on the device, y and fold
// must be on the device too.
static int plan_residence(oem_ctx* ctx, const void* X, const void* y, const uint8_t* fold, int64_t n,
                          int64_t ldx, int32_t xtype, StreamBufs& sb, int64_t* rows, cudaStream_t s) {
  sb.on = host_resident(X);
  if (sb.on && capturing(s))
    return fail(ctx, OEM_EINVAL, "X in host memory cannot be streamed inside a stream capture");
  if (!sb.on) {
    if (host_resident(y) || (fold && host_resident(fold)))
      return fail(ctx, OEM_EINVAL, "y and fold must be in device memory when X is");
    *rows = n;
    return OEM_OK;
  }
  sb.y_host = host_resident(y);
  sb.fold_host = fold && host_resident(fold);
  sb.rows = stream_block_rows(n, ldx, xtype);
  *rows = sb.rows;
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
  StreamBufs sb;
  int64_t rows;
  if ((r = plan_residence(ctx, X, y, nullptr, n, ldx, xtype, sb, &rows, s))) return r;
  GramPlan g = plan_gram(ctx, rows, p, 1, m, false, 0, direct_x_ok(X, xtype, sb));
  GramBufs b;
  Arena A;
  gram_request(A, g, rows, b);
  if (sb.on) stream_request(A, sb, rows, ldx, xtype, 1, g.q, false);
  int64_t* nk = nullptr;
  A.add(&nk, 1);
  if ((r = arena_commit(ctx, A, s))) return r;
  const double* Zg;
  const int64_t* foff;
  if ((r = run_gram_any(ctx, g, b, sb, X, xtype, n, p, ldx, y, nullptr, false, s, &Zg, &foff))) return r;
  LAUNCH(OEM_PROF_ASSEMBLE, launch_extract_folds(Zg, 1, g.q, (int)p, g.ycols, G, c, yty, nk, foff, s));
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
  StreamBufs sb;
  int64_t rows;
  if ((r = plan_residence(ctx, X, y, fold, n, ldx, xtype, sb, &rows, s))) return r;
  GramPlan g = plan_gram(ctx, rows, p, K, m, true);
  GramBufs b;
  Arena A;
  gram_request(A, g, rows, b);
  if (sb.on) stream_request(A, sb, rows, ldx, xtype, K, g.q, true);
  if ((r = arena_commit(ctx, A, s))) return r;
  const double* Zg;
  const int64_t* foff;
  if ((r = run_gram_any(ctx, g, b, sb, X, xtype, n, p, ldx, y, fold, false, s, &Zg, &foff))) return r;
  LAUNCH(OEM_PROF_ASSEMBLE, launch_extract_folds(Zg, K, g.q, (int)p, g.ycols, Gk, ck, ytyk, nk, foff, s));
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
  lanczos_request(A, w, p, batch, steps);
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
    CU(upload(lam, o->lambdas, sizeof(double) * P.npen * o->nlambda, s));
  } else {
    LAUNCH(OEM_PROF_LAMBDA, launch_lambda_grid(c, (int)p, P.dpens, P.npen, o->nlambda, o->lambda_min_ratio, lam, s));
  }
  ctx->last_iters = iters;
  ctx->last_B = B;
  ctx->last_npen = P.npen;
  ctx->last_L = o->nlambda;
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
  IterPlan I;
  if ((r = plan_iter(ctx, p, 1, P, opt, I))) return r;
  float* G32 = nullptr;
  double* dd = nullptr;
  LanczosWork w{};
  Arena A;
  if (opt->iter_precision == OEM_ITER_F32) A.add(&G32, (size_t)p * ldg32);
  A.add(&dd, 1);
  lanczos_request(A, w, p, 1, opt->lanczos_steps);
  pens_request(A, P);
  iter_request(A, p, 1, I);
  if ((r = arena_commit(ctx, A, s))) return r;
  if (G32) LAUNCH(OEM_PROF_ASSEMBLE, launch_convert_g(G, p, 1, G32, ldg32, s));
  if (d > 0.0) {
    CU(upload(dd, &d, sizeof(double), s));
  } else {
    cudaError_t e = lanczos_prof(ctx, s, G, p, p, 1, p * p, opt->lanczos_steps, w, dd, s, &ctx->launches);
    if (e != cudaSuccess) return fail(ctx, OEM_ECUDA, "Lanczos launch failed: %s", cudaGetErrorString(e));
  }
  return fit_tail(ctx, p, 1, G, G32, ldg32, c, dd, P, I, opt, lambdas_out, beta, iters, converged, s);
}

int oem_fit(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
            const void* y, const oem_penalty* pens, int32_t npen, const oem_options* opt,
            double* beta, double* lambdas_out, int32_t* iters, uint8_t* converged, double* d_out,
            double* beta0, void* stream) {
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
  IterPlan I;
  if ((r = plan_iter(ctx, p, 1, P, opt, I))) return r;
  const bool centre = opt->intercept || opt->standardize;
  StreamBufs sb;
  int64_t rows;
  if ((r = plan_residence(ctx, X, y, nullptr, n, ldx, xtype, sb, &rows, s))) return r;
  GramPlan g = plan_gram(ctx, rows, p, 1, m, false, opt->intercept ? kOnesShifted : 0,
                         direct_x_ok(X, xtype, sb));
  GramBufs b;
  double *G64 = nullptr, *c = nullptr, *N = nullptr, *cnt = nullptr, *dd = nullptr, *cen = nullptr;
  float* G32 = nullptr;
  LanczosWork w{};
  Arena A;
  gram_request(A, g, rows, b);
  if (sb.on) stream_request(A, sb, rows, ldx, xtype, 1, g.q, false);
  if (centre) A.add(&cen, (size_t)(2 * p + 1));
  A.add(&G64, (size_t)p * p);
  if (opt->iter_precision == OEM_ITER_F32) A.add(&G32, (size_t)p * ldg32);
  A.add(&c, (size_t)p);
  A.add(&N, 1);
  A.add(&cnt, 1);
  A.add(&dd, 1);
  lanczos_request(A, w, p, 1, opt->lanczos_steps);
  pens_request(A, P);
  iter_request(A, p, 1, I);
  if ((r = arena_commit(ctx, A, s))) return r;
  const double* Zg;
  const int64_t* foff;
  if ((r = run_gram_any(ctx, g, b, sb, X, xtype, n, p, ldx, y, nullptr, false, s, &Zg, &foff))) return r;
  CentreArgs ce;
  if (centre) {
    ce.ocol = opt->intercept ? (int32_t)p + g.ycols : -1;
    ce.intercept = opt->intercept;
    ce.standardize = opt->standardize;
    ce.cen = cen;
  }
  LAUNCH(OEM_PROF_ASSEMBLE, launch_assemble(Zg, 1, g.q, (int)p, g.ycols, foff, 0, G64, G32, ldg32, c, N,
                         cnt, s, ce));
  cudaError_t e = lanczos_prof(ctx, s, G64, p, p, 1, p * p, opt->lanczos_steps, w, dd, s, &ctx->launches);
  if (e != cudaSuccess) return fail(ctx, OEM_ECUDA, "Lanczos launch failed: %s", cudaGetErrorString(e));
  if (d_out) CU(cudaMemcpyAsync(d_out, dd, sizeof(double), cudaMemcpyDeviceToDevice, s));
  if ((r = fit_tail(ctx, p, 1, G64, G32, ldg32, c, dd, P, I, opt, lambdas_out, beta, iters, converged, s)))
    return r;
  if (centre) {
    LAUNCH(OEM_PROF_COPY, launch_unstandardize(beta, 1, P.npen, opt->nlambda, (int)p, cen, b.shift,
                                               opt->intercept, nullptr, beta0, s));
  } else if (beta0) {
    CU(cudaMemsetAsync(beta0, 0, sizeof(double) * P.npen * opt->nlambda, s));
  }
  return OEM_OK;
}

int oem_cv(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
           const void* y, const uint8_t* fold, int32_t K, const oem_penalty* pens, int32_t npen,
           const oem_options* opt, double* beta_full, double* lambdas_out, double* cvm,
           double* cvsd, int32_t* idx_min, int32_t* idx_1se, int32_t* best_penalty, double* beta0_full,
           void* stream) {
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
  IterPlan I;
  if ((r = plan_iter(ctx, p, B, P, opt, I))) return r;
  const bool centre = opt->intercept || opt->standardize;
  StreamBufs sb;
  int64_t rows;
  if ((r = plan_residence(ctx, X, y, fold, n, ldx, xtype, sb, &rows, s))) return r;
  GramPlan g = plan_gram(ctx, rows, p, K, m, true, opt->intercept ? kOnesShifted : 0);
  GramBufs b;
  double *G64 = nullptr, *c = nullptr, *N = nullptr, *cnt = nullptr, *dd = nullptr;
  double *beta_all = nullptr, *mse = nullptr, *cen = nullptr, *bprime = nullptr;
  int32_t* it_all = nullptr;
  uint8_t* cv_all = nullptr;
  float* G32 = nullptr;
  LanczosWork w{};
  Arena A;
  gram_request(A, g, rows, b);
  if (sb.on) stream_request(A, sb, rows, ldx, xtype, K, g.q, true);
  A.add(&G64, (size_t)B * p * p);
  if (opt->iter_precision == OEM_ITER_F32) A.add(&G32, (size_t)B * p * ldg32);
  A.add(&c, (size_t)B * p);
  A.add(&N, (size_t)B);
  A.add(&cnt, (size_t)B);
  A.add(&dd, (size_t)B);
  lanczos_request(A, w, p, B, opt->lanczos_steps);
  A.add(&beta_all, (size_t)B * npen * L * p);
  A.add(&it_all, (size_t)B * npen * L);
  A.add(&cv_all, (size_t)B * npen * L);
  A.add(&mse, (size_t)npen * K * L);
  if (centre) {
    A.add(&cen, (size_t)B * (2 * p + 1));
    A.add(&bprime, (size_t)B * npen * L);
  }
  pens_request(A, P);
  iter_request(A, p, B, I);
  if ((r = arena_commit(ctx, A, s))) return r;
  const double* Zg;
  const int64_t* foff;
  if ((r = run_gram_any(ctx, g, b, sb, X, xtype, n, p, ldx, y, fold, true, s, &Zg, &foff))) return r;
  CentreArgs ce;
  if (centre) {
    ce.ocol = opt->intercept ? (int32_t)p + g.ycols : -1;
    ce.intercept = opt->intercept;
    ce.standardize = opt->standardize;
    ce.cen = cen;
  }
  LAUNCH(OEM_PROF_ASSEMBLE, launch_assemble(Zg, K, g.q, (int)p, g.ycols, foff, 1, G64, G32, ldg32, c, N,
                         cnt, s, ce));
  cudaError_t e = lanczos_prof(ctx, s, G64, p, p, B, p * p, opt->lanczos_steps, w, dd, s, &ctx->launches);
  if (e != cudaSuccess) return fail(ctx, OEM_ECUDA, "Lanczos launch failed: %s", cudaGetErrorString(e));
  if ((r = fit_tail(ctx, p, B, G64, G32, ldg32, c, dd, P, I, opt, lambdas_out, beta_all, it_all,
                    cv_all, s)))
    return r;
  if (centre)
    LAUNCH(OEM_PROF_COPY, launch_unstandardize(beta_all, B, npen, L, (int)p, cen, b.shift, opt->intercept,
                                               bprime, beta0_full, s));
  else if (beta0_full)
    CU(cudaMemsetAsync(beta0_full, 0, sizeof(double) * npen * L, s));
  LAUNCH(OEM_PROF_CV, launch_cv_score(Zg, K, g.q, (int)p, g.ycols, foff, beta_all, npen, L, mse, cvm,
                         cvsd, idx_min, idx_1se, best_penalty, s, ce.ocol, bprime));
  LAUNCH(OEM_PROF_COPY, launch_copy_paths(beta_all, it_all, cv_all, npen, L, (int)p, beta_full, nullptr, nullptr,
                           ctx->dstatus, s));
  return OEM_OK;
}

int oem_fit_logistic(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
                     const void* y, const oem_penalty* pens, int32_t npen, const oem_options* opt,
                     double* beta, double* beta0, double* lambdas_out, int32_t* iters,
                     uint8_t* converged, double* d_out, void* stream) {
  if (!ctx) return OEM_EINVAL;
  int r = check_x(ctx, X, xtype, n, p, ldx, y);
  if (r) return r;
  if ((r = check_opts(ctx, opt))) return r;
  if (!beta || !lambdas_out || !iters || !converged) return fail(ctx, OEM_EINVAL, "NULL pointer argument");
  if (p > 1023) return fail(ctx, OEM_EINVAL, "logistic regression: p=%lld exceeds 1023", (long long)p);
  if (host_resident(X) || host_resident(y))
    return fail(ctx, OEM_EUNSUPPORTED, "logistic regression: X and y must be in device memory");
  if (opt->standardize) return fail(ctx, OEM_EUNSUPPORTED, "logistic regression: standardize is not supported");
  if (!pens || npen < 1 || npen > 8) return fail(ctx, OEM_EINVAL, "npen=%d must be in [1,8]", npen);
  for (int i = 0; i < npen; ++i)
    if (pens[i].kind > OEM_SCAD)
      return fail(ctx, OEM_EUNSUPPORTED, "logistic regression: penalty %d is a group penalty", i);
  int32_t m;
  if ((r = resolve_mode(ctx, opt->gram_mode, xtype, &m))) return r;
  if ((r = check_user_lambdas(ctx, opt, npen))) return r;
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  const int icpt = opt->intercept ? 1 : 0;
  const int64_t pq = p + icpt;  // coefficients incl. the unpenalised intercept (last)
  const int L = opt->nlambda;
  // penalties on [X | 1]: the user's weights (or 1), weight 0 on the intercept
  std::vector<std::vector<double>> wext(npen);
  std::vector<oem_penalty> ext(pens, pens + npen);
  for (int i = 0; i < npen; ++i) {
    wext[i].assign((size_t)pq, 1.0);
    if (pens[i].w) std::copy(pens[i].w, pens[i].w + p, wext[i].begin());
    if (icpt) wext[i][p] = 0.0;
    ext[i].w = wext[i].data();
  }
  PenPlan P;
  if ((r = prepare_pens(ctx, ext.data(), npen, pq, P))) return r;
  oem_options inner = *opt;  // one lambda per inner launch, fixed layout
  inner.nlambda = 1;
  inner.lambdas = nullptr;
  inner.autotune = 0;
  const int ldg32 = (int)((pq + 3) & ~3LL);
  IterPlan I;
  if ((r = plan_iter(ctx, pq, 1, P, &inner, I))) return r;
  GramPlan g = plan_gram(ctx, n, p, 1, m, false, kOnes);
  GramBufs b;
  int sms = ctx->num_sms;
  // score pass: one CTA per SM, two row chunks of ~80 KB each in shared memory
  const int grid = sms;
  const int64_t lds = (p + 3) & ~3LL;
  int rc = (int)std::min<int64_t>(64, std::max<int64_t>(8, (81920 / (4 * lds)) / 8 * 8));
  double *G64 = nullptr, *dd = nullptr, *lam = nullptr, *lam_l = nullptr, *bcur = nullptr, *gv = nullptr;
  double *bnew = nullptr, *st_u = nullptr, *st_beta = nullptr;
  int32_t *it_new = nullptr, *its_l = nullptr, *flags = nullptr, *st_ctl = nullptr;
  uint8_t *conv_l = nullptr, *conv_in = nullptr;
  float* G32 = nullptr;
  float2* part = nullptr;
  LanczosWork w{};
  Arena A;
  gram_request(A, g, n, b);
  A.add(&G64, (size_t)pq * pq);
  if (opt->iter_precision == OEM_ITER_F32) A.add(&G32, (size_t)pq * ldg32);
  A.add(&dd, 1);
  lanczos_request(A, w, pq, 1, opt->lanczos_steps);
  A.add(&lam, (size_t)npen * L);
  A.add(&lam_l, (size_t)npen);
  A.add(&bcur, (size_t)npen * pq);
  A.add(&gv, (size_t)npen * pq);
  A.add(&bnew, (size_t)npen * pq);
  A.add(&st_u, (size_t)npen * pq * 2);
  A.add(&st_beta, (size_t)npen * pq);
  A.add(&st_ctl, (size_t)40 * npen);
  A.add(&it_new, (size_t)npen);
  A.add(&its_l, (size_t)npen);
  A.add(&flags, (size_t)npen);
  A.add(&conv_l, (size_t)npen);
  A.add(&conv_in, (size_t)npen);
  A.add(&part, (size_t)grid * npen * pq);
  pens_request(A, P);
  iter_request(A, pq, 1, I);
  if ((r = arena_commit(ctx, A, s))) return r;
  if ((r = pens_upload(ctx, P, s))) return r;
  // ---- the Gram pass (one pass over [X | y | 1]) and G = Z^T Z / (4n)
  if ((r = run_gram(ctx, g, b, X, xtype, n, p, ldx, y, nullptr, false, s))) return r;
  const int ocol = (int)p + g.ycols;
  LAUNCH(OEM_PROF_ASSEMBLE, launch_logit_gram(b.Zg, g.q, (int)p, ocol, icpt, n, G64, G32, ldg32, s));
  cudaError_t e = lanczos_prof(ctx, s, G64, pq, pq, 1, pq * pq, opt->lanczos_steps, w, dd, s, &ctx->launches);
  if (e != cudaSuccess) return fail(ctx, OEM_ECUDA, "Lanczos launch failed: %s", cudaGetErrorString(e));
  if (d_out) CU(cudaMemcpyAsync(d_out, dd, sizeof(double), cudaMemcpyDeviceToDevice, s));
  // ---- null model and its score: lambda_max
  LogitArgs la{};
  la.X = X; la.xtype = xtype; la.n = n; la.p = p; la.ldx = ldx; la.y = y;
  la.ytype = xtype == OEM_F64 ? OEM_F64 : OEM_F32;
  la.beta = bcur; la.ldb = (int32_t)pq; la.intercept = icpt; la.rc = rc; la.part = part; la.g = gv;
  LAUNCH(OEM_PROF_CHUNKS, launch_logit_null(bcur, npen, (int)pq, (int)pq, icpt, b.Zg, g.q, (int)p, g.ycols, ocol, n, s));
  LAUNCH(OEM_PROF_LOGIT, launch_logit_grad(la, npen, grid, s));
  if (opt->lambdas) {
    CU(upload(lam, opt->lambdas, sizeof(double) * npen * L, s));
  } else {
    LAUNCH(OEM_PROF_LAMBDA, launch_lambda_grid(gv, (int)p, P.dpens, npen, L, opt->lambda_min_ratio, lam, s));
  }
  // ---- the path: for each lambda, outer (proximal Newton) steps, each an
  // X pass, the surrogate's resume state, one inner OEM launch and the step
  constexpr int kMaxOuter = 100;
  std::vector<IterTask> tasks;
  int32_t* hflags = nullptr;
  CU(cudaMallocHost(&hflags, sizeof(int32_t) * npen));
  int rr = OEM_OK;
  for (int l = 0; l < L && !rr; ++l) {
    CU(cudaMemcpy2DAsync(lam_l, sizeof(double), lam + l, sizeof(double) * L, sizeof(double), npen,
                         cudaMemcpyDeviceToDevice, s));
    CU(cudaMemsetAsync(flags, 0, sizeof(int32_t) * npen, s));
    CU(cudaMemsetAsync(its_l, 0, sizeof(int32_t) * npen, s));
    CU(cudaMemsetAsync(conv_l, 0, npen, s));
    for (int t = 1; t <= kMaxOuter; ++t) {
      if (l > 0 || t > 1) LAUNCH(OEM_PROF_LOGIT, launch_logit_grad(la, npen, grid, s));
      LAUNCH(OEM_PROF_LOGIT, launch_logit_state(gv, bcur, npen, (int)pq, (int)pq, dd, P.dpens, opt->iter_precision,
                                               st_u, st_beta, st_ctl, 40 * npen, s));
      if ((rr = launch_iter_layout(ctx, pq, 1, G32, ldg32, G64, gv, dd, lam_l, P, &inner, I, bnew, it_new,
                                   conv_in, 0, tasks, s, st_u, st_beta, st_ctl)))
        break;
      LAUNCH(OEM_PROF_LOGIT, launch_logit_step(bcur, bnew, npen, (int)pq, (int)pq, it_new, its_l, opt->tol, flags,
                                              t == kMaxOuter ? 1 : 0, conv_l, s));
      CU(cudaMemcpyAsync(hflags, flags, sizeof(int32_t) * npen, cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      bool all = true;
      for (int k = 0; k < npen; ++k) all &= hflags[k] != 0;
      if (all) break;
    }
    if (rr) break;
    // beta[k][l][:p], beta0[k][l], iters, converged
    CU(cudaMemcpy2DAsync(beta + (size_t)l * p, sizeof(double) * L * p, bcur, sizeof(double) * pq,
                         sizeof(double) * p, npen, cudaMemcpyDeviceToDevice, s));
    if (beta0) {
      if (icpt)
        CU(cudaMemcpy2DAsync(beta0 + l, sizeof(double) * L, bcur + p, sizeof(double) * pq, sizeof(double), npen,
                             cudaMemcpyDeviceToDevice, s));
      else
        CU(cudaMemset2DAsync(beta0 + l, sizeof(double) * L, 0, sizeof(double), npen, s));
    }
    CU(cudaMemcpy2DAsync(iters + l, sizeof(int32_t) * L, its_l, sizeof(int32_t), sizeof(int32_t), npen,
                         cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpy2DAsync(converged + l, L, conv_l, 1, 1, npen, cudaMemcpyDeviceToDevice, s));
  }
  CU(cudaMemcpyAsync(lambdas_out, lam, sizeof(double) * npen * L, cudaMemcpyDeviceToDevice, s));
  cudaFreeHost(hflags);
  return rr;
}

}  // extern "C"
