// Host-side helpers shared by the C-ABI entry points (api.cu) and the
// serving runtime (server.cu): the context, the workspace arena, argument
// checks, the Gram-pass plan, penalty upload and the iteration plan.
#pragma once

#include "oem_internal.cuh"

#include <algorithm>
#include <numeric>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
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
  // iteration layouts chosen by timing, per (p, Grams, penalties, precision,
  // groups): CTAs per task, instances per task, grid mode
  std::map<std::array<int64_t, 5>, std::array<int, 3>> iter_tuned;
  int64_t tune_runs = 0;
  // iteration counts of the last oem_fit_path / oem_fit / oem_cv call (device
  // [B][npen][L], in the workspace until the next call), for oem_iter_stats
  const int32_t* last_iters = nullptr;
  int last_B = 0, last_npen = 0, last_L = 0;
};

namespace oem {
namespace host {

inline int fail(oem_ctx* ctx, int code, const char* fmt, ...) {
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

// Whether `s` is being captured into a CUDA graph.
inline bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

// Host data to device memory, ordered on `s`: cudaMemcpyAsync, or inside a
// stream capture kernels that carry the bytes (the host buffer may be gone
// by the time the graph is replayed).
inline cudaError_t upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!bytes) return cudaSuccess;
  if (capturing(s)) return launch_upload(dst, src, bytes, s);
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
}

inline cudaEvent_t prof_event(oem_ctx* ctx) {
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
    // no timing inside a stream capture (its events are never recorded)
    if (ctx->prof && !capturing(s) && (e0 = prof_event(ctx))) cudaEventRecord(e0, s);
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

// LAUNCH that stores the failure in r instead of returning.
#define LAUNCH_R(cls, call, r)                                                           \
  do {                                                                                   \
    cudaError_t e_;                                                                      \
    {                                                                                    \
      ProfScope ps_(ctx, s, (cls), 1);                                                   \
      e_ = (call);                                                                       \
    }                                                                                    \
    ++ctx->launches;                                                                     \
    if (e_ != cudaSuccess)                                                               \
      r = fail(ctx, OEM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));          \
  } while (0)

inline cudaError_t lanczos_prof(oem_ctx* ctx, cudaStream_t s, const double* G, int64_t p, int64_t ldg,
                         int batch, int64_t strideG, int steps, LanczosWork w, double* d,
                         cudaStream_t s2, int64_t* launches) {
  const int64_t before = *launches;
  cudaEvent_t e0 = ctx->prof ? prof_event(ctx) : nullptr;
  if (e0) cudaEventRecord(e0, s);
  cudaError_t e = launch_lanczos(G, p, ldg, batch, strideG, steps, w, d, ctx->dstatus, s2, launches);
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

// Lanczos work space for `batch` Grams of order p.
template <typename A>
inline void lanczos_request(A& ar, LanczosWork& w, int64_t p, int batch, int steps) {
  ar.add(&w.V, (size_t)batch * (lanczos_steps_eff(steps, p) + 3) * p);
  ar.add(&w.alpha, (size_t)batch * kLzMax);
  ar.add(&w.beta, (size_t)batch * kLzMax);
  ar.add(&w.fro, (size_t)batch);
  ar.add(&w.gmax, (size_t)batch);
  ar.add(&w.mlen, (size_t)batch);
  ar.add(&w.Gs, (size_t)batch * p * p);
}

inline int arena_commit(oem_ctx* ctx, Arena& A, cudaStream_t s) {
  const size_t need = A.total();
  if (need > ctx->budget)
    return fail(ctx, OEM_EBUDGET, "workspace of %zu bytes exceeds the budget of %zu bytes", need,
                ctx->budget);
  if (need > ctx->arena_cap) {
    if (capturing(s))
      return fail(ctx, OEM_EINVAL,
                  "inside a stream capture the workspace cannot grow to %zu bytes: make the same call "
                  "once outside the capture first", need);
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

inline size_t elem_size(int32_t xtype) { return xtype == OEM_F64 ? 8 : xtype == OEM_F32 ? 4 : 2; }

inline int check_x(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
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

inline int resolve_mode(oem_ctx* ctx, int32_t mode, int32_t xtype, int32_t* out) {
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

inline bool tc_mode(int32_t mode) {
  return mode == OEM_GRAM_TF32 || mode == OEM_GRAM_BF16 || mode == OEM_GRAM_SPLIT_BF16;
}

// Everything the Gram pass needs in the workspace.
struct GramPlan {
  int32_t mode, q, ycols, T, nt, ntiles;
  int32_t ocols = 0;     // column of ones (centring)
  bool centre = false;
  int64_t chunk_rows, nblk;
  int max_chunks;
  int K;
  bool sorted;
  // TMA-fed tensor-core path (split-BF16 / bfloat16): packed copy of Z
  bool tma = false;
  int32_t qp = 0;
  int64_t rows_cap = 0;
  int pmax_chunks = 0;
  // direct TMA from X (bfloat16, one fold, no ones): only the tail is packed
  bool direct = false;
  int32_t nbx = 0, tail_cols = 0;
};

// ones: 0 = Z = [X | y]; kOnesShifted = Z = [X | y | 1] on X and y shifted
// by sampled column means (the intercept option of the linear model; a
// bfloat16 request then runs in split mode, since the shifted X is not
// bfloat16); kOnes = Z = [X | y | 1] unshifted (logistic regression).
constexpr int kOnesShifted = 1, kOnes = 2;
// x_direct: X is bfloat16 device memory at a 16-byte aligned address (the
// TMA may read it in place).
inline GramPlan plan_gram(oem_ctx* ctx, int64_t n, int64_t p, int K, int32_t mode, bool sorted,
                          int ones = 0, bool x_direct = false) {
  GramPlan g;
  const bool centre = ones == kOnesShifted;
  if (centre && mode == OEM_GRAM_BF16) mode = OEM_GRAM_SPLIT_BF16;
  g.mode = mode;
  g.centre = centre;
  // bfloat16 mode carries the float32 y as three bfloat16 pieces (exact)
  g.ycols = (mode == OEM_GRAM_BF16) ? 3 : 1;
  g.ocols = ones ? 1 : 0;
  g.q = (int32_t)p + g.ycols + g.ocols;
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
  // the TMA path needs a bfloat16 copy of Z (hi, and lo in split mode); it
  // is taken while that copy uses at most half of the context's budget,
  // otherwise the converting kernel reads X directly
  if (mode == OEM_GRAM_SPLIT_BF16 || mode == OEM_GRAM_BF16) {
    g.qp = (g.q + 127) / 128 * 128;
    g.rows_cap = n + kGramPackRows * (int64_t)K;
    // The persistent kernel takes items (chunk, tile) in turn; a chunk count
    // that is a multiple of sms / gcd(ntiles, sms) gives every SM the same
    // number of items.
    const int64_t sms = ctx->num_sms;
    const int64_t unit = sms / std::gcd((int64_t)g.ntiles, sms);
    const int64_t want = std::max<int64_t>(1, (target_items / g.ntiles + unit / 2) / unit) * unit;
    int64_t tcr = (g.rows_cap + want - 1) / want;
    tcr = std::max<int64_t>(1024, (tcr + 127) / 128 * 128);
    g.pmax_chunks = (int)((g.rows_cap + tcr - 1) / tcr + K);
    g.direct = x_direct && mode == OEM_GRAM_BF16 && !sorted && ones == 0 && K == 1;
    if (g.direct) {
      g.nbx = (int32_t)(p / 64);
      g.tail_cols = (g.q - 64 * g.nbx + 63) / 64 * 64;
    }
    const size_t bytes = g.direct ? (size_t)g.rows_cap * g.tail_cols * 2
                                  : (size_t)g.rows_cap * g.qp * 2 * (mode == OEM_GRAM_SPLIT_BF16 ? 2 : 1);
    const size_t partial = (size_t)g.pmax_chunks * g.ntiles * g.T * g.T * sizeof(double);
    g.tma = bytes + partial <= ctx->budget / 2;
    if (!g.tma) g.direct = false;
    if (g.tma) {
      g.chunk_rows = tcr;
      g.max_chunks = (int)((n + tcr - 1) / tcr + K);
    }
  }
  return g;
}

struct GramBufs {
  int32_t *blk_counts = nullptr, *blk_offsets = nullptr, *perm = nullptr;
  int32_t* ipos = nullptr;  // packed copy in fold order: each row's packed row
  ChunkTable ct{};
  double* partial = nullptr;
  double* Zg = nullptr;
  TmaBufs t{};
  uint16_t *zhi = nullptr, *zlo = nullptr;
  float* shift = nullptr;  // [p + 1] column shifts (centring)
};

inline void gram_request(Arena& A, const GramPlan& g, int64_t n, GramBufs& b) {
  if (g.sorted) {
    A.add(&b.blk_counts, (size_t)g.nblk * g.K);
    A.add(&b.blk_offsets, (size_t)g.nblk * g.K);
    A.add(&b.perm, (size_t)n);
    if (g.tma && !g.direct) A.add(&b.ipos, (size_t)n);
  }
  A.add(&b.ct.row0, (size_t)g.max_chunks);
  A.add(&b.ct.row1, (size_t)g.max_chunks);
  A.add(&b.ct.fold, (size_t)g.max_chunks);
  A.add(&b.ct.count, 1);
  A.add(&b.ct.fold_c0, (size_t)g.K + 1);
  A.add(&b.ct.fold_off, (size_t)g.K + 1);
  A.add(&b.partial, (size_t)(g.tma ? g.pmax_chunks : g.max_chunks) * g.ntiles * g.T * g.T);
  A.add(&b.Zg, (size_t)g.K * g.q * g.q);
  if (g.centre) A.add(&b.shift, (size_t)(g.q - g.ycols - g.ocols) + 1);
  if (g.tma) {
    A.add(&b.zhi, (size_t)g.rows_cap * (g.direct ? g.tail_cols : g.qp));
    if (g.mode == OEM_GRAM_SPLIT_BF16) A.add(&b.zlo, (size_t)g.rows_cap * g.qp);
    A.add(&b.t.pc.row0, (size_t)g.pmax_chunks);
    A.add(&b.t.pc.row1, (size_t)g.pmax_chunks);
    A.add(&b.t.pc.fold, (size_t)g.pmax_chunks);
    A.add(&b.t.pc.count, 1);
    A.add(&b.t.pc.fold_c0, (size_t)g.K + 1);
    A.add(&b.t.pc.fold_off, (size_t)g.K + 1);
  }
}

// fold sort (if any) -> chunk table -> Gram partials -> per-fold Z Grams.
inline int run_gram(oem_ctx* ctx, const GramPlan& g, GramBufs& b, const void* X, int32_t xtype,
             int64_t n, int64_t p, int64_t ldx, const void* y, const uint8_t* fold,
             bool require_nonempty, cudaStream_t s, bool shift_ready = false) {
  if (g.sorted) {
    LAUNCH(OEM_PROF_FOLD_SORT, launch_fold_count(fold, n, g.K, b.blk_counts, g.nblk, s));
    LAUNCH(OEM_PROF_FOLD_SORT, launch_fold_scan(b.blk_counts, g.nblk, g.K, g.chunk_rows, b.blk_offsets, b.ct,
                            g.max_chunks, ctx->dstatus, require_nonempty ? 1 : 0, s));
    LAUNCH(OEM_PROF_FOLD_SORT, launch_fold_scatter(fold, n, g.K, b.blk_offsets, b.perm, b.ipos, b.ct.fold_off, s));
  } else {
    LAUNCH(OEM_PROF_CHUNKS, launch_identity_chunks(n, g.chunk_rows, b.ct, g.max_chunks, s));
  }
  GramArgs a{};
  a.X = X; a.xtype = xtype; a.n = n; a.p = p; a.ldx = ldx; a.y = y;
  a.perm = g.sorted ? b.perm : nullptr;
  a.ipos = g.sorted ? b.ipos : nullptr;
  a.mode = g.mode; a.q = g.q; a.ycols = g.ycols; a.T = g.T; a.ntile1 = g.nt; a.ntiles = g.ntiles;
  a.ocols = g.ocols;
  if (g.centre) {
    if (!shift_ready) LAUNCH(OEM_PROF_CHUNKS, launch_col_shift(X, xtype, n, p, ldx, y, b.shift, s));
    a.shift = b.shift;
  }
  a.ct = b.ct; a.max_chunks = g.max_chunks; a.partial = b.partial; a.dstatus = ctx->dstatus;
  if (g.tma) {
    b.t.zhi = b.zhi;
    b.t.zlo = b.zlo;
    b.t.qp = g.qp;
    b.t.rows_cap = g.rows_cap;
    b.t.max_chunks = g.pmax_chunks;
    b.t.chunk_rows = g.chunk_rows;
    b.t.direct = g.direct ? 1 : 0;
    b.t.nbx = g.nbx;
    b.t.tail_cols = g.tail_cols;
    // The hi.hi product is summed over 128 rows (split mode) or 256 rows
    // (bfloat16) in float32 tensor memory before it is added to the
    // compensated sum; the cross terms, 2^-8 smaller, over 1,024 rows.
    const int flush = g.mode == OEM_GRAM_SPLIT_BF16 ? 128 : 256;
    if (g.direct) LAUNCH(OEM_PROF_GRAM_TC, launch_tail_pack(a, b.t, s));
    else LAUNCH(OEM_PROF_GRAM_TC, launch_zpack(a, g.K, b.t, s));
    LAUNCH(OEM_PROF_GRAM_TC, launch_gram_tma(a, b.t, flush, s));
    GramArgs r = a;
    r.ct.fold_c0 = b.t.pc.fold_c0;
    LAUNCH(OEM_PROF_GRAM_REDUCE, launch_gram_reduce(r, g.K, b.Zg, s));
    return OEM_OK;
  }
  if (tc_mode(g.mode)) {
    // Rows summed in float32 tensor memory before the compensated flush. The
    // tensor cores' float32 accumulation rounds toward zero, so the error
    // grows with the number of MMAs per window (measured at n = 2e6, p = 100,
    // split mode: 32 rows 3.2e-7, 64 rows 5.2e-7, 256 rows 1.6e-6 relative
    // Frobenius): split mode (4 products) uses 64-row windows, bfloat16 / tf32
    // 256 / 128. OEM_GRAM_FLUSH_ROWS overrides.
    int flush = g.mode == OEM_GRAM_SPLIT_BF16 ? 64 : g.mode == OEM_GRAM_TF32 ? 128 : 256;
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

// ---------------------------------------------------------------- X in host memory
// X (and y, fold) may live in host memory (the out-of-memory case of the
// paper's big.oem, Section 5.7, done as a stream): row blocks are copied into
// two device staging buffers on a copy stream while the previous block's
// Gram pass runs, and the blocks' fold Grams of Z and row counts are added up.
// Pinned host memory overlaps the copies with the passes; pageable memory
// works without overlap.
inline bool host_resident(const void* ptr) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

struct StreamBufs {
  bool on = false;          // X is streamed from host memory
  bool y_host = false, fold_host = false;
  int64_t rows = 0;         // rows per block
  unsigned char* X[2] = {nullptr, nullptr};
  unsigned char* y[2] = {nullptr, nullptr};
  uint8_t* fold[2] = {nullptr, nullptr};
  double* Zg = nullptr;     // [K][q][q] accumulated
  int64_t* cnt = nullptr;   // [K]
  int64_t* off = nullptr;   // [K+1]
};
// The Gram pass may read bfloat16 X in place by TMA (direct mode): device X
// at a 16-byte aligned address, or X streamed through the (aligned) staging
// buffers.
inline bool direct_x_ok(const void* X, int32_t xtype, const StreamBufs& sb) {
  return xtype == OEM_BF16 && (sb.on || ((uintptr_t)X & 15) == 0);
}

// Rows per block: about 256 MB of X, a multiple of 64, at most n
// (OEM_STREAM_ROWS overrides, for experiments).
inline int64_t stream_block_rows(int64_t n, int64_t ldx, int32_t xtype) {
  int64_t rb = std::max<int64_t>(65536, ((int64_t)256 << 20) / (ldx * elem_size(xtype))) / 64 * 64;
  if (const char* ev = getenv("OEM_STREAM_ROWS")) {
    const long long v = atoll(ev);
    if (v >= 64) rb = v / 64 * 64;
  }
  return std::min<int64_t>(n, rb);
}

template <typename A>
inline void stream_request(A& ar, StreamBufs& sb, int64_t rows, int64_t ldx, int32_t xtype, int K, int q,
                           bool with_fold) {
  const size_t ye = xtype == OEM_F64 ? 8 : 4;
  for (int i = 0; i < 2; ++i) {
    ar.add(&sb.X[i], (size_t)rows * ldx * elem_size(xtype));
    if (sb.y_host) ar.add(&sb.y[i], (size_t)rows * ye);
    if (with_fold && sb.fold_host) ar.add(&sb.fold[i], (size_t)rows);
  }
  ar.add(&sb.Zg, (size_t)K * q * q);
  ar.add(&sb.cnt, (size_t)K);
  ar.add(&sb.off, (size_t)K + 1);
}

// The Gram pass over X wherever it lives; *Zg and *fold_off receive the fold
// Grams of Z and the fold offsets the assembly reads.
inline int run_gram_any(oem_ctx* ctx, const GramPlan& g, GramBufs& b, StreamBufs& sb, const void* X,
                        int32_t xtype, int64_t n, int64_t p, int64_t ldx, const void* y,
                        const uint8_t* fold, bool require_nonempty, cudaStream_t s, const double** Zg,
                        const int64_t** fold_off) {
  if (!sb.on) {
    int r = run_gram(ctx, g, b, X, xtype, n, p, ldx, y, fold, require_nonempty, s);
    *Zg = b.Zg;
    *fold_off = b.ct.fold_off;
    return r;
  }
  const size_t xrow = (size_t)ldx * elem_size(xtype), ye = xtype == OEM_F64 ? 8 : 4;
  cudaStream_t cs = nullptr;
  cudaEvent_t start = nullptr, copied[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};
  int r = OEM_OK;
  auto cleanup = [&]() {
    if (cs) cudaStreamDestroy(cs);
    if (start) cudaEventDestroy(start);
    for (int i = 0; i < 2; ++i) {
      if (copied[i]) cudaEventDestroy(copied[i]);
      if (used[i]) cudaEventDestroy(used[i]);
    }
  };
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) {
    cleanup();
    return fail(ctx, OEM_ECUDA, "stream / event creation failed");
  }
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&used[i], cudaEventDisableTiming) != cudaSuccess) {
      cleanup();
      return fail(ctx, OEM_ECUDA, "event creation failed");
    }
  const int64_t nblocks = (n + sb.rows - 1) / sb.rows;
  const int64_t zlen = (int64_t)g.K * g.q * g.q;
  cudaError_t e = cudaEventRecord(start, s);  // the copies follow the caller's earlier work
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, start, 0);
  for (int64_t blk = 0; blk < nblocks && e == cudaSuccess && !r; ++blk) {
    const int i = (int)(blk & 1);
    const int64_t r0 = blk * sb.rows, rows = std::min<int64_t>(sb.rows, n - r0);
    // ---- copy stream: block blk into buffer i once the pass of block blk-2 is done
    if (blk >= 2) e = cudaStreamWaitEvent(cs, used[i], 0);
    const void* Xb = X;
    const void* yb = y;
    const uint8_t* fb = fold;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sb.X[i], (const unsigned char*)X + r0 * xrow, (size_t)rows * xrow,
                          cudaMemcpyHostToDevice, cs);
    Xb = sb.X[i];
    if (e == cudaSuccess && sb.y_host) {
      e = cudaMemcpyAsync(sb.y[i], (const unsigned char*)y + r0 * ye, (size_t)rows * ye, cudaMemcpyHostToDevice, cs);
      yb = sb.y[i];
    } else {
      yb = (const unsigned char*)y + r0 * ye;
    }
    if (fold) {
      if (e == cudaSuccess && sb.fold_host) {
        e = cudaMemcpyAsync(sb.fold[i], fold + r0, (size_t)rows, cudaMemcpyHostToDevice, cs);
        fb = sb.fold[i];
      } else {
        fb = fold + r0;
      }
    }
    if (e == cudaSuccess) e = cudaEventRecord(copied[i], cs);
    // ---- compute stream: the block's Gram pass and the accumulation
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, copied[i], 0);
    if (e != cudaSuccess) break;
    r = run_gram(ctx, g, b, Xb, xtype, rows, p, ldx, yb, fb, false, s, blk > 0);
    if (r) break;
    LAUNCH_R(OEM_PROF_GRAM_REDUCE, launch_zg_accumulate(sb.Zg, b.Zg, zlen, blk == 0 ? 1 : 0, sb.cnt, b.ct.fold_off,
                                                     g.K, s), r);
    if (r) break;
    e = cudaEventRecord(used[i], s);
  }
  if (!r && e != cudaSuccess) r = fail(ctx, OEM_ECUDA, "streamed Gram pass: %s", cudaGetErrorString(e));
  if (!r)
    LAUNCH_R(OEM_PROF_GRAM_REDUCE, launch_zg_offsets(sb.cnt, sb.off, g.K, require_nonempty ? 1 : 0, ctx->dstatus, s), r);
  cleanup();
  *Zg = sb.Zg;
  *fold_off = sb.off;
  return r;
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

inline int prepare_pens(oem_ctx* ctx, const oem_penalty* pens, int npen, int64_t p, PenPlan& P) {
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
    if (q.kind < OEM_LASSO || q.kind > OEM_SPARSE_GROUP_LASSO)
      return fail(ctx, OEM_EINVAL, "penalty %d: unknown kind %d", i, q.kind);
    const bool grouped = q.kind >= OEM_GROUP_LASSO;
    if (q.kind == OEM_ENET && !(q.alpha >= 0.0 && q.alpha <= 1.0))
      return fail(ctx, OEM_EINVAL, "penalty %d: elastic net alpha=%g not in [0,1]", i, q.alpha);
    if ((q.kind == OEM_MCP || q.kind == OEM_GROUP_MCP) && !(q.gamma > 1.0))
      return fail(ctx, OEM_EINVAL, "penalty %d: MCP gamma=%g must exceed 1", i, q.gamma);
    if ((q.kind == OEM_SCAD || q.kind == OEM_GROUP_SCAD) && !(q.gamma > 2.0))
      return fail(ctx, OEM_EINVAL, "penalty %d: SCAD gamma=%g must exceed 2", i, q.gamma);
    if (q.kind == OEM_SPARSE_GROUP_LASSO && !(q.alpha >= 0.0 && q.alpha <= 1.0))
      return fail(ctx, OEM_EINVAL, "penalty %d: sparse group lasso tau=%g not in [0,1]", i, q.alpha);
    DevPenalty d{};
    d.kind = q.kind;
    d.alpha64 = (q.kind == OEM_ENET || q.kind == OEM_SPARSE_GROUP_LASSO) ? q.alpha : 1.0;
    d.gamma64 = (q.kind == OEM_MCP || q.kind == OEM_SCAD || q.kind == OEM_GROUP_MCP ||
                 q.kind == OEM_GROUP_SCAD) ? q.gamma : 3.0;
    d.alpha = (float)d.alpha64;
    d.gamma = (float)d.gamma64;
    if (q.w && (!grouped || q.kind == OEM_SPARSE_GROUP_LASSO)) {
      P.w64[i].assign(q.w, q.w + p);
      P.w32[i].resize(p);
      for (int64_t j = 0; j < p; ++j) {
        if (!(q.w[j] >= 0.0) || !std::isfinite(q.w[j]))
          return fail(ctx, OEM_EINVAL, "penalty %d: weight %lld is %g", i, (long long)j, q.w[j]);
        P.w32[i][j] = (float)q.w[j];
      }
    }
    if (grouped) {
      if (!q.group || q.ngroups < 1)
        return fail(ctx, OEM_EINVAL, "penalty %d: a group penalty needs group ids and ngroups >= 1", i);
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

inline void pens_request(Arena& A, PenPlan& P) {
  A.add(&P.dpens, (size_t)P.npen);
  for (int i = 0; i < P.npen; ++i) {
    if (!P.w64[i].empty()) { A.add(&P.d_w64[i], P.w64[i].size()); A.add(&P.d_w32[i], P.w32[i].size()); }
    if (!P.grp[i].empty()) { A.add(&P.d_grp[i], P.grp[i].size()); A.add(&P.d_cg[i], P.cg[i].size()); }
  }
}

inline int pens_upload(oem_ctx* ctx, PenPlan& P, cudaStream_t s) {
  for (int i = 0; i < P.npen; ++i) {
    DevPenalty& d = P.host[i];
    if (!P.w64[i].empty()) {
      CU(upload(P.d_w64[i], P.w64[i].data(), P.w64[i].size() * 8, s));
      CU(upload(P.d_w32[i], P.w32[i].data(), P.w32[i].size() * 4, s));
      d.w64 = P.d_w64[i];
      d.w32 = P.d_w32[i];
    }
    if (!P.grp[i].empty()) {
      CU(upload(P.d_grp[i], P.grp[i].data(), P.grp[i].size() * 4, s));
      CU(upload(P.d_cg[i], P.cg[i].data(), P.cg[i].size() * 8, s));
      d.grp = P.d_grp[i];
      d.cg = P.d_cg[i];
    }
  }
  CU(upload(P.dpens, P.host.data(), sizeof(DevPenalty) * P.npen, s));
  return OEM_OK;
}

inline int check_opts(oem_ctx* ctx, const oem_options* o) {
  if (!o) return fail(ctx, OEM_EINVAL, "options are NULL");
  if (o->nlambda < 1 || o->nlambda > 100000) return fail(ctx, OEM_EINVAL, "nlambda=%d", o->nlambda);
  if (!o->lambdas && !(o->lambda_min_ratio > 0.0 && o->lambda_min_ratio <= 1.0))
    return fail(ctx, OEM_EINVAL, "lambda_min_ratio=%g not in (0,1]", o->lambda_min_ratio);
  if (!(o->tol > 0.0)) return fail(ctx, OEM_EINVAL, "tol=%g must be > 0", o->tol);
  if (o->max_iter < 1) return fail(ctx, OEM_EINVAL, "max_iter=%lld must be >= 1", (long long)o->max_iter);
  if (o->iter_precision != OEM_ITER_F32 && o->iter_precision != OEM_ITER_F64)
    return fail(ctx, OEM_EINVAL, "iter_precision=%d", o->iter_precision);
  const int c = o->cluster_ctas;
  if (!(c == 0 || c == 1 || c == 2 || c == 4 || c == 8 || (c >= 16 && c <= 4096)))
    return fail(ctx, OEM_EINVAL, "cluster_ctas=%d not in {0,1,2,4,8} or [16,4096]", c);
  const int g = o->instances_per_task;
  if (!(g == 0 || g == 1 || g == 2 || g == 4 || g == 8))
    return fail(ctx, OEM_EINVAL, "instances_per_task=%d not in {0,1,2,4,8}", g);
  if (o->autotune != 0 && o->autotune != 1)
    return fail(ctx, OEM_EINVAL, "autotune=%d not in {0,1}", o->autotune);
  if (o->intercept != 0 && o->intercept != 1)
    return fail(ctx, OEM_EINVAL, "intercept=%d not in {0,1}", o->intercept);
  if (o->standardize != 0 && o->standardize != 1)
    return fail(ctx, OEM_EINVAL, "standardize=%d not in {0,1}", o->standardize);
  return OEM_OK;
}

// Row slices of p rows over a cluster of C CTAs: even boundaries moved forward
// to the next row where a slice may start (group starts for group penalties).
// Slice boundaries are multiples of 4 rows (the iteration kernel moves whole
// 16-byte rows of 4 float32 between CTAs) and allowed rows (group starts).
inline void make_slices(int64_t p, int C, const std::vector<char>& allowed, int32_t* slice, int* max_rows) {
  slice[0] = 0;
  slice[C] = (int32_t)p;
  for (int r = 1; r < C; ++r) {
    int64_t bnd = std::max<int64_t>(slice[r - 1], (p * r) / C);
    bnd = (bnd + 3) & ~(int64_t)3;
    while (bnd < p && (!allowed[bnd] || (bnd & 3))) ++bnd;
    slice[r] = (int32_t)std::min<int64_t>(bnd, p);
  }
  int mr = 1;
  for (int r = 0; r < C; ++r) mr = std::max(mr, slice[r + 1] - slice[r]);
  *max_rows = mr;
}

// Even row slices for the replicated kernel (no group alignment: every CTA
// holds all rows for the thresholds). align = 4 in cluster mode (16-byte
// units of the exchanged words), 1 in grid mode.
inline void make_slices_even(int64_t p, int C, int align, int32_t* slice, int* max_rows) {
  slice[0] = 0;
  for (int r = 1; r < C; ++r) {
    int64_t bnd = (p * r) / C;
    bnd = (bnd + align - 1) / align * align;
    slice[r] = (int32_t)std::min<int64_t>(std::max<int64_t>(bnd, slice[r - 1]), p);
  }
  slice[C] = (int32_t)p;
  int mr = 1;
  for (int r = 0; r < C; ++r) mr = std::max(mr, slice[r + 1] - slice[r]);
  *max_rows = mr;
}

// Which iteration kernel serves order p: the replicated one (oem_iter.cu)
// up to kIterRepMaxP, the row-owned one (oem_iter_rows.cu) beyond.
inline bool iter_rows_kernel(int64_t p) { return p > kIterRepMaxP; }

// Bound of every device wait of the iteration kernels, in clock cycles
// (about 2 s at 2 GHz). OEM_DEVICE_WAIT_CYCLES overrides it (tests of the
// timeout path).
inline int64_t iter_wait_cycles() {
  const char* v = std::getenv("OEM_DEVICE_WAIT_CYCLES");
  if (v && *v) {
    const long long c = std::atoll(v);
    if (c > 0) return c;
  }
  return 4000000000LL;
}

// Tests of the timeout path only: OEM_DEVICE_WAIT_TEST=1 makes the first
// exchange of every iteration launch wait for data that nobody sends, so
// that its bounded wait expires.
inline int iter_test_stall() {
  const char* v = std::getenv("OEM_DEVICE_WAIT_TEST");
  return (v && v[0] == '1') ? 1 : 0;
}

inline int iter_smem_probe(const IterLaunch& P, bool rows) {
  return rows ? oem_iter_rows_max_cluster(P) : oem_iter_max_cluster(P);
}

constexpr size_t kIterSmemCap = 227 * 1024;

// Iteration launch plan for B tasks of the same shape (a fit or the K+1
// Grams of a cross validation): cluster size, slices, shared memory.
struct IterPlan {
  int C = 1, M = 1, Mg = 1, max_rows = 0, smem_rows = 0;
  int ucache = 0;         // row-owned kernel, float32: column-block cache slots
  size_t smem = 0;
  int32_t slice[kMaxCluster + 1] = {0};
  bool grid = false;      // cooperative grid mode (C CTAs per task, any C)
  bool rows = false;      // row-owned kernel (p > kIterRepMaxP)
  std::vector<int32_t> gslice;  // grid mode: C + 1 row boundaries
  bool groups = false;
  bool tune = false;      // time the candidate layouts at the first run
  int max_tasks = 0;      // task-table capacity (B x npen)
  IterTask* d_tasks = nullptr;
  uint8_t* d_allowed = nullptr;
  // grid mode exchange space: per task [2][ldgs][8] float64 dbeta + slots +
  // barrier (sized for the widest case), and the row boundaries
  unsigned char* d_xbuf = nullptr;
  size_t xbuf_task = 0;
  int32_t* d_gslice = nullptr;
  int gslice_cap = 0;     // boundaries per task
};

// Grid-mode exchange space of one task, the larger of the two kernels'
// needs (row-owned: tagged words of dbeta and of every CTA's maxima, barrier
// words; replicated: tagged words of G dbeta). At most kMaxGridCtas CTAs
// per task.
constexpr int kMaxGridCtas = 256;
inline size_t grid_xbuf_task_bytes(int64_t p) {
  return std::max(oem_iter_rows_xbuf_bytes((int)p, 8, OEM_ITER_F64, kMaxGridCtas),
                  oem_iter_xbuf_bytes((int)p, 8, OEM_ITER_F64));
}

// Cluster size C and Mg instances per task for B Grams of npen instances;
// returns OK with the shared-memory plan, or an error when nothing fits. In
// grid mode C is the number of CTAs per task (one per SM, every task's CTAs
// resident together) and every Gram row must fit in shared memory.
inline int layout_iter(oem_ctx* ctx, int64_t p, int B, const PenPlan& P, int prec, int C, int Mg,
                       bool grid, IterPlan& I) {
  I.Mg = Mg;
  I.M = oem_iter_mpad(Mg);
  I.grid = grid;
  I.rows = iter_rows_kernel(p);
  const int ntasks = B * ((P.npen + Mg - 1) / Mg);
  const bool rows = I.rows;
  auto fixed_of = [&](int max_rows) {
    return rows ? oem_iter_rows_smem_fixed((int)p, Mg, max_rows, prec)
                : oem_iter_smem_fixed((int)p, Mg, max_rows, prec, grid, I.groups);
  };
  auto probe_of = [&](int CC) {
    IterLaunch probe{};
    probe.ntasks = ntasks; probe.C = CC; probe.M = I.M; probe.precision = prec;
    probe.smem = I.smem; probe.max_rows = I.max_rows; probe.grid = grid ? 1 : 0;
    probe.groups = I.groups ? 1 : 0;
    probe.wide = (!rows && prec == OEM_ITER_F32 && p > kIterWideP && I.max_rows <= 16 && I.M <= 2) ? 1 : 0;
    return iter_smem_probe(probe, rows);
  };
  if (grid) {
    C = std::min<int>(C, ctx->num_sms / std::max(1, ntasks));
    C = std::min(C, kMaxGridCtas);
    C = (int)std::min<int64_t>(C, rows ? (p + 3) / 4 : p);
    if (C < 2) return fail(ctx, OEM_EUNSUPPORTED, "grid mode needs at least 2 CTAs per task");
    I.gslice.assign((size_t)C + 1, 0);
    if (rows) make_slices(p, C, P.allowed, I.gslice.data(), &I.max_rows);
    else make_slices_even(p, C, 1, I.gslice.data(), &I.max_rows);
    const size_t fixed = fixed_of(I.max_rows);
    const size_t per = rows ? oem_iter_rows_smem_per_row((int)p, prec) : oem_iter_smem_per_row((int)p, prec);
    I.smem_rows = I.max_rows;
    I.ucache = 0;
    I.smem = fixed + (size_t)I.max_rows * per;
    I.C = C;
    if (rows && prec == OEM_ITER_F32) {
      // float32 row-owned kernel: every column block of the slice cached
      I.smem_rows = 0;
      I.ucache = oem_iter_rows_ucache_slots((int)p, Mg, I.max_rows, prec, kIterSmemCap - 1024);
      I.smem = oem_iter_rows_smem_ucache((int)p, Mg, I.max_rows, prec, I.ucache);
      if (I.ucache < oem_iter_rows_blocks((int)p))
        return fail(ctx, OEM_EUNSUPPORTED, "grid mode: %d rows per CTA do not fit", I.max_rows);
    }
    if (I.smem + 1024 > kIterSmemCap)
      return fail(ctx, OEM_EUNSUPPORTED, "grid mode: %d rows per CTA do not fit", I.max_rows);
    if (probe_of(C) < 1) return fail(ctx, OEM_EUNSUPPORTED, "grid mode: no CTA fits on an SM");
    return OEM_OK;
  }
  for (;; C /= 2) {
    if (rows) {
      make_slices(p, C, P.allowed, I.slice, &I.max_rows);
    } else {
      make_slices_even(p, C, 4, I.slice, &I.max_rows);
    }
    const size_t fixed = fixed_of(I.max_rows);
    if (fixed + 1024 > kIterSmemCap)
      return fail(ctx, OEM_EUNSUPPORTED, "p=%lld with %d instances per task too large for the iteration kernel",
                  (long long)p, Mg);
    const size_t per = rows ? oem_iter_rows_smem_per_row((int)p, prec) : oem_iter_smem_per_row((int)p, prec);
    I.smem_rows = (int)std::min<size_t>((size_t)I.max_rows, (kIterSmemCap - fixed) / per);
    I.smem = fixed + (size_t)I.smem_rows * per;
    I.ucache = 0;
    if (rows && prec == OEM_ITER_F32) {
      // float32 row-owned kernel: the 16-column blocks of G that nonzero
      // dbeta entries touch, cached while slots last (the rest read from L2)
      I.smem_rows = 0;
      I.ucache = oem_iter_rows_ucache_slots((int)p, Mg, I.max_rows, prec, kIterSmemCap - 1024);
      I.smem = oem_iter_rows_smem_ucache((int)p, Mg, I.max_rows, prec, I.ucache);
    }
    I.C = C;
    if (probe_of(C) >= 1) return OEM_OK;
    if (C == 1) return fail(ctx, OEM_ECUDA, "no cluster configuration of the iteration kernel fits");
  }
}

inline std::array<int64_t, 5> tune_key(int64_t p, int B, const PenPlan& P, int prec, bool groups) {
  return {p, (int64_t)B, (int64_t)P.npen, (int64_t)prec, (int64_t)groups};
}

// Default layout: about 32 rows per CTA (at most 16 CTAs per cluster, and the
// clusters of all B Grams resident at once), then the fewest instances per
// task whose clusters all fit on the device at once (more clusters share the
// work of one Gram; each iterates fewer instances per step).
// cluster_ctas above 16 selects grid mode with that many CTAs per task (at
// most the SMs the tasks leave each).
inline int plan_iter(oem_ctx* ctx, int64_t p, int B, const PenPlan& P, const oem_options* o, IterPlan& I) {
  const int prec = o->iter_precision;
  I.groups = false;
  for (int i = 0; i < P.npen; ++i) I.groups |= P.host[i].kind >= OEM_GROUP_LASSO;
  I.max_tasks = B * P.npen;
  int C = o->cluster_ctas;
  if (C <= 0) {
    const int want = (int)std::min<int64_t>(16, std::max<int64_t>(1, (p + 31) / 32));
    const int byB = std::max(1, ctx->num_sms / std::max(1, B));
    C = 1;
    while (C * 2 <= std::min(want, byB) && C < 16) C *= 2;
  }
  int Mg = o->instances_per_task;
  if (Mg <= 0) {
    Mg = oem_iter_mpad(P.npen);
    while (Mg > 1 && (int64_t)B * ((P.npen + Mg / 2 - 1) / (Mg / 2)) * C <= ctx->num_sms) Mg /= 2;
  }
  Mg = std::min(Mg, std::max(1, P.npen));
  // the replicated kernel keeps every row of its Mg instances in shared
  // memory: fewer instances per task where they do not fit
  while (o->instances_per_task <= 0 && Mg > 1 && !iter_rows_kernel(p) &&
         oem_iter_smem_fixed((int)p, Mg, (int)std::min<int64_t>(p, 256), prec, false, I.groups) + 1024 >
             kIterSmemCap)
    Mg /= 2;
  bool grid = o->cluster_ctas > kMaxCluster;
  I.gslice_cap = std::max(ctx->num_sms, o->cluster_ctas) + 1;
  if (grid) C = o->cluster_ctas;
  if (o->cluster_ctas <= 0) {
    // grid mode when a cluster cannot keep all its Gram rows (float32
    // row-owned kernel: all column blocks of its slices) in shared memory
    // but the whole device can
    IterPlan J = I;
    if (layout_iter(ctx, p, B, P, prec, C, Mg, false, J) == OEM_OK &&
        (J.ucache > 0 ? J.ucache < oem_iter_rows_blocks((int)p) : J.smem_rows < J.max_rows)) {
      IterPlan K = I;
      if (layout_iter(ctx, p, B, P, prec, ctx->num_sms, Mg, true, K) == OEM_OK) {
        grid = true;
        C = ctx->num_sms;
      }
    }
  }
  auto it = ctx->iter_tuned.find(tune_key(p, B, P, prec, I.groups));
  I.tune = false;
  if (o->autotune && o->cluster_ctas <= 0 && o->instances_per_task <= 0) {
    if (it != ctx->iter_tuned.end()) { C = it->second[0]; Mg = it->second[1]; grid = it->second[2] != 0; }
    else I.tune = true;
  }
  return layout_iter(ctx, p, B, P, prec, C, Mg, grid, I);
}

inline void iter_request(Arena& A, int64_t p, int B, IterPlan& I) {
  const size_t T = (size_t)std::max(B, I.max_tasks);
  A.add(&I.d_tasks, T);
  if (I.groups) A.add(&I.d_allowed, (size_t)p + 1);
  I.xbuf_task = grid_xbuf_task_bytes(p);
  A.add(&I.d_xbuf, T * I.xbuf_task);
  A.add(&I.d_gslice, T * (size_t)I.gslice_cap);
}

// Launch the iteration for B Grams with the layout in I (task table written
// on stream s); max_loops > 0 stops every task after that many iterations.
inline int launch_iter_layout(oem_ctx* ctx, int64_t p, int B, const float* G32, int ldg,
                              const double* G64, const double* c, const double* d,
                              const double* lam, PenPlan& P, const oem_options* o, IterPlan& I,
                              double* beta, int32_t* iters, uint8_t* conv, int64_t max_loops,
                              std::vector<IterTask>& tasks, cudaStream_t s,
                              double* st_u = nullptr, double* st_beta = nullptr,
                              int32_t* st_ctl = nullptr) {
  const int L = o->nlambda, npen = P.npen, Mg = I.Mg;
  const int S = (npen + Mg - 1) / Mg;
  tasks.assign((size_t)B * S, IterTask{});
  for (int b = 0; b < B; ++b)
    for (int q = 0; q < S; ++q) {
      IterTask& t = tasks[(size_t)b * S + q];
      const int k0 = q * Mg;
      t.p = (int)p; t.npen = std::min(Mg, npen - k0); t.L = L; t.ldg = ldg;
      t.max_rows = I.max_rows; t.smem_rows = I.smem_rows; t.ucache = I.ucache; t.resume = 0;
      for (int r = 0; r <= kMaxCluster; ++r) t.slice[r] = r <= I.C ? I.slice[r] : (int32_t)p;
      t.G32 = G32 ? G32 + (size_t)b * p * ldg : nullptr;
      t.G64 = G64 ? G64 + (size_t)b * p * p : nullptr;
      t.c = c + (size_t)b * p;
      t.d = d + b;
      t.lam = lam + (size_t)k0 * L;
      t.pens = P.dpens + k0;
      t.allowed = I.groups ? I.d_allowed : nullptr;
      t.beta = beta + ((size_t)b * npen + k0) * L * p;
      t.iters = iters + ((size_t)b * npen + k0) * L;
      t.conv = conv + ((size_t)b * npen + k0) * L;
      if (st_u) {  // resume every instance from the given (u, beta) state
        t.resume = 1;
        t.st_u = st_u + ((size_t)b * npen + k0) * p * 2;
        t.st_beta = st_beta + ((size_t)b * npen + k0) * p;
        t.st_ctl = st_ctl + (size_t)(b * S + q) * 40;
      }
      if (I.grid) {
        const size_t ldgs = (size_t)((p + 3) & ~3LL);
        unsigned char* x = I.d_xbuf + (size_t)(b * S + q) * I.xbuf_task;
        t.xD = x;
        t.xslot = reinterpret_cast<unsigned*>(x + 2 * ldgs * 8 * sizeof(double));
        t.xbar = t.xslot + 3 * 16;
        t.gslice = I.d_gslice;
      }
    }
  if (I.grid) {
    if ((int)I.gslice.size() > I.gslice_cap || tasks.size() * I.xbuf_task == 0)
      return fail(ctx, OEM_ECUDA, "grid mode buffers too small");
    CU(cudaMemsetAsync(I.d_xbuf, 0, tasks.size() * I.xbuf_task, s));
    CU(upload(I.d_gslice, I.gslice.data(), sizeof(int32_t) * I.gslice.size(), s));
  }
  CU(upload(I.d_tasks, tasks.data(), sizeof(IterTask) * tasks.size(), s));
  IterLaunch Lc{};
  Lc.tasks = I.d_tasks; Lc.ntasks = (int)tasks.size(); Lc.C = I.C; Lc.M = I.M;
  Lc.precision = o->iter_precision;
  Lc.tol = o->tol; Lc.max_iter = o->max_iter; Lc.max_loops = max_loops; Lc.dstatus = ctx->dstatus;
  Lc.smem = I.smem;
  Lc.grid = I.grid ? 1 : 0;
  Lc.max_rows = I.max_rows;
  Lc.groups = I.groups ? 1 : 0;
  Lc.wide = (!I.rows && o->iter_precision == OEM_ITER_F32 && p > kIterWideP && I.max_rows <= 16 &&
             I.M <= 2) ? 1 : 0;
  Lc.wait_cycles = iter_wait_cycles();
  Lc.test_stall = iter_test_stall();
  if (I.rows) LAUNCH(OEM_PROF_ITER, launch_oem_iter_rows(Lc, s));
  else LAUNCH(OEM_PROF_ITER, launch_oem_iter(Lc, s));
  return OEM_OK;
}

// Autotuner: time each candidate layout (cluster CTAs around the default, and
// 1, 2, 4, 8 instances per task) for a fixed number of iterations on the real
// inputs, keep the fastest for this shape in the context. The candidates'
// partial outputs are overwritten by the full run that follows.
inline int tune_iter(oem_ctx* ctx, int64_t p, int B, const float* G32, int ldg, const double* G64,
                     const double* c, const double* d, const double* lam, PenPlan& P,
                     const oem_options* o, IterPlan& I, double* beta, int32_t* iters,
                     uint8_t* conv, cudaStream_t s) {
  constexpr int64_t kLoops = 48;
  std::vector<std::array<int, 3>> cand;  // (CTAs per task, instances per task, grid)
  const int C0 = I.grid ? 16 : I.C;
  for (int Mg : {1, 2, 4, 8}) {
    if (!(Mg <= oem_iter_mpad(P.npen) && (Mg == 1 || Mg / 2 < P.npen))) continue;
    for (int C : {C0 / 2, C0, C0 * 2})
      if (C >= 1 && C <= kMaxCluster) cand.push_back({C, Mg, 0});
    cand.push_back({ctx->num_sms, Mg, 1});
  }
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  std::vector<IterTask> tasks;
  float best = 1e30f;
  std::array<int, 3> pick{I.C, I.Mg, I.grid ? 1 : 0};
  const bool prof = ctx->prof;
  ctx->prof = false;  // tuning launches are not part of the profile
  int rc = OEM_OK;
  for (auto cd : cand) {
    const int C = cd[0], Mg = cd[1];
    const bool grid = cd[2] != 0;
    IterPlan J = I;
    if (layout_iter(ctx, p, B, P, o->iter_precision, C, Mg, grid, J) != OEM_OK) continue;
    if (!grid && J.C != C) continue;
    // once untimed (module load), once timed
    if ((rc = launch_iter_layout(ctx, p, B, G32, ldg, G64, c, d, lam, P, o, J, beta, iters, conv,
                                 2, tasks, s)))
      break;
    if (cudaEventRecord(e0, s) != cudaSuccess) { rc = fail(ctx, OEM_ECUDA, "event record failed"); break; }
    if ((rc = launch_iter_layout(ctx, p, B, G32, ldg, G64, c, d, lam, P, o, J, beta, iters, conv,
                                 kLoops, tasks, s)))
      break;
    float ms = 0.f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = fail(ctx, OEM_ECUDA, "timing the iteration layouts failed");
      break;
    }
    ++ctx->tune_runs;
    if (ms < best) { best = ms; pick = {J.C, Mg, grid ? 1 : 0}; }
  }
  ctx->prof = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  ctx->iter_tuned[tune_key(p, B, P, o->iter_precision, I.groups)] = pick;
  return layout_iter(ctx, p, B, P, o->iter_precision, pick[0], pick[1], pick[2] != 0, I);
}

// B tasks: Gram b uses G32 + b p ldg (or G64 + b p p), c + b p, d + b, and
// writes beta + b npen L p, iters / conv + b npen L.
inline int run_iter(oem_ctx* ctx, int64_t p, int B, const float* G32, int ldg, const double* G64,
             const double* c, const double* d, const double* lam, PenPlan& P,
             const oem_options* o, IterPlan& I, double* beta, int32_t* iters, uint8_t* conv,
             cudaStream_t s) {
  if (I.groups) {
    std::vector<uint8_t> al(P.allowed.begin(), P.allowed.end());
    CU(upload(I.d_allowed, al.data(), al.size(), s));
  }
  if (I.tune) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      int r = tune_iter(ctx, p, B, G32, ldg, G64, c, d, lam, P, o, I, beta, iters, conv, s);
      if (r) return r;
    }
  }
  std::vector<IterTask> tasks;
  return launch_iter_layout(ctx, p, B, G32, ldg, G64, c, d, lam, P, o, I, beta, iters, conv, 0,
                            tasks, s);
}


}  // namespace host
}  // namespace oem
