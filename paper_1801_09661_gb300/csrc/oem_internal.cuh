// Internal declarations shared by the CUDA translation units of liboem.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/oem.h"

namespace oem {

constexpr int kNumSMsHint = 152;
// Packed copies of Z pad every fold's rows to a multiple of this.
constexpr int kGramPackRows = 64;

// Device-side status word bits (ctx->dstatus[0]); oem_sync() maps them to codes.
enum : unsigned {
  kStatNotConv = 1u,
  kStatNonFinite = 2u,
  kStatTimeout = 4u,
  kStatEmptyFold = 8u,
};

// ----------------------------------------------------------------------------
// Gram pass work decomposition. The augmented matrix Z = [X | y-columns] has q
// columns; its upper triangle is cut into T x T tiles (ti <= tj). Rows are
// processed in fold order (perm) as "chunks", each inside one fold. One work
// item = (tile, chunk); it writes a T x T float64 partial sum. The reduction
// adds the partials of each fold's chunks in a fixed order (deterministic).
// ----------------------------------------------------------------------------
struct ChunkTable {
  int64_t* row0;     // [max_chunks] first sorted row of the chunk
  int64_t* row1;     // [max_chunks] one past the last sorted row
  int32_t* fold;     // [max_chunks] fold of the chunk
  int32_t* count;    // [1] number of valid chunks
  int32_t* fold_c0;  // [K+1] first chunk of each fold (prefix)
  int64_t* fold_off; // [K+1] row offsets of each fold in sorted order
};

struct GramArgs {
  const void* X;
  int32_t xtype;
  int64_t n, p, ldx;
  const void* y;
  const int32_t* perm;  // sorted row -> original row (NULL = identity)
  const int32_t* ipos;  // original row -> packed row (-1: no fold), or NULL
  int32_t mode;         // OEM_GRAM_*
  int32_t q;            // augmented columns: p + ycols + ocols
  int32_t ycols;        // y columns appended (1, or 3 bfloat16 pieces)
  int32_t ocols;        // 1: a column of ones after the y columns (column sums, n)
  const float* shift;   // [p + 1] or NULL: subtracted from X's columns and y
  int32_t T;            // tile size
  int32_t ntile1;       // tiles per side
  int32_t ntiles;       // upper-triangular tile count
  ChunkTable ct;
  int32_t max_chunks;
  double* partial;      // [max_chunks][ntiles][T][T]
  unsigned* dstatus;
};

// Packed bfloat16 copy of Z for the TMA-fed Gram kernel (split-BF16 and
// bfloat16 modes): every fold's rows padded with zero rows to a multiple of
// 32, qp = round_up(q, 128) columns.
struct TmaBufs {
  void* zhi;            // [rows_cap][qp] bfloat16 (direct: [rows_cap][tail_cols], the tail)
  void* zlo;            // [rows_cap][qp] bfloat16 (split mode) or NULL
  int32_t qp;
  int64_t rows_cap;     // n + kGramPackRows K
  ChunkTable pc;        // chunks of packed rows; pc.fold_off = packed fold offsets
  int32_t max_chunks;
  int64_t chunk_rows;
  // direct mode (bfloat16 X, one fold, no column of ones): the first nbx
  // 64-column boxes of Z are read by TMA from X itself; only the tail --
  // X's columns [64 nbx, p), the y columns, zeros up to tail_cols -- is packed
  int32_t direct, nbx, tail_cols;
};

// tile index -> (ti, tj), ti <= tj, row-major over the upper triangle
__host__ __device__ inline void tile_coords(int t, int nt, int* ti, int* tj) {
  int i = 0, rem = t;
  while (rem >= nt - i) { rem -= nt - i; ++i; }
  *ti = i;
  *tj = i + rem;
}

// Launchers (return cudaError_t of the launch).
cudaError_t launch_fold_count(const uint8_t* fold, int64_t n, int K, int32_t* blk_counts,
                              int64_t nblk, cudaStream_t s);
cudaError_t launch_fold_scan(const int32_t* blk_counts, int64_t nblk, int K, int64_t chunk_rows,
                             int32_t* blk_offsets, ChunkTable ct, int max_chunks,
                             unsigned* dstatus, int require_nonempty, cudaStream_t s);
// ipos (or NULL): each row's row in the packed copy of Z, in fold order with
// every fold padded with zero rows to a multiple of kGramPackRows (-1 for a
// row outside every fold); fold_off: the folds' offsets in sorted order
cudaError_t launch_fold_scatter(const uint8_t* fold, int64_t n, int K, const int32_t* blk_offsets,
                                int32_t* perm, int32_t* ipos, const int64_t* fold_off, cudaStream_t s);
cudaError_t launch_identity_chunks(int64_t n, int64_t chunk_rows, ChunkTable ct, int max_chunks,
                                   cudaStream_t s);

cudaError_t launch_gram_simt(const GramArgs& a, cudaStream_t s);
cudaError_t launch_gram_tc(const GramArgs& a, int flush_rows, cudaStream_t s);
cudaError_t launch_check_finite(const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
                                const void* y, unsigned* dstatus, cudaStream_t s);

// Reduce partials into per-fold raw Grams of Z (float64, full symmetric,
// [K][q][q]).
size_t gram_tma_smem_bytes();
// packed chunk table + the packing pass (fold order, zero-padded folds)
cudaError_t launch_zpack(const GramArgs& a, int K, const TmaBufs& t, cudaStream_t s);
// direct mode: packed chunk table and the tail of Z (bfloat16 X, one fold)
cudaError_t launch_tail_pack(const GramArgs& a, const TmaBufs& t, cudaStream_t s);
cudaError_t launch_gram_tma(const GramArgs& a, const TmaBufs& t, int flush_rows, cudaStream_t s);
cudaError_t launch_gram_reduce(const GramArgs& a, int K, double* Zg, cudaStream_t s);

// Extract per-fold X^T X, X^T y, y^T y from Z Grams (raw) in the public layout.
cudaError_t launch_extract_folds(const double* Zg, int K, int q, int p, int ycols, double* Gk,
                                 double* ck, double* ytyk, int64_t* nk, const int64_t* fold_off,
                                 cudaStream_t s);

// Centring and scaling of the assembled statistics (intercept / standardize
// options): ocol = column of ones in Z (or -1); cen [B][2p+1] receives the
// means of the (shifted) X columns, the scales sd and the mean of the
// (shifted) y of each fit.
struct CentreArgs {
  int32_t ocol = -1;
  int32_t intercept = 0, standardize = 0;
  double* cen = nullptr;
};

// Assemble scaled statistics: b = 0 full data, b = k+1 leave fold k out.
// G64 [B][p][p], G32 [B][p][ldg32] (may be NULL), c [B][p], N [B], cnt [B].
cudaError_t launch_assemble(const double* Zg, int K, int q, int p, int ycols,
                            const int64_t* fold_off, int with_leave_out, double* G64, float* G32,
                            int ldg32, double* c, double* N, double* cnt, cudaStream_t s,
                            const CentreArgs& ce = CentreArgs());
// Column shifts for centring: shift[j] = the mean of column j over a sample
// of at most 8,192 rows (exactly the common value when the sample is
// constant), shift[p] the same for y.
cudaError_t launch_col_shift(const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
                             const void* y, float* shift, cudaStream_t s);
// Streamed Gram pass: acc (+)= blk ([len] float64, K fold Grams of Z) and
// the fold row counts from the block's sorted offsets; then the offsets.
// Copy `bytes` of host memory to device memory by kernels that carry the
// bytes in their launch parameters, so that a stream capture records the
// data itself (a captured cudaMemcpyAsync would read the host buffer again
// at every replay).
cudaError_t launch_upload(void* dst, const void* src, size_t bytes, cudaStream_t s);
cudaError_t launch_zg_accumulate(double* acc, const double* blk, int64_t len, int first, int64_t* cnt,
                                 const int64_t* fold_off, int K, cudaStream_t s);
cudaError_t launch_zg_offsets(const int64_t* cnt, int64_t* off, int K, int require_nonempty, unsigned* dstatus,
                              cudaStream_t s);
// Standardized paths back to the original scale: beta_all [B][npen][L][p]
// divided by sd in place; bprime [B][npen][L] (may be NULL) = the intercept
// in the shifted coordinates of the Gram pass; beta0 [npen][L] (may be
// NULL) = the intercept of fit b = 0 on the original scale.
cudaError_t launch_unstandardize(double* beta_all, int B, int npen, int nlambda, int p,
                                 const double* cen, const float* shift, int intercept,
                                 double* bprime, double* beta0, cudaStream_t s);

// Lanczos d for a batch of float64 Grams.
#ifdef __CUDACC__
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier of the nctas CTAs of one task in a cooperative launch (all of them
// resident): bar[0] counts arrivals, bar[1] is the generation; gen is the
// caller's copy of the generation (thread 0). Every wait is bounded (lim
// cycles); returns false in every thread of the CTA on timeout.
__device__ __forceinline__ bool group_barrier(unsigned* bar, unsigned nctas, unsigned& gen, long long lim) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    const unsigned g = gen;
    __threadfence();  // this CTA's global writes before its arrival
    if (atomicAdd(&bar[0], 1u) == nctas - 1) {
      atomicExch(&bar[0], 0u);  // nobody arrives again before the generation moves
      __threadfence();
      atomicExch(&bar[1], g + 1);
    } else {
      const long long t0 = clock64();
      int spins = 0;
      while (ld_acquire_gpu(&bar[1]) == g) {
        if (++spins > 8) __nanosleep(32);  // fewer polls on the shared line
        if (clock64() - t0 > lim) { ok = 0; break; }
      }
    }
    __threadfence();
    gen = g + 1;
  }
  return __syncthreads_and(ok) != 0;
}
#endif

struct LanczosWork {
  double* V;       // [batch][steps + 3][p]: basis rows (double-float pairs) when they stay out of shared memory
  float2* alpha;   // [batch][kLzMax] double-float, of s_b G_b
  float2* beta;    // [batch][kLzMax]
  double* fro;     // [batch] ||s_b G_b||_F^2
  float* gmax;     // [batch] max |G_b| (sets the power-of-two scaling s_b)
  int32_t* mlen;   // [batch] steps taken
  float2* Gs;      // [batch][p][p] (hi, lo) float32 copy of G_b
};
constexpr int kLzMax = 128;       // longest recurrence kept per Gram
constexpr int kLzThreads = 512;
constexpr size_t kLzSmemMax = 230400;  // dynamic shared memory per CTA (227 KB less room for static arrays)

// Cluster layout of the Lanczos kernel for a Gram of order p: C CTAs own
// `per` rows each; byte offsets of its shared-memory arrays; whether the
// basis rows (vsm) and the (hi, lo) rows of G (gsm) fit in shared memory.
struct LzPlan {
  int C;
  int64_t per, vstride;
  bool vsm, gsm;
  size_t off_X, off_P1, off_P2, off_B, off_W, off_V, off_G, smem;
};
inline LzPlan lanczos_plan(int64_t p, int steps, int C) {
  LzPlan L{};
  L.C = C;
  L.per = (p + C - 1) / C;
  L.vstride = L.per | 1;  // odd stride: projections of different i hit different banks
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o += (bytes + 15) & ~(size_t)15; return at; };
  // every array holds double-float pairs (8 bytes)
  L.off_X = take(8 * (size_t)p);
  L.off_P1 = take(8 * (size_t)C * kLzMax);
  L.off_P2 = take(8 * (size_t)C * kLzMax);
  L.off_B = take(8 * 16);
  L.off_W = take(8 * (size_t)L.per);
  const size_t vbytes = 8 * (size_t)(steps + 1) * (size_t)L.vstride;
  L.vsm = o + vbytes <= kLzSmemMax;
  L.off_V = L.vsm ? take(vbytes) : 0;
  const size_t gbytes = 8 * (size_t)L.per * (size_t)p;
  L.gsm = o + gbytes <= kLzSmemMax;
  L.off_G = L.gsm ? take(gbytes) : 0;
  L.smem = o;
  return L;
}
// CTAs per Gram: 16 rows per CTA at least, a power of two up to 16.
inline int lanczos_cluster(int64_t p) {
  int C = 1;
  while (C < 16 && (int64_t)(2 * C) * 16 <= p) C *= 2;
  return C;
}
// Lanczos steps actually taken for a request of `steps` (0 = 64) at order p.
inline int lanczos_steps_eff(int steps, int64_t p) {
  if (steps <= 0) steps = 64;
  if (steps > kLzMax) steps = kLzMax;
  if (steps > p) steps = (int)p;
  return steps < 1 ? 1 : steps;
}
cudaError_t launch_lanczos(const double* G, int64_t p, int64_t ldg, int batch, int64_t strideG,
                           int steps, LanczosWork w, double* d, unsigned* dstatus, cudaStream_t s,
                           int64_t* launches);

// Penalty descriptor on the device.
struct DevPenalty {
  int32_t kind;
  float alpha, gamma;
  double alpha64, gamma64;
  const float* w32;     // [p] or NULL
  const double* w64;    // [p] or NULL
  const int32_t* grp;   // [p] group ids (group lasso) or NULL
  const double* cg;     // [ngroups]
  int32_t ngroups;
};

// Scalar updates of Section 2.2 (Eqs. lasso, net, mcp, scad); wl = w_j lambda.
template <typename T>
__device__ __forceinline__ T thr_scalar(int kind, T u, T wl, T alpha, T gamma, T d) {
  // Every branch is sign(u) num / den for one (num, den) pair and zero where
  // |u| does not pass the threshold; the pair is chosen by selects, so lanes
  // of a warp that hold different penalties do not diverge. In the regions
  // |u| > gamma wl d (MCP) and |u| > (d + 1) wl (SCAD) the update is u / d
  // and s > 0 holds there (gamma d > 1).
  const T au = fabs(u);
  const T s = au - (kind == OEM_ENET ? wl * alpha : wl);
  T num = s, den = d;
  if (kind == OEM_ENET) {
    den = d + wl * (T(1) - alpha);
  } else if (kind == OEM_MCP) {
    if (au <= wl * gamma * d) { num = gamma * s; den = gamma * d - T(1); }
    else num = au;
  } else if (kind == OEM_SCAD) {
    if (au > (d + T(1)) * wl) {
      if (au <= wl * gamma * d) { num = (gamma - T(1)) * au - wl * gamma; den = (gamma - T(1)) * d - T(1); }
      else num = au;
    }
  }
  return s > T(0) ? copysign(num / den, u) : T(0);
}

// Plain form of the iteration (one launch per OEM iteration, one instance):
// beta_new = threshold(c + d beta - G beta) with float64 dot products of the
// float32 Gram rows; red[0] = max|beta_new - beta|, red[1] = max|beta_new|
// (float64 bit patterns, must start at zero).
cudaError_t launch_plain_iter(int p, const float* G32, int ldg, const double* c, double d,
                              const double* beta, double* beta_new, const DevPenalty* pen,
                              double lam, unsigned long long* red, cudaStream_t s);

// Lambda grid: lam[pen][l] from c (full data).
cudaError_t launch_lambda_grid(const double* c, int p, const DevPenalty* pens, int npen,
                               int nlambda, double ratio, double* lam, cudaStream_t s);

// OEM iteration. One task = one Gram and its instances (penalties); a launch
// runs one thread-block cluster per task. Tasks of one launch may differ in p.
constexpr int kMaxCluster = 16;
struct IterTask {
  int32_t p, npen, L, ldg;
  int32_t max_rows;      // longest CTA slice
  int32_t smem_rows;     // leading rows of each slice kept in shared memory
  int32_t ucache;        // row-owned kernel, float32: column-block cache slots
                         // (resident rows unused: smem_rows = 0)
  int32_t resume;        // 1: start from st_* instead of beta = 0, u = c
  int32_t slice[kMaxCluster + 1];  // CTA r owns rows [slice[r], slice[r+1])
  const float* G32;      // [p][ldg] (float32 iteration)
  const double* G64;     // [p][p]   (float64 iteration)
  const double* c;       // [p] scaled X^T y
  const double* d;       // [1]
  const double* lam;     // [npen][L]
  const DevPenalty* pens;// [npen]
  const uint8_t* allowed;// [p+1] rows where a slice may start (group starts) or NULL
  double* beta;          // [npen][L][p]
  int32_t* iters;        // [npen][L]
  uint8_t* conv;         // [npen][L]
  double* st_u;          // [npen][p][2] saved u (hi, lo) or NULL (no state)
  double* st_beta;       // [npen][p]
  int32_t* st_ctl;       // [40]: per instance (lambda index, iterations, done, -);
                         // [32] = every instance done
  int32_t* fin_out;      // where the launch writes "every instance done" (or NULL)
  // grid mode only (IterLaunch::grid): the C CTAs of the task exchange
  // through global memory instead of a cluster's shared memory
  const int32_t* gslice; // [C+1] CTA r owns rows [gslice[r], gslice[r+1])
  void* xD;              // zeroed before the launch; replicated kernel: [2][p][M]
                         // tagged words of G dbeta (two per float64 value);
                         // row-owned kernel: [2][round_up(p,4)][M] dbeta (T)
  unsigned* xslot;       // [3][2M] maxima slots, zeroed (row-owned kernel)
  unsigned* xbar;        // [2] barrier count and generation, zeroed (row-owned kernel)
};
struct IterLaunch {
  const IterTask* tasks; // device array
  int32_t ntasks, C, M, precision;
  int32_t grid;          // 1: cooperative launch, C CTAs per task, global-memory exchange
  int32_t max_rows;      // longest CTA slice of the launch (picks the row group)
  int32_t groups;        // some task has a group penalty (group arrays in shared memory)
  int32_t wide;          // long rows: 512 threads, one G row per warp (replicated kernel, float32)
  double tol;
  int64_t max_iter;      // per lambda
  int64_t max_loops;     // per launch (<= 0: run to completion)
  int64_t wait_cycles;   // bound of every device wait (clock64 cycles)
  int32_t test_stall;    // tests only: the first exchange waits for data nobody sends,
                         // so its bounded wait runs out (both iteration kernels)
  unsigned* dstatus;
  size_t smem;
};
// Instances per Gram are padded to M in {1, 2, 4, 8}.
int oem_iter_mpad(int npen);

// Replicated-update kernel (oem_iter.cu), used for p <= kIterRepMaxP: every
// CTA of a task keeps u, beta and dbeta of all p rows and applies the
// thresholds to all of them; only the mat-vec rows are split between CTAs.
// Above it the replicated threshold work outweighs the exchange it saves and
// the row-owned kernel serves.
constexpr int kIterRepMaxP = 1024;
constexpr int kIterWideP = 512;    // above, with at most 16 rows per CTA: the long-row variant
// Shared memory besides the resident Gram rows, and per resident row.
size_t oem_iter_smem_fixed(int p, int M, int max_rows, int precision, bool grid, bool groups);
size_t oem_iter_smem_per_row(int p, int precision);
// Clusters of this configuration the device can co-schedule (0: none); in
// grid mode, CTAs per SM.
int oem_iter_max_cluster(const IterLaunch& P);
cudaError_t launch_oem_iter(const IterLaunch& P, cudaStream_t s);
// Grid-mode exchange buffer of one task (tagged 64-bit words, both parities).
size_t oem_iter_xbuf_bytes(int p, int M, int precision);

// Row-owned kernel (oem_iter_rows.cu), used for p > kIterRepMaxP: CTA r owns
// rows of u and beta and exchanges dbeta and the maxima (grid mode: tagged
// words in the exchange buffer, which needs oem_iter_rows_xbuf_bytes).
size_t oem_iter_rows_xbuf_bytes(int p, int M, int precision, int C);
size_t oem_iter_rows_smem_fixed(int p, int npen, int max_rows, int precision);
// Column-block cache of the row-owned kernel (float32): the most slots
// (16 columns of every row of a slice each) whose shared memory stays within
// cap (0 when none fit).
int oem_iter_rows_ucache_slots(int p, int npen, int max_rows, int precision, size_t cap);
int oem_iter_rows_blocks(int p);  // 16-column blocks of order p (one cache slot each)
size_t oem_iter_rows_smem_ucache(int p, int npen, int max_rows, int precision, int slots);
size_t oem_iter_rows_smem_per_row(int p, int precision);
int oem_iter_rows_max_cluster(const IterLaunch& P);
cudaError_t launch_oem_iter_rows(const IterLaunch& P, cudaStream_t s);

// CV scoring from raw fold Grams of Z and the fold paths.
// With ocol >= 0 the model has the intercept bprime [B][npen][L] on the
// column of ones (shifted coordinates).
cudaError_t launch_cv_score(const double* Zg, int K, int q, int p, int ycols,
                            const int64_t* fold_off, const double* beta_all, int npen,
                            int nlambda, double* mse, double* cvm, double* cvsd,
                            int32_t* idx_min, int32_t* idx_1se, int32_t* best, cudaStream_t s,
                            int ocol = -1, const double* bprime = nullptr);

// Logistic regression (Section 4, Hessian bound 1/4): one pass over X per
// outer step for every penalty's beta ([npen][ldb] float64, the intercept
// last), partial sums per CTA, g = Z^T (y - mu) / n into g [npen][ldb].
struct LogitArgs {
  const void* X;
  int32_t xtype;
  int64_t n, p, ldx;
  const void* y;
  int32_t ytype;        // OEM_F32 or OEM_F64
  const double* beta;
  int32_t ldb;
  int32_t intercept;
  int32_t rc;           // rows per shared-memory chunk
  float2* part;         // [grid][npen][pq] (hi, lo)
  double* g;            // [npen][ldb]
};
size_t logit_grad_smem(int64_t p, int rc, int npen, int intercept);
cudaError_t launch_logit_grad(const LogitArgs& a, int npen, int grid, cudaStream_t s);
cudaError_t launch_logit_state(const double* g, const double* beta, int npen, int pq, int ldb,
                               const double* d, const DevPenalty* pens, int precision, double* st_u,
                               double* st_beta, int32_t* st_ctl, int nctl, cudaStream_t s);
cudaError_t launch_logit_step(double* beta, const double* bnew, int npen, int pq, int ldb,
                              const int32_t* it_new, int32_t* its, double tol, int32_t* flags,
                              int last_outer, uint8_t* conv, cudaStream_t s);
cudaError_t launch_logit_null(double* beta, int npen, int pq, int ldb, int intercept, const double* Zg,
                              int q, int p, int ycols, int ocol, int64_t n, cudaStream_t s);
cudaError_t launch_logit_gram(const double* Zg, int q, int p, int ocol, int intercept, int64_t n,
                              double* G64, float* G32, int ldg, cudaStream_t s);

// Copy the full-data (b = 0) paths out of the batched buffers.
cudaError_t launch_copy_paths(const double* beta_all, const int32_t* it_all, const uint8_t* cv_all,
                              int npen, int nlambda, int p, double* beta, int32_t* iters,
                              uint8_t* conv, unsigned* dstatus, cudaStream_t s);

}  // namespace oem
