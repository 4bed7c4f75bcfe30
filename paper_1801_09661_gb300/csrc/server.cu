// Serving runtime (include/oem.h, oem_server_*): admission by device-memory
// budget, per-job preparation on the job's own stream (fold sort, Gram pass,
// fold assembly, d, lambda grid), continuous batching of the OEM iterations
// of every ready job in rounds of one cluster launch (state saved between
// rounds), CV scoring and copy-out per job. The plain form runs jobs one at
// a time with a float32 CUDA-core Gram and one launch per OEM iteration.
#include "host.cuh"

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

using namespace oem::host;

namespace oem {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One OEM iteration of one instance (plain form): one warp per row.
__global__ void plain_iter_kernel(int p, const float* __restrict__ G, int ldg,
                                  const double* __restrict__ c, double d,
                                  const double* __restrict__ beta, double* __restrict__ beta_new,
                                  const DevPenalty* __restrict__ pen, double lam,
                                  unsigned long long* red) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * warps + (threadIdx.x >> 5);
  if (row >= p) return;
  const float* g = G + (size_t)row * ldg;
  double s = 0.0;
  for (int j = lane; j < p; j += 32) s = fma((double)g[j], beta[j], s);
  s = warp_sum_d(s);
  if (lane == 0) {
    const DevPenalty pe = *pen;
    double de = d;
    if (pe.kind == OEM_MCP) de = fmax(de, 1.01 / pe.gamma64);
    if (pe.kind == OEM_SCAD) de = fmax(de, 1.01 / (pe.gamma64 - 1.0));
    const double w = pe.w64 ? pe.w64[row] : 1.0;
    const double u = c[row] + de * beta[row] - s;
    const double b = thr_scalar<double>(pe.kind, u, w * lam, pe.alpha64, pe.gamma64, de);
    beta_new[row] = b;
    atomicMax(&red[0], (unsigned long long)__double_as_longlong(fabs(b - beta[row])));
    atomicMax(&red[1], (unsigned long long)__double_as_longlong(fabs(b)));
  }
}

cudaError_t launch_plain_iter(int p, const float* G32, int ldg, const double* c, double d,
                              const double* beta, double* beta_new, const DevPenalty* pen,
                              double lam, unsigned long long* red, cudaStream_t s) {
  plain_iter_kernel<<<(p + 7) / 8, 256, 0, s>>>(p, G32, ldg, c, d, beta, beta_new, pen, lam, red);
  return cudaGetLastError();
}

}  // namespace oem

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void arena_assign(Arena& A, void* base) {
  char* q = (char*)base;
  for (auto& r : A.req) {
    *r.first = r.second ? q : nullptr;
    q += (r.second + 255) & ~(size_t)255;
  }
}

struct SrvJob {
  int64_t id = 0;
  oem_job spec{};
  int state = OEM_JOB_QUEUED;
  int status = OEM_OK;
  double t_submit = 0.0, t_done = 0.0;
  int B = 1, L = 0, q = 0, ycols = 1, ldg = 0, K = 0, gram_mode = OEM_GRAM_FP32;
  int64_t p = 0;
  bool groups = false;
  GramPlan gp{};
  PenPlan P;
  Arena prep, res;
  size_t prep_bytes = 0, res_bytes = 0;
  void* prep_mem = nullptr;
  void* res_mem = nullptr;
  bool prep_held = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t prep_ev = nullptr, done_ev = nullptr;
  int rounds = 0;
  // prep-only device buffers
  int32_t *blk_counts = nullptr, *blk_offsets = nullptr, *perm = nullptr;
  double* partial = nullptr;
  uint16_t *zhi = nullptr, *zlo = nullptr;  // packed bfloat16 copy of Z (TMA-fed Gram)
  ChunkTable tpc{};                         // its chunk table
  double* G64 = nullptr;
  double *N = nullptr, *cnt = nullptr;
  LanczosWork lw{};
  // resident device buffers
  ChunkTable ct{};
  double* Zg = nullptr;
  float* G32 = nullptr;
  double *c = nullptr, *d = nullptr, *lam = nullptr;
  double* beta_all = nullptr;
  int32_t* it_all = nullptr;
  uint8_t* cv_all = nullptr;
  double *st_u = nullptr, *st_beta = nullptr;
  int32_t* st_ctl = nullptr;
  double *mse = nullptr, *cvm = nullptr, *cvsd = nullptr;
  int32_t *imin = nullptr, *i1se = nullptr, *best = nullptr;
  uint8_t* allowed = nullptr;
  unsigned* status_dev = nullptr;
  // pinned host results
  double* h_beta = nullptr;
  double* h_lam = nullptr;
  double* h_cvm = nullptr;
  double* h_cvsd = nullptr;
  int32_t* h_idx = nullptr;
  int32_t* h_its = nullptr;
  unsigned* h_status = nullptr;
  double* h_d = nullptr;
};

}  // namespace

struct oem_server {
  oem_ctx* ctx = nullptr;
  int device = 0;
  int form = OEM_SERVE_BATCHED;
  int64_t iters_per_round = 2000;
  size_t budget = 0, used = 0, peak = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<SrvJob*> queue;
  std::vector<SrvJob*> live;
  std::map<int64_t, SrvJob*> all;
  int64_t next_id = 1;
  std::thread worker;
  bool stop = false;
  cudaStream_t iter_stream = nullptr;
  IterTask* d_tasks = nullptr;
  int32_t* d_fin = nullptr;
  int32_t* h_fin = nullptr;
  int tasks_cap = 0;
  int64_t jobs_done = 0, paths_done = 0, rounds = 0;
};

namespace {

// Device-memory plan of a job: preparation scratch and resident state.
void plan_job(oem_server* S, SrvJob* J) {
  const oem_job& j = J->spec;
  const int64_t n = j.n, p = j.p;
  const int L = j.nlambda, B = J->B;
  // the Gram pass takes the TMA-fed kernel (and its packed copy of Z, in the
  // job's preparation scratch) on the same terms as a direct call, so a
  // served result equals the direct one
  J->gp = plan_gram(S->ctx, n, p, J->K > 0 ? J->K : 1, J->gram_mode, J->K > 0);
  const GramPlan& g = J->gp;
  J->q = g.q;
  J->ycols = g.ycols;
  J->ldg = (int)((p + 3) & ~3LL);
  Arena& A = J->prep;
  A.req.clear();
  if (g.sorted) {
    A.add(&J->blk_counts, (size_t)g.nblk * g.K);
    A.add(&J->blk_offsets, (size_t)g.nblk * g.K);
    A.add(&J->perm, (size_t)n);
  }
  A.add(&J->partial, (size_t)(g.tma ? g.pmax_chunks : g.max_chunks) * g.ntiles * g.T * g.T);
  if (g.tma) {
    A.add(&J->zhi, (size_t)g.rows_cap * g.qp);
    if (g.mode == OEM_GRAM_SPLIT_BF16) A.add(&J->zlo, (size_t)g.rows_cap * g.qp);
    A.add(&J->tpc.row0, (size_t)g.pmax_chunks);
    A.add(&J->tpc.row1, (size_t)g.pmax_chunks);
    A.add(&J->tpc.fold, (size_t)g.pmax_chunks);
    A.add(&J->tpc.count, 1);
    A.add(&J->tpc.fold_c0, (size_t)g.K + 1);
    A.add(&J->tpc.fold_off, (size_t)g.K + 1);
  }
  A.add(&J->G64, (size_t)B * p * p);
  A.add(&J->N, (size_t)B);
  A.add(&J->cnt, (size_t)B);
  lanczos_request(A, J->lw, p, B, 64);
  Arena& R = J->res;
  R.req.clear();
  R.add(&J->ct.row0, (size_t)g.max_chunks);
  R.add(&J->ct.row1, (size_t)g.max_chunks);
  R.add(&J->ct.fold, (size_t)g.max_chunks);
  R.add(&J->ct.count, 1);
  R.add(&J->ct.fold_c0, (size_t)g.K + 1);
  R.add(&J->ct.fold_off, (size_t)g.K + 1);
  R.add(&J->Zg, (size_t)g.K * g.q * g.q);
  R.add(&J->G32, (size_t)B * p * J->ldg);
  R.add(&J->c, (size_t)B * p);
  R.add(&J->d, (size_t)B);
  R.add(&J->lam, (size_t)L);
  R.add(&J->beta_all, (size_t)B * L * p);
  R.add(&J->it_all, (size_t)B * L);
  R.add(&J->cv_all, (size_t)B * L);
  R.add(&J->st_u, (size_t)B * p * 2);
  R.add(&J->st_beta, (size_t)B * p);
  R.add(&J->st_ctl, (size_t)B * 40);
  R.add(&J->mse, (size_t)(J->K > 0 ? J->K : 1) * L);
  R.add(&J->cvm, (size_t)L);
  R.add(&J->cvsd, (size_t)L);
  R.add(&J->imin, 1);
  R.add(&J->i1se, 1);
  R.add(&J->best, 1);
  R.add(&J->status_dev, 4);
  if (J->groups) R.add(&J->allowed, (size_t)p + 1);
  pens_request(R, J->P);
  J->prep_bytes = A.total();
  J->res_bytes = R.total();
}

int alloc_job(oem_server* S, SrvJob* J) {
  oem_ctx* ctx = S->ctx;
  CU(cudaStreamCreateWithFlags(&J->stream, cudaStreamNonBlocking));
  CU(cudaEventCreateWithFlags(&J->prep_ev, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&J->done_ev, cudaEventDisableTiming));
  CU(cudaMallocAsync(&J->prep_mem, J->prep_bytes, J->stream));
  CU(cudaMallocAsync(&J->res_mem, J->res_bytes, J->stream));
  arena_assign(J->prep, J->prep_mem);
  arena_assign(J->res, J->res_mem);
  const int L = J->spec.nlambda;
  CU(cudaMallocHost(&J->h_beta, sizeof(double) * (size_t)L * J->p));
  CU(cudaMallocHost(&J->h_lam, sizeof(double) * L));
  CU(cudaMallocHost(&J->h_cvm, sizeof(double) * L));
  CU(cudaMallocHost(&J->h_cvsd, sizeof(double) * L));
  CU(cudaMallocHost(&J->h_idx, sizeof(int32_t) * 2));
  CU(cudaMallocHost(&J->h_its, sizeof(int32_t) * (size_t)J->B * L));
  CU(cudaMallocHost(&J->h_status, sizeof(unsigned)));
  CU(cudaMallocHost(&J->h_d, sizeof(double) * J->B));
  return OEM_OK;
}

// Fold sort, Gram pass, fold assembly, d, lambda grid on the job's stream.
int prep_job(oem_server* S, SrvJob* J) {
  oem_ctx* ctx = S->ctx;
  cudaStream_t s = J->stream;
  const oem_job& j = J->spec;
  const int64_t p = j.p;
  unsigned* saved = ctx->dstatus;
  ctx->dstatus = J->status_dev;  // this job's conditions land in its own word
  CU(cudaMemsetAsync(J->status_dev, 0, sizeof(unsigned) * 4, s));
  int r = pens_upload(ctx, J->P, s);
  if (!r && J->groups) {
    std::vector<uint8_t> al(J->P.allowed.begin(), J->P.allowed.end());
    CU(cudaMemcpyAsync(J->allowed, al.data(), al.size(), cudaMemcpyHostToDevice, s));
  }
  GramBufs b;
  b.blk_counts = J->blk_counts;
  b.blk_offsets = J->blk_offsets;
  b.perm = J->perm;
  b.ct = J->ct;
  b.partial = J->partial;
  b.Zg = J->Zg;
  b.zhi = J->zhi;
  b.zlo = J->zlo;
  b.t.pc = J->tpc;
  if (!r) r = run_gram(ctx, J->gp, b, j.X, j.xtype, j.n, p, j.ldx, j.y, j.fold, J->K > 0, s);
  if (!r) {
    const int Kf = J->K > 0 ? J->K : 1;
    LAUNCH(OEM_PROF_ASSEMBLE, launch_assemble(J->Zg, Kf, J->q, (int)p, J->ycols, J->ct.fold_off,
                                              J->K > 0 ? 1 : 0, J->G64, J->G32, J->ldg, J->c, J->N,
                                              J->cnt, s));
    cudaError_t e = lanczos_prof(ctx, s, J->G64, p, p, J->B, p * p, 64, J->lw, J->d, s, &ctx->launches);
    if (e != cudaSuccess) r = fail(ctx, OEM_ECUDA, "Lanczos launch failed: %s", cudaGetErrorString(e));
  }
  if (!r) LAUNCH(OEM_PROF_LAMBDA, launch_lambda_grid(J->c, (int)p, J->P.dpens, 1, j.nlambda,
                                                     j.lambda_min_ratio, J->lam, s));
  if (!r) CU(cudaMemsetAsync(J->st_ctl, 0, sizeof(int32_t) * J->B * 40, s));
  ctx->dstatus = saved;
  if (r) return r;
  CU(cudaEventRecord(J->prep_ev, s));
  return OEM_OK;
}

void release_prep(oem_server* S, SrvJob* J) {
  if (!J->prep_held) return;
  cudaFreeAsync(J->prep_mem, J->stream);
  J->prep_mem = nullptr;
  S->used -= J->prep_bytes;
  J->prep_held = false;
}

// CV scoring and copy-out of the results on the job's stream.
int finish_job(oem_server* S, SrvJob* J) {
  oem_ctx* ctx = S->ctx;
  cudaStream_t s = J->stream;
  const int L = J->spec.nlambda;
  const int64_t p = J->p;
  if (J->K > 0)
    LAUNCH(OEM_PROF_CV, launch_cv_score(J->Zg, J->K, J->q, (int)p, J->ycols, J->ct.fold_off,
                                        J->beta_all, 1, L, J->mse, J->cvm, J->cvsd, J->imin,
                                        J->i1se, J->best, s));
  CU(cudaMemcpyAsync(J->h_beta, J->beta_all, sizeof(double) * L * p, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(J->h_lam, J->lam, sizeof(double) * L, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(J->h_its, J->it_all, sizeof(int32_t) * J->B * L, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(J->h_status, J->status_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  if (J->K > 0) {
    CU(cudaMemcpyAsync(J->h_cvm, J->cvm, sizeof(double) * L, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(J->h_cvsd, J->cvsd, sizeof(double) * L, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(J->h_idx, J->imin, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(J->h_idx + 1, J->i1se, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  }
  CU(cudaEventRecord(J->done_ev, s));
  J->state = OEM_JOB_FINISH;
  return OEM_OK;
}

void complete_job(oem_server* S, SrvJob* J) {
  J->t_done = now_s();
  const unsigned st = *J->h_status;
  if (st & kStatNonFinite) J->status = OEM_ENONFINITE;
  else if (st & kStatEmptyFold) J->status = OEM_EINVAL;
  else if (st & kStatTimeout) J->status = OEM_ETIMEOUT;
  release_prep(S, J);
  cudaFreeAsync(J->res_mem, J->stream);
  J->res_mem = nullptr;
  S->used -= J->res_bytes;
  cudaStreamSynchronize(J->stream);
  cudaStreamDestroy(J->stream);
  J->stream = nullptr;
  J->state = J->status < 0 ? OEM_JOB_FAILED : OEM_JOB_DONE;
  S->jobs_done += 1;
  S->paths_done += J->B;
}

void fail_job(oem_server* S, SrvJob* J, int code) {
  J->status = code;
  J->t_done = now_s();
  if (J->stream) cudaStreamSynchronize(J->stream);
  if (J->prep_held && J->prep_mem) { cudaFree(J->prep_mem); S->used -= J->prep_bytes; J->prep_held = false; }
  if (J->res_mem) { cudaFree(J->res_mem); S->used -= J->res_bytes; J->res_mem = nullptr; }
  J->state = OEM_JOB_FAILED;
}

// One launch of the iteration kernel over the tasks [t0, t0 + T) of the
// round: the jobs in `jobs`, all served by the same kernel (replicated
// row-owned, replicated column-segment, or row-owned for very large p), so
// that a job's arithmetic does not depend on the jobs it shares a round with.
static int launch_class(oem_server* S, const std::vector<SrvJob*>& jobs, int t0, cudaStream_t s) {
  oem_ctx* ctx = S->ctx;
  int T = 0;
  int64_t pmax = 1;
  bool groups = false;
  for (SrvJob* J : jobs) { T += J->B; pmax = std::max(pmax, J->p); groups = groups || J->groups; }
  const bool rows = iter_rows_kernel(pmax);
  // cluster size: all clusters resident at once, about 32 rows per CTA
  int C = 1;
  const int byT = std::max(1, ctx->num_sms / std::max(1, T));
  const int byP = (int)std::min<int64_t>(16, std::max<int64_t>(1, (pmax + 31) / 32));
  while (C * 2 <= std::min(byT, byP) && C < 16) C *= 2;
  std::vector<IterTask> tasks(T);
  std::vector<size_t> fixed(T);
  for (;; C /= 2) {
    size_t smem = 0;
    int t = 0;
    for (SrvJob* J : jobs) {
      for (int b = 0; b < J->B; ++b, ++t) {
        IterTask& k = tasks[t];
        k = IterTask{};
        if (rows) make_slices(J->p, C, J->P.allowed, k.slice, &k.max_rows);
        else make_slices_even(J->p, C, 4, k.slice, &k.max_rows);
        for (int r = C + 1; r <= kMaxCluster; ++r) k.slice[r] = (int32_t)J->p;
        fixed[t] = rows ? oem_iter_rows_smem_fixed((int)J->p, 1, k.max_rows, OEM_ITER_F32)
                        : oem_iter_smem_fixed((int)J->p, 1, k.max_rows, OEM_ITER_F32, false, groups);
        const size_t per = rows ? oem_iter_rows_smem_per_row((int)J->p, OEM_ITER_F32)
                                : oem_iter_smem_per_row((int)J->p, OEM_ITER_F32);
        // row-owned kernel: the column-block cache (all blocks when they fit)
        const size_t want = rows ? fixed[t] + (size_t)oem_iter_rows_blocks((int)J->p) * k.max_rows * 64
                                 : fixed[t] + (size_t)k.max_rows * per;
        smem = std::max(smem, std::min(kIterSmemCap, want));
      }
    }
    smem = std::max<size_t>(smem, 1024);
    int max_rows = 0;
    for (int u = 0; u < T; ++u) max_rows = std::max(max_rows, tasks[u].max_rows);
    IterLaunch probe{};
    probe.ntasks = T; probe.C = C; probe.M = 1; probe.precision = OEM_ITER_F32; probe.smem = smem;
    probe.max_rows = max_rows; probe.groups = groups ? 1 : 0; probe.wide = 0;
    if (iter_smem_probe(probe, rows) >= 1 || C == 1) {
      t = 0;
      for (SrvJob* J : jobs) {
        const int L = J->spec.nlambda;
        for (int b = 0; b < J->B; ++b, ++t) {
          IterTask& k = tasks[t];
          const size_t per = rows ? oem_iter_rows_smem_per_row((int)J->p, OEM_ITER_F32)
                                  : oem_iter_smem_per_row((int)J->p, OEM_ITER_F32);
          k.p = (int)J->p; k.npen = 1; k.L = L; k.ldg = J->ldg;
          k.smem_rows = smem > fixed[t] ? (int)std::min<size_t>(k.max_rows, (smem - fixed[t]) / per) : 0;
          if (rows) {
            k.smem_rows = 0;
            k.ucache = oem_iter_rows_ucache_slots((int)J->p, 1, k.max_rows, OEM_ITER_F32, smem);
          }
          k.resume = J->rounds > 0 ? 1 : 0;
          k.G32 = J->G32 + (size_t)b * J->p * J->ldg;
          k.c = J->c + (size_t)b * J->p;
          k.d = J->d + b;
          k.lam = J->lam;
          k.pens = J->P.dpens;
          k.allowed = J->groups ? J->allowed : nullptr;
          k.beta = J->beta_all + (size_t)b * L * J->p;
          k.iters = J->it_all + (size_t)b * L;
          k.conv = J->cv_all + (size_t)b * L;
          k.st_u = J->st_u + (size_t)b * J->p * 2;
          k.st_beta = J->st_beta + (size_t)b * J->p;
          k.st_ctl = J->st_ctl + (size_t)b * 40;
          k.fin_out = S->d_fin + t0 + t;
        }
      }
      CU(cudaMemcpyAsync(S->d_tasks + t0, tasks.data(), sizeof(IterTask) * T, cudaMemcpyHostToDevice, s));
      IterLaunch Lc{};
      Lc.tasks = S->d_tasks + t0; Lc.ntasks = T; Lc.C = C; Lc.M = 1; Lc.precision = OEM_ITER_F32;
      Lc.tol = jobs[0]->spec.tol;  // per-job tolerance: jobs of one round share it (see submit)
      Lc.max_iter = jobs[0]->spec.max_iter;
      Lc.max_loops = S->iters_per_round;
      Lc.dstatus = ctx->dstatus;
      Lc.smem = smem;
      Lc.max_rows = max_rows;
      Lc.groups = groups ? 1 : 0;
      Lc.wide = 0;
      Lc.wait_cycles = iter_wait_cycles();
      if (rows) LAUNCH(OEM_PROF_ITER, launch_oem_iter_rows(Lc, s));
      else LAUNCH(OEM_PROF_ITER, launch_oem_iter(Lc, s));
      return OEM_OK;
    }
  }
}

// One batched round over every job whose preparation is complete.
int run_round(oem_server* S, std::vector<SrvJob*>& ready) {
  oem_ctx* ctx = S->ctx;
  cudaStream_t s = S->iter_stream;
  int T = 0;
  for (SrvJob* J : ready) T += J->B;
  if (T > S->tasks_cap) {
    if (S->d_tasks) { cudaFree(S->d_tasks); cudaFree(S->d_fin); cudaFreeHost(S->h_fin); }
    S->tasks_cap = std::max(T, 2 * S->tasks_cap);
    CU(cudaMalloc(&S->d_tasks, sizeof(IterTask) * S->tasks_cap));
    CU(cudaMalloc(&S->d_fin, sizeof(int32_t) * S->tasks_cap));
    CU(cudaMallocHost(&S->h_fin, sizeof(int32_t) * S->tasks_cap));
  }
  // the round's jobs by kernel class, in their order within `ready`
  std::vector<SrvJob*> cls[3];
  for (SrvJob* J : ready) cls[iter_rows_kernel(J->p) ? 2 : 0].push_back(J);
  std::vector<SrvJob*> order;
  int t0 = 0;
  for (auto& c : cls) {
    if (c.empty()) continue;
    int r = launch_class(S, c, t0, s);
    if (r) return r;
    for (SrvJob* J : c) { order.push_back(J); t0 += J->B; }
  }
  ready = order;
  CU(cudaMemcpyAsync(S->h_fin, S->d_fin, sizeof(int32_t) * T, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  S->rounds += 1;
  int t = 0;
  for (SrvJob* J : ready) {
    bool fin = true;
    for (int b = 0; b < J->B; ++b, ++t) fin = fin && S->h_fin[t];
    J->rounds += 1;
    if (fin) {
      int r = finish_job(S, J);
      if (r) fail_job(S, J, r);
    }
  }
  return OEM_OK;
}

// The plain per-job form: float32 CUDA-core Gram (prep), then one launch and
// one host convergence check per OEM iteration.
int run_plain(oem_server* S, SrvJob* J) {
  oem_ctx* ctx = S->ctx;
  cudaStream_t s = J->stream;
  const oem_job& j = J->spec;
  const int64_t p = J->p;
  const int L = j.nlambda;
  CU(cudaStreamSynchronize(s));
  CU(cudaMemcpy(J->h_lam, J->lam, sizeof(double) * L, cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(J->h_d, J->d, sizeof(double) * J->B, cudaMemcpyDeviceToHost));
  // two beta vectors and the reduction pair live in the (now unused) Lanczos scratch
  double* bcur = J->lw.V;
  double* bnew = J->lw.V + p;
  unsigned long long* red = (unsigned long long*)J->lw.alpha;
  unsigned long long hred[2];
  std::vector<int32_t> its((size_t)J->B * L, 0);
  for (int b = 0; b < J->B; ++b) {
    CU(cudaMemsetAsync(bcur, 0, sizeof(double) * p, s));
    const float* G = J->G32 + (size_t)b * p * J->ldg;
    const double* c = J->c + (size_t)b * p;
    for (int l = 0; l < L; ++l) {
      int it = 0;
      for (;;) {
        ++it;
        CU(cudaMemsetAsync(red, 0, sizeof(unsigned long long) * 2, s));
        LAUNCH(OEM_PROF_ITER, launch_plain_iter((int)p, G, J->ldg, c, J->h_d[b], bcur, bnew, J->P.dpens,
                                                J->h_lam[l], red, s));
        CU(cudaMemcpyAsync(hred, red, sizeof(hred), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        std::swap(bcur, bnew);
        const double md = __builtin_bit_cast(double, hred[0]);
        const double mb = __builtin_bit_cast(double, hred[1]);
        if (md <= j.tol * std::max(1.0, mb) || it >= j.max_iter) break;
      }
      its[(size_t)b * L + l] = it;
      CU(cudaMemcpyAsync(J->beta_all + ((size_t)b * L + l) * p, bcur, sizeof(double) * p,
                         cudaMemcpyDeviceToDevice, s));
    }
  }
  CU(cudaMemcpyAsync(J->it_all, its.data(), sizeof(int32_t) * its.size(), cudaMemcpyHostToDevice, s));
  return finish_job(S, J);
}

void worker_loop(oem_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<SrvJob*> admitted;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->live.empty() && S->queue.empty()) {
        if (S->stop) return;
        S->cv.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
      // admission in arrival order while the budget allows (the plain form
      // runs one job at a time)
      while (!S->queue.empty()) {
        SrvJob* J = S->queue.front();
        if (S->form == OEM_SERVE_PLAIN && !S->live.empty()) break;
        if (S->used + J->prep_bytes + J->res_bytes > S->budget) break;
        S->queue.pop_front();
        S->used += J->prep_bytes + J->res_bytes;
        S->peak = std::max(S->peak, S->used);
        J->prep_held = true;
        S->live.push_back(J);
        admitted.push_back(J);
      }
    }
    for (SrvJob* J : admitted) {
      int r = alloc_job(S, J);
      if (!r) r = prep_job(S, J);
      std::lock_guard<std::mutex> lk(S->mu);
      if (r) fail_job(S, J, r);
      else J->state = OEM_JOB_PREP;
    }
    std::vector<SrvJob*> ready;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (SrvJob* J : S->live) {
        if (J->state == OEM_JOB_PREP && cudaEventQuery(J->prep_ev) == cudaSuccess) {
          // the plain form keeps its scratch (its iteration vectors live there)
          if (S->form == OEM_SERVE_BATCHED) release_prep(S, J);
          J->state = OEM_JOB_ITER;
        }
        if (J->state == OEM_JOB_ITER) ready.push_back(J);
      }
    }
    if (!ready.empty()) {
      int r = OEM_OK;
      if (S->form == OEM_SERVE_PLAIN) {
        r = run_plain(S, ready[0]);
        if (r) { std::lock_guard<std::mutex> lk(S->mu); fail_job(S, ready[0], r); }
      } else {
        // one tolerance / iteration cap per round: group the ready jobs
        std::vector<SrvJob*> grp;
        for (SrvJob* J : ready)
          if (J->spec.tol == ready[0]->spec.tol && J->spec.max_iter == ready[0]->spec.max_iter)
            grp.push_back(J);
        r = run_round(S, grp);
        if (r) { std::lock_guard<std::mutex> lk(S->mu); for (SrvJob* J : grp) fail_job(S, J, r); }
      }
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      std::vector<SrvJob*> still;
      for (SrvJob* J : S->live) {
        if (J->state == OEM_JOB_FINISH && cudaEventQuery(J->done_ev) == cudaSuccess) complete_job(S, J);
        if (J->state != OEM_JOB_DONE && J->state != OEM_JOB_FAILED) still.push_back(J);
      }
      S->live.swap(still);
    }
    if (ready.empty()) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" {

int oem_server_create(oem_server** out, int device, size_t budget, int32_t form, int64_t iters_per_round) {
  if (!out || (form != OEM_SERVE_BATCHED && form != OEM_SERVE_PLAIN)) return OEM_EINVAL;
  *out = nullptr;
  oem_server* S = new oem_server();
  S->device = device;
  S->form = form;
  S->budget = budget ? budget : ((size_t)8 << 30);
  S->iters_per_round = iters_per_round > 0 ? iters_per_round : 2000;
  int r = oem_create(&S->ctx, device, S->budget);
  if (r) { delete S; return r; }
  if (cudaStreamCreateWithFlags(&S->iter_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    oem_destroy(S->ctx);
    delete S;
    return OEM_ECUDA;
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return OEM_OK;
}

int oem_server_submit(oem_server* S, const oem_job* job, int64_t* id) {
  if (!S || !job || !id) return OEM_EINVAL;
  oem_ctx* ctx = S->ctx;
  SrvJob* J = new SrvJob();
  J->spec = *job;
  const oem_job& j = J->spec;
  int r = check_x(ctx, j.X, j.xtype, j.n, j.p, j.ldx, j.y);
  if (!r && !(j.K == 0 || (j.K >= 2 && j.K <= 64))) r = fail(ctx, OEM_EINVAL, "K=%d", j.K);
  if (!r && j.K > 0 && !j.fold) r = fail(ctx, OEM_EINVAL, "CV job without fold labels");
  if (!r && (j.nlambda < 1 || j.nlambda > 100000 || !(j.tol > 0.0) || j.max_iter < 1 ||
             !(j.lambda_min_ratio > 0.0 && j.lambda_min_ratio <= 1.0)))
    r = fail(ctx, OEM_EINVAL, "bad nlambda / tol / max_iter / lambda_min_ratio");
  if (!r && j.p > 4096) r = fail(ctx, OEM_EUNSUPPORTED, "p=%lld exceeds 4096 for serving", (long long)j.p);
  if (!r) r = prepare_pens(ctx, &j.pen, 1, j.p, J->P);
  if (!r) {
    J->groups = j.pen.kind >= OEM_GROUP_LASSO;
    if (S->form == OEM_SERVE_PLAIN && J->groups)
      r = fail(ctx, OEM_EUNSUPPORTED, "the plain form serves lasso, elastic net, MCP and SCAD");
  }
  int32_t mode = OEM_GRAM_FP32;
  if (!r && S->form == OEM_SERVE_BATCHED) r = resolve_mode(ctx, j.gram_mode, j.xtype, &mode);
  if (!r && S->form == OEM_SERVE_PLAIN && j.xtype == OEM_F64) mode = OEM_GRAM_FP64;
  if (r) { delete J; return r; }
  J->gram_mode = mode;
  J->K = j.K;
  J->B = j.K > 0 ? j.K + 1 : 1;
  J->L = j.nlambda;
  J->p = j.p;
  plan_job(S, J);
  if (J->prep_bytes + J->res_bytes > S->budget) {
    r = fail(ctx, OEM_EBUDGET, "job needs %zu bytes, budget %zu", J->prep_bytes + J->res_bytes, S->budget);
    delete J;
    return r;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  J->id = S->next_id++;
  J->t_submit = now_s();
  S->all[J->id] = J;
  S->queue.push_back(J);
  *id = J->id;
  S->cv.notify_one();
  return OEM_OK;
}

int oem_server_poll(oem_server* S, int64_t id, int32_t* state, double* latency_ms) {
  if (!S) return OEM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return OEM_EINVAL;
  SrvJob* J = it->second;
  if (state) *state = J->state;
  if (latency_ms) *latency_ms = (J->state == OEM_JOB_DONE || J->state == OEM_JOB_FAILED)
                                    ? 1000.0 * (J->t_done - J->t_submit) : -1.0;
  return J->state == OEM_JOB_FAILED ? J->status : OEM_OK;
}

int oem_server_result(oem_server* S, int64_t id, double* beta, double* lambdas, double* cvm,
                      double* cvsd, int32_t* idx_min, int32_t* idx_1se, int64_t* iters) {
  if (!S) return OEM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end() || it->second->state != OEM_JOB_DONE) return OEM_EINVAL;
  SrvJob* J = it->second;
  const int L = J->spec.nlambda;
  if (beta) std::memcpy(beta, J->h_beta, sizeof(double) * L * J->p);
  if (lambdas) std::memcpy(lambdas, J->h_lam, sizeof(double) * L);
  if (J->K > 0) {
    if (cvm) std::memcpy(cvm, J->h_cvm, sizeof(double) * L);
    if (cvsd) std::memcpy(cvsd, J->h_cvsd, sizeof(double) * L);
    if (idx_min) *idx_min = J->h_idx[0];
    if (idx_1se) *idx_1se = J->h_idx[1];
  }
  if (iters) {
    int64_t t = 0;
    for (int i = 0; i < J->B * L; ++i) t += J->h_its[i];
    *iters = t;
  }
  return OEM_OK;
}

int oem_server_stats(oem_server* S, int64_t* jobs_done, int64_t* paths_done, int64_t* launches,
                     int64_t* rounds, int64_t* peak_bytes) {
  if (!S) return OEM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (jobs_done) *jobs_done = S->jobs_done;
  if (paths_done) *paths_done = S->paths_done;
  if (launches) *launches = S->ctx->launches;
  if (rounds) *rounds = S->rounds;
  if (peak_bytes) *peak_bytes = (int64_t)S->peak;
  return OEM_OK;
}

int oem_server_destroy(oem_server* S) {
  if (!S) return OEM_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_one();
  }
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  cudaDeviceSynchronize();
  for (auto& kv : S->all) {
    SrvJob* J = kv.second;
    cudaFreeHost(J->h_beta); cudaFreeHost(J->h_lam); cudaFreeHost(J->h_cvm); cudaFreeHost(J->h_cvsd);
    cudaFreeHost(J->h_idx); cudaFreeHost(J->h_its); cudaFreeHost(J->h_status); cudaFreeHost(J->h_d);
    if (J->prep_ev) cudaEventDestroy(J->prep_ev);
    if (J->done_ev) cudaEventDestroy(J->done_ev);
    delete J;
  }
  if (S->d_tasks) { cudaFree(S->d_tasks); cudaFree(S->d_fin); cudaFreeHost(S->h_fin); }
  cudaStreamDestroy(S->iter_stream);
  oem_destroy(S->ctx);
  delete S;
  return OEM_OK;
}

}  // extern "C"
