// Penalised logistic regression (Section 4): the proximal Newton algorithm
// with the Hessian weights replaced by their upper bound 1/4, so that every
// surrogate has the same G = Z^T Z / (4n) (Z = [X | 1] with an intercept) and
// only its linear term moves: c_t = G beta_t + Z^T (y - mu(beta_t)) / n. The
// Gram pass and the OEM iteration kernel are shared with the linear model;
// this file holds the per-outer-step kernels:
//   logit_grad_kernel — one pass over X: for every penalty's current beta,
//     eta_i = z_i^T beta, r_i = y_i - sigmoid(eta_i), and the per-CTA partial
//     sums of z_i r_i (float32 chunk sums folded into TwoSum pairs);
//   logit_grad_reduce_kernel — the partials summed in CTA order: g = Z^T r / n;
//   logit_state_kernel — the iteration kernel's resume state for the surrogate
//     at beta_t: u = c_t + d beta_t - G beta_t = g + d_eff beta_t;
//   logit_step_kernel — the outer step's change, the stopping rule, the
//     accepted iterate (penalties whose outer loop has stopped keep theirs).
#include "oem_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace oem {

namespace {

__device__ __forceinline__ float2 lg_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}
}  // namespace

// 16-byte global -> shared copy, asynchronous (float32 X rows)
__device__ __forceinline__ void lg_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

// grid: persistent CTAs; each takes chunks of RC rows. Float32 X streams
// into a double-buffered shared-memory chunk by cp.async (the next chunk's
// copies in flight while this one is used; other types by plain loads).
// A warp per row forms eta = z^T beta for every penalty (float32 FMAs: the
// sigmoid needs ~1e-7) and r = y - sigmoid(eta); a thread per column adds
// r z over the chunk's rows in float32 (RC terms) and folds that chunk sum
// into a TwoSum (hi, lo) pair, so the CTA's partial of the score carries no
// drift over the many chunks it takes.
constexpr int kLgThreads = 512;

template <int NPEN>
__global__ void __launch_bounds__(kLgThreads) logit_grad_kernel(LogitArgs a) {
  extern __shared__ __align__(16) unsigned char lg_smem[];
  const int p = (int)a.p;
  const int pq = p + (a.intercept ? 1 : 0);  // coefficients incl. the intercept
  const int lds = (p + 3) & ~3;              // row stride in shared memory
  float* Xbuf = reinterpret_cast<float*>(lg_smem);                     // [2][RC][lds]
  float* Bs = Xbuf + (size_t)2 * a.rc * lds;                           // [NPEN][lds]
  float* Rs = Bs + (size_t)NPEN * lds;                                 // [RC][NPEN]
  float* B0 = Rs + (size_t)a.rc * NPEN;                                // [NPEN] intercepts
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < NPEN * lds; e += blockDim.x) {
    const int k = e / lds, c = e % lds;
    Bs[e] = c < p ? (float)a.beta[(size_t)k * a.ldb + c] : 0.f;
  }
  if (threadIdx.x < NPEN) B0[threadIdx.x] = a.intercept ? (float)a.beta[(size_t)threadIdx.x * a.ldb + p] : 0.f;
  // column accumulators: thread owns columns tid and tid + 512
  float ah[2][NPEN], al[2][NPEN];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < NPEN; ++k) { ah[q][k] = 0.f; al[q][k] = 0.f; }
  const bool f32 = a.xtype == OEM_F32;
  const int nq = lds / 4;  // float4 per row (the row stride of X is a multiple of 16 bytes)
  const int64_t nchunks = (a.n + a.rc - 1) / a.rc;
  // float32: issue the copies of chunk ch into buffer buf
  auto issue = [&](int64_t ch, int buf) {
    if (ch >= nchunks) return;
    const int64_t r0 = ch * a.rc;
    const int rows = (int)min((int64_t)a.rc, a.n - r0);
    float* xs = Xbuf + (size_t)buf * a.rc * lds;
    for (int e = threadIdx.x; e < rows * nq; e += blockDim.x) {
      const int rr = e / nq, j = (e - rr * nq) * 4;
      lg_cp16(xs + (size_t)rr * lds + j, (const float*)a.X + (r0 + rr) * a.ldx + j);
    }
  };
  if (f32) issue(blockIdx.x, 0);
  asm volatile("cp.async.commit_group;" ::: "memory");
  int buf = 0;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x, buf ^= 1) {
    const int64_t r0 = ch * a.rc;
    const int rows = (int)min((int64_t)a.rc, a.n - r0);
    float* Xs = Xbuf + (size_t)buf * a.rc * lds;
    if (f32) {
      issue(ch + gridDim.x, buf ^ 1);
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      for (int e = threadIdx.x; e < rows * lds; e += blockDim.x) {
        const int rr = e / lds, c = e - rr * lds;
        const int64_t o = (r0 + rr) * a.ldx + c;
        float v = 0.f;
        if (c < p) v = a.xtype == OEM_BF16 ? __bfloat162float(((const __nv_bfloat16*)a.X)[o])
                                           : (float)((const double*)a.X)[o];
        Xs[(size_t)rr * lds + c] = v;
      }
    }
    __syncthreads();
    // ---- a warp per row: eta, r
    for (int rr = warp; rr < rows; rr += kLgThreads / 32) {
      const float* xs = Xs + (size_t)rr * lds;
      float eta[NPEN];
#pragma unroll
      for (int k = 0; k < NPEN; ++k) eta[k] = 0.f;
      for (int j4 = lane * 4; j4 < p; j4 += 128) {
        const float4 v = *reinterpret_cast<const float4*>(xs + j4);
#pragma unroll
        for (int k = 0; k < NPEN; ++k) {
          const float4 b4 = *reinterpret_cast<const float4*>(Bs + (size_t)k * lds + j4);
          eta[k] = fmaf(v.x, b4.x, fmaf(v.y, b4.y, fmaf(v.z, b4.z, fmaf(v.w, b4.w, eta[k]))));
        }
      }
#pragma unroll
      for (int k = 0; k < NPEN; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) eta[k] += __shfl_xor_sync(0xffffffffu, eta[k], o);
      if (lane < NPEN) {
        float e = eta[0];
#pragma unroll
        for (int k = 1; k < NPEN; ++k)
          if (lane == k) e = eta[k];
        e += B0[lane];
        const float yv = a.ytype == OEM_F64 ? (float)((const double*)a.y)[r0 + rr] : ((const float*)a.y)[r0 + rr];
        // sigmoid, stable for either sign of eta
        const float t = __expf(-fabsf(e));
        const float mu = e >= 0.f ? 1.f / (1.f + t) : t / (1.f + t);
        Rs[rr * NPEN + lane] = yv - mu;
      }
    }
    __syncthreads();
    // ---- column sums of z_i r_i over the chunk's rows
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = threadIdx.x + q * kLgThreads;
      if (c >= pq) break;
      float acc[2][NPEN];  // even / odd rows: two independent chains
#pragma unroll
      for (int k = 0; k < NPEN; ++k) { acc[0][k] = 0.f; acc[1][k] = 0.f; }
      int rr = 0;
      for (; rr + 1 < rows; rr += 2) {
        const float x0 = c < p ? Xs[(size_t)rr * lds + c] : 1.f;
        const float x1 = c < p ? Xs[(size_t)(rr + 1) * lds + c] : 1.f;
#pragma unroll
        for (int k = 0; k < NPEN; ++k) {
          acc[0][k] = fmaf(Rs[rr * NPEN + k], x0, acc[0][k]);
          acc[1][k] = fmaf(Rs[(rr + 1) * NPEN + k], x1, acc[1][k]);
        }
      }
      if (rr < rows) {
        const float x0 = c < p ? Xs[(size_t)rr * lds + c] : 1.f;
#pragma unroll
        for (int k = 0; k < NPEN; ++k) acc[0][k] = fmaf(Rs[rr * NPEN + k], x0, acc[0][k]);
      }
#pragma unroll
      for (int k = 0; k < NPEN; ++k) {
        const float2 s2 = lg_two_sum(ah[q][k], acc[0][k] + acc[1][k]);
        ah[q][k] = s2.x;
        al[q][k] += s2.y;
      }
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // ---- this CTA's partial sums
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int c = threadIdx.x + q * kLgThreads;
    if (c >= pq) break;
#pragma unroll
    for (int k = 0; k < NPEN; ++k)
      a.part[((size_t)blockIdx.x * NPEN + k) * pq + c] = lg_two_sum(ah[q][k], al[q][k]);
  }
}

// g[k][c] = (sum over CTAs of the partials, in CTA order) / n, float64.
__global__ void logit_grad_reduce_kernel(const float2* __restrict__ part, int nparts, int npen, int pq,
                                         int64_t n, double* __restrict__ g, int ldb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npen * pq) return;
  const int k = e / pq, c = e % pq;
  float h = 0.f, l = 0.f;
  for (int b = 0; b < nparts; ++b) {
    const float2 v = part[((size_t)b * npen + k) * pq + c];
    const float2 s = lg_two_sum(h, v.x);
    h = s.x;
    l += s.y + v.y;
  }
  g[(size_t)k * ldb + c] = ((double)h + (double)l) / (double)n;
}

// Resume state of the iteration kernel for the surrogate at beta:
// u = g + d_eff beta (float32 iteration: (hi, lo) split of u).
__global__ void logit_state_kernel(const double* __restrict__ g, const double* __restrict__ beta,
                                   int npen, int pq, int ldb, const double* __restrict__ d,
                                   const DevPenalty* __restrict__ pens, int precision,
                                   double* st_u, double* st_beta, int32_t* st_ctl, int nctl) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nctl) st_ctl[e] = 0;
  if (e >= npen * pq) return;
  const int k = e / pq, c = e % pq;
  const DevPenalty& pen = pens[k];
  double de = d[0];
  if (pen.kind == OEM_MCP) de = fmax(de, 1.01 / pen.gamma64);
  if (pen.kind == OEM_SCAD) de = fmax(de, 1.01 / (pen.gamma64 - 1.0));
  const double b = beta[(size_t)k * ldb + c];
  const double u = g[(size_t)k * ldb + c] + de * b;
  const size_t o = (size_t)k * pq + c;
  if (precision == OEM_ITER_F32) {
    const double hi = (double)(float)u;
    st_u[2 * o] = hi;
    st_u[2 * o + 1] = (double)(float)(u - hi);
  } else {
    st_u[2 * o] = u;
    st_u[2 * o + 1] = 0.0;
  }
  st_beta[o] = b;
}

// One block per penalty: delta = max |new - beta|, the stopping rule, the
// accepted iterate and the iteration count. flags[k]: 1 = this outer loop
// has stopped (converged or reached the cap).
__global__ void logit_step_kernel(double* __restrict__ beta, const double* __restrict__ bnew, int pq,
                                  int ldb, const int32_t* __restrict__ it_new, int32_t* __restrict__ its,
                                  double tol, int32_t* __restrict__ flags, int last_outer,
                                  uint8_t* __restrict__ conv) {
  __shared__ double rd[2][8];
  const int k = blockIdx.x;
  if (flags[k]) return;  // stopped earlier: keeps its iterate
  double dmax = 0.0, bmax = 0.0;
  for (int c = threadIdx.x; c < pq; c += blockDim.x) {
    const double v = bnew[(size_t)k * pq + c];
    dmax = fmax(dmax, fabs(v - beta[(size_t)k * ldb + c]));
    bmax = fmax(bmax, fabs(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { rd[0][w] = dmax; rd[1][w] = bmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) { dmax = fmax(dmax, rd[0][i]); bmax = fmax(bmax, rd[1][i]); }
    rd[0][0] = dmax;
    rd[1][0] = bmax;
  }
  __syncthreads();
  const bool done = rd[0][0] <= tol * fmax(1.0, rd[1][0]);
  for (int c = threadIdx.x; c < pq; c += blockDim.x) beta[(size_t)k * ldb + c] = bnew[(size_t)k * pq + c];
  if (threadIdx.x == 0) {
    its[k] += it_new[k];
    if (done || last_outer) {
      flags[k] = 1;
      conv[k] = done ? 1 : 0;
    }
  }
}

// Null model: beta = 0, intercept logit(ybar), ybar = y^T 1 / n from the
// Gram of Z = [X | y | 1] (y in ycols pieces at columns p.., ones at ocol).
__global__ void logit_null_kernel(double* beta, int npen, int pq, int ldb, int intercept,
                                  const double* __restrict__ Zg, int q, int p, int ycols, int ocol,
                                  int64_t n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npen * pq) return;
  const int k = e / pq, c = e % pq;
  double v = 0.0;
  if (intercept && c == pq - 1) {
    double ys = 0.0;
    for (int t = 0; t < ycols; ++t) ys += Zg[(int64_t)(p + t) * q + ocol];
    const double yb = fmin(fmax(ys / (double)n, 1e-12), 1.0 - 1e-12);
    v = log(yb / (1.0 - yb));
  }
  beta[(size_t)k * ldb + c] = v;
}

// G = Z^T Z / (4n), Z = [X | 1] (intercept) from the Gram of [X | y | 1]:
// float64 [pq][pq] and float32 [pq][ldg] (zero padding columns).
__global__ void logit_gram_kernel(const double* __restrict__ Zg, int q, int p, int ocol, int intercept,
                                  int64_t n, double* G64, float* G32, int ldg) {
  const int pq = p + (intercept ? 1 : 0);
  const double sc = 0.25 / (double)n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)pq * ldg;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ldg), j = (int)(e % ldg);
    if (j >= pq) {
      if (G32) G32[e] = 0.f;
      continue;
    }
    const int ci = i < p ? i : ocol, cj = j < p ? j : ocol;
    const double v = Zg[(int64_t)ci * q + cj] * sc;
    if (G64) G64[(int64_t)i * pq + j] = v;
    if (G32) G32[e] = (float)v;
  }
}

cudaError_t launch_logit_grad(const LogitArgs& a, int npen, int grid, cudaStream_t s) {
  const int pq = (int)a.p + (a.intercept ? 1 : 0);
  const size_t smem = logit_grad_smem(a.p, a.rc, npen, a.intercept);
  cudaError_t e = cudaSuccess;
  switch (npen) {
#define OEM_LG(N)                                                                                 \
  case N:                                                                                         \
    e = cudaFuncSetAttribute(logit_grad_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                             (int)smem);                                                          \
    if (e != cudaSuccess) return e;                                                               \
    logit_grad_kernel<N><<<grid, kLgThreads, smem, s>>>(a);                                              \
    break;
    OEM_LG(1) OEM_LG(2) OEM_LG(3) OEM_LG(4) OEM_LG(5) OEM_LG(6) OEM_LG(7) OEM_LG(8)
#undef OEM_LG
    default: return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int tot = npen * pq;
  logit_grad_reduce_kernel<<<(tot + 255) / 256, 256, 0, s>>>(a.part, grid, npen, pq, a.n, a.g, a.ldb);
  return cudaGetLastError();
}

size_t logit_grad_smem(int64_t p, int rc, int npen, int intercept) {
  (void)intercept;
  const size_t lds = (size_t)((p + 3) & ~3LL);
  return sizeof(float) * ((size_t)2 * rc * lds + (size_t)npen * lds + (size_t)rc * npen + (size_t)npen) + 64;
}

cudaError_t launch_logit_state(const double* g, const double* beta, int npen, int pq, int ldb,
                               const double* d, const DevPenalty* pens, int precision, double* st_u,
                               double* st_beta, int32_t* st_ctl, int nctl, cudaStream_t s) {
  const int tot = std::max(npen * pq, nctl);
  logit_state_kernel<<<(tot + 255) / 256, 256, 0, s>>>(g, beta, npen, pq, ldb, d, pens, precision, st_u,
                                                       st_beta, st_ctl, nctl);
  return cudaGetLastError();
}

cudaError_t launch_logit_step(double* beta, const double* bnew, int npen, int pq, int ldb,
                              const int32_t* it_new, int32_t* its, double tol, int32_t* flags,
                              int last_outer, uint8_t* conv, cudaStream_t s) {
  logit_step_kernel<<<npen, 256, 0, s>>>(beta, bnew, pq, ldb, it_new, its, tol, flags, last_outer, conv);
  return cudaGetLastError();
}

cudaError_t launch_logit_null(double* beta, int npen, int pq, int ldb, int intercept, const double* Zg,
                              int q, int p, int ycols, int ocol, int64_t n, cudaStream_t s) {
  const int tot = npen * pq;
  logit_null_kernel<<<(tot + 255) / 256, 256, 0, s>>>(beta, npen, pq, ldb, intercept, Zg, q, p, ycols, ocol, n);
  return cudaGetLastError();
}

cudaError_t launch_logit_gram(const double* Zg, int q, int p, int ocol, int intercept, int64_t n,
                              double* G64, float* G32, int ldg, cudaStream_t s) {
  const int pq = p + (intercept ? 1 : 0);
  const int64_t tot = (int64_t)pq * ldg;
  const unsigned gx = (unsigned)std::min<int64_t>(2048, (tot + 255) / 256);
  logit_gram_kernel<<<gx, 256, 0, s>>>(Zg, q, p, ocol, intercept, n, G64, G32, ldg);
  return cudaGetLastError();
}

}  // namespace oem
