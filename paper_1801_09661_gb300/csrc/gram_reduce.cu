// Fold assembly (Section 3): reduce the Gram pass's chunk partials into
// per-fold raw sums of Z^T Z (float64), then form the full-data statistics
// X^T X / n, X^T y / n, y^T y / n and the leave-fold-out statistics by the
// paper's identity X_{-k}^T X_{-k} = sum_{c != k} X_c^T X_c.
#include "oem_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace oem {

__global__ void gram_reduce_kernel(GramArgs a, int K, double* __restrict__ Zg) {
  const int T = a.T, TT = T * T;
  const int k = blockIdx.y;
  const int64_t e_all = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int tile = (int)(e_all / TT), e = (int)(e_all % TT);
  if (tile >= a.ntiles) return;
  int ti, tj;
  tile_coords(tile, a.ntile1, &ti, &tj);
  const int r = ti * T + e / T, c = tj * T + e % T;
  if (r >= a.q || c >= a.q || (ti == tj && c < r)) return;
  const int c0 = a.ct.fold_c0[k], c1 = a.ct.fold_c0[k + 1];
  double s = 0.0;
  for (int ch = c0; ch < c1; ++ch) s += a.partial[((int64_t)ch * a.ntiles + tile) * TT + e];
  if (!isfinite(s)) atomicOr(a.dstatus, kStatNonFinite);
  double* Z = Zg + (int64_t)k * a.q * a.q;
  Z[(int64_t)r * a.q + c] = s;
  Z[(int64_t)c * a.q + r] = s;
}

cudaError_t launch_gram_reduce(const GramArgs& a, int K, double* Zg, cudaStream_t s) {
  const int64_t total = (int64_t)a.ntiles * a.T * a.T;
  dim3 grid((unsigned)((total + 255) / 256), (unsigned)K);
  gram_reduce_kernel<<<grid, 256, 0, s>>>(a, K, Zg);
  return cudaGetLastError();
}

// X^T y and y^T y from the y column(s): when y is carried as pieces
// y = y_0 + y_1 + ... (columns p, p+1, ...), X^T y = sum_s X^T y_s and
// y^T y = sum_{s,t} y_s^T y_t.
__device__ __forceinline__ double zc(const double* Z, int q, int p, int ycols, int i) {
  double v = 0.0;
  for (int s = 0; s < ycols; ++s) v += Z[(int64_t)i * q + p + s];
  return v;
}
__device__ __forceinline__ double zn(const double* Z, int q, int p, int ycols) {
  double v = 0.0;
  for (int s = 0; s < ycols; ++s)
    for (int t = 0; t < ycols; ++t) v += Z[(int64_t)(p + s) * q + p + t];
  return v;
}

__global__ void extract_folds_kernel(const double* __restrict__ Zg, int K, int q, int p, int ycols,
                                     double* Gk, double* ck, double* ytyk, int64_t* nk,
                                     const int64_t* fold_off) {
  const int k = blockIdx.y;
  const double* Z = Zg + (int64_t)k * q * q;
  const int64_t pp = (int64_t)p * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < pp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / p), j = (int)(e % p);
    Gk[(int64_t)k * pp + e] = Z[(int64_t)i * q + j];
    if (j == 0) ck[(int64_t)k * p + i] = zc(Z, q, p, ycols, i);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ytyk[k] = zn(Z, q, p, ycols);
    nk[k] = fold_off[k + 1] - fold_off[k];
  }
}

cudaError_t launch_extract_folds(const double* Zg, int K, int q, int p, int ycols, double* Gk,
                                 double* ck, double* ytyk, int64_t* nk, const int64_t* fold_off,
                                 cudaStream_t s) {
  int64_t pp = (int64_t)p * p;
  unsigned gx = (unsigned)((pp + 255) / 256);
  if (gx > 1024) gx = 1024;
  extract_folds_kernel<<<dim3(gx, K), 256, 0, s>>>(Zg, K, q, p, ycols, Gk, ck, ytyk, nk, fold_off);
  return cudaGetLastError();
}

// Sum over the folds of one entry of the fold Grams of Z, less fold b-1
// (b > 0: the leave-fold-out set).
__device__ __forceinline__ double fold_sum(const double* Zg, int K, int64_t qq, int b, int64_t o) {
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += Zg[k * qq + o];
  if (b > 0) s -= Zg[(b - 1) * qq + o];
  return s;
}
__device__ __forceinline__ double fold_sum_c(const double* Zg, int K, int64_t qq, int b, int q, int p,
                                             int ycols, int i) {
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += zc(Zg + k * qq, q, p, ycols, i);
  if (b > 0) s -= zc(Zg + (b - 1) * qq, q, p, ycols, i);
  return s;
}
__device__ __forceinline__ double fold_sum_n(const double* Zg, int K, int64_t qq, int b, int q, int p,
                                             int ycols) {
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += zn(Zg + k * qq, q, p, ycols);
  if (b > 0) s -= zn(Zg + (b - 1) * qq, q, p, ycols);
  return s;
}

// Centring and scale of column i of fit b (from the raw sums of the shifted
// Z): mean mu_i (0 without an intercept), variance var_i, sd_i and whether
// the column is constant (variance zero or below 1e-14 of its second moment;
// it then keeps scale 1 and drops out).
struct ColStat {
  double mu, sd;
  bool konst;
};
__device__ __forceinline__ ColStat col_stat(const double* Zg, int K, int64_t qq, int b, int q, int i,
                                            double inv, const CentreArgs& ce) {
  ColStat r;
  const double sxx = fold_sum(Zg, K, qq, b, (int64_t)i * q + i) * inv;
  r.mu = ce.intercept ? fold_sum(Zg, K, qq, b, (int64_t)i * q + ce.ocol) * inv : 0.0;
  const double var = sxx - r.mu * r.mu;
  r.konst = !(var > 1e-14 * sxx);
  r.sd = (ce.standardize && !r.konst) ? sqrt(var) : 1.0;
  return r;
}

// b = 0: full data / n; b = k+1: (sum - fold k) / (n - n_k). With centring
// (Section 2.1's standardized design; the intercept / standardize options):
// G = D (S_xx / n_b - mu mu^T) D, c = D (S_xy / n_b - mu ybar),
// N = S_yy / n_b - ybar^2, D = diag(1 / sd), constant columns zeroed; the
// means, scales and ybar go to ce.cen.
__global__ void assemble_kernel(const double* __restrict__ Zg, int K, int q, int p, int ycols,
                                const int64_t* __restrict__ fold_off, int B, double* G64,
                                float* G32, int ldg32, double* c, double* N, double* cnt,
                                CentreArgs ce) {
  const int b = blockIdx.y;
  const int64_t n = fold_off[K] - fold_off[0];
  const int64_t nb = (b == 0) ? n : n - (fold_off[b] - fold_off[b - 1]);
  const double inv = nb > 0 ? 1.0 / (double)nb : 0.0;
  const int64_t pp = (int64_t)p * p, qq = (int64_t)q * q;
  const bool centre = ce.intercept || ce.standardize;
  double ybar = 0.0;
  if (ce.intercept) {
    double t = 0.0;
    for (int s2 = 0; s2 < ycols; ++s2) t += fold_sum(Zg, K, qq, b, (int64_t)(p + s2) * q + ce.ocol);
    ybar = t * inv;
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < pp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / p), j = (int)(e % p);
    const int64_t o = (int64_t)i * q + j;
    double v;
    if (!centre) {
      v = fold_sum(Zg, K, qq, b, o) * inv;
    } else {
      const ColStat si = col_stat(Zg, K, qq, b, q, i, inv, ce);
      const ColStat sj = (i == j) ? si : col_stat(Zg, K, qq, b, q, j, inv, ce);
      v = (si.konst || sj.konst) ? 0.0
                                 : (fold_sum(Zg, K, qq, b, o) * inv - si.mu * sj.mu) / (si.sd * sj.sd);
    }
    if (G64) G64[b * pp + e] = v;
    if (G32) {
      float* row = G32 + (int64_t)b * p * ldg32 + (int64_t)i * ldg32;
      row[j] = (float)v;
      if (j == p - 1)  // zero the padding columns of the float32 copy
        for (int jj = p; jj < ldg32; ++jj) row[jj] = 0.f;
    }
    if (j == 0) {
      const double sc = fold_sum_c(Zg, K, qq, b, q, p, ycols, i) * inv;
      if (!centre) {
        c[(int64_t)b * p + i] = sc;
      } else {
        const ColStat si = col_stat(Zg, K, qq, b, q, i, inv, ce);
        c[(int64_t)b * p + i] = si.konst ? 0.0 : (sc - si.mu * ybar) / si.sd;
        double* cb = ce.cen + (int64_t)b * (2 * p + 1);
        cb[i] = si.mu;
        cb[p + i] = si.sd;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    N[b] = fold_sum_n(Zg, K, qq, b, q, p, ycols) * inv - ybar * ybar;
    cnt[b] = (double)nb;
    if (centre) ce.cen[(int64_t)b * (2 * p + 1) + 2 * p] = ybar;
  }
}

cudaError_t launch_assemble(const double* Zg, int K, int q, int p, int ycols,
                            const int64_t* fold_off, int with_leave_out, double* G64, float* G32,
                            int ldg32, double* c, double* N, double* cnt, cudaStream_t s,
                            const CentreArgs& ce) {
  const int B = with_leave_out ? K + 1 : 1;
  int64_t pp = (int64_t)p * p;
  unsigned gx = (unsigned)((pp + 255) / 256);
  if (gx > 2048) gx = 2048;
  assemble_kernel<<<dim3(gx, B), 256, 0, s>>>(Zg, K, q, p, ycols, fold_off, B, G64, G32, ldg32,
                                              c, N, cnt, ce);
  return cudaGetLastError();
}

// Streamed Gram pass (X in host memory, row blocks): acc += blk over the
// fold Grams of Z, and the fold row counts from the block's sorted offsets.
__global__ void zg_accumulate_kernel(double* __restrict__ acc, const double* __restrict__ blk, int64_t len,
                                     int first, int64_t* __restrict__ cnt,
                                     const int64_t* __restrict__ fold_off, int K) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x)
    acc[e] = first ? blk[e] : acc[e] + blk[e];
  if (blockIdx.x == 0 && threadIdx.x < K) {
    const int64_t c = fold_off[threadIdx.x + 1] - fold_off[threadIdx.x];
    cnt[threadIdx.x] = first ? c : cnt[threadIdx.x] + c;
  }
}

// Offsets of the accumulated folds (the layout the assembly reads:
// off[k+1] - off[k] = rows of fold k); flags an empty fold when asked.
__global__ void zg_offsets_kernel(const int64_t* __restrict__ cnt, int64_t* off, int K, int require_nonempty,
                                  unsigned* dstatus) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  off[0] = 0;
  for (int k = 0; k < K; ++k) {
    off[k + 1] = off[k] + cnt[k];
    if (cnt[k] == 0 && require_nonempty) atomicOr(dstatus, kStatEmptyFold);
  }
}

cudaError_t launch_zg_accumulate(double* acc, const double* blk, int64_t len, int first, int64_t* cnt,
                                 const int64_t* fold_off, int K, cudaStream_t s) {
  const unsigned gx = (unsigned)std::min<int64_t>(1024, (len + 255) / 256);
  zg_accumulate_kernel<<<gx, 256, 0, s>>>(acc, blk, len, first, cnt, fold_off, K);
  return cudaGetLastError();
}

cudaError_t launch_zg_offsets(const int64_t* cnt, int64_t* off, int K, int require_nonempty, unsigned* dstatus,
                              cudaStream_t s) {
  zg_offsets_kernel<<<1, 32, 0, s>>>(cnt, off, K, require_nonempty, dstatus);
  return cudaGetLastError();
}

// Column shifts: lane = column within a group of 32, warp = a stride of the
// sampled rows; float32 sums, min and max per column. A column whose sampled
// values are all equal gets that value exactly (its shifted copy is zero).
__global__ void col_shift_kernel(const void* __restrict__ X, int32_t xtype, int64_t n, int64_t p,
                                 int64_t ldx, const void* __restrict__ y, float* shift) {
  __shared__ float ssum[8][33], smin[8][33], smax[8][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * 32 + lane;
  const int64_t S = n < 8192 ? n : 8192;
  float sum = 0.f, mn = 3.4e38f, mx = -3.4e38f;
  if (col <= p) {
    for (int64_t i = warp; i < S; i += 8) {
      const int64_t row = (S == n) ? i : (i * n) / S;
      float v;
      if (col < p) {
        const int64_t o = row * ldx + col;
        v = xtype == OEM_F64 ? (float)((const double*)X)[o]
            : xtype == OEM_F32 ? ((const float*)X)[o]
                               : __bfloat162float(((const __nv_bfloat16*)X)[o]);
      } else {
        v = xtype == OEM_F64 ? (float)((const double*)y)[row] : ((const float*)y)[row];
      }
      sum += v;
      mn = fminf(mn, v);
      mx = fmaxf(mx, v);
    }
  }
  ssum[warp][lane] = sum;
  smin[warp][lane] = mn;
  smax[warp][lane] = mx;
  __syncthreads();
  if (warp == 0 && col <= p) {
    float t = 0.f, a = 3.4e38f, z = -3.4e38f;
    for (int w = 0; w < 8; ++w) {
      t += ssum[w][lane];
      a = fminf(a, smin[w][lane]);
      z = fmaxf(z, smax[w][lane]);
    }
    shift[col] = (a == z) ? a : t / (float)S;
  }
}

cudaError_t launch_col_shift(const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
                             const void* y, float* shift, cudaStream_t s) {
  const unsigned gx = (unsigned)((p + 1 + 31) / 32);
  col_shift_kernel<<<gx, 256, 0, s>>>(X, xtype, n, p, ldx, y, shift);
  return cudaGetLastError();
}

// One block per (fit b, penalty, lambda): beta_j /= sd_j; the intercept in
// the shifted coordinates bprime = ybar - mu^T beta; on the original scale
// beta0 = bprime + shift_y - shift_x^T beta.
__global__ void unstandardize_kernel(double* beta_all, int npen, int nlambda, int p,
                                     const double* __restrict__ cen, const float* __restrict__ shift,
                                     int intercept, double* bprime, double* beta0) {
  __shared__ double red[2][8];
  const int l = blockIdx.x, pen = blockIdx.y, b = blockIdx.z;
  const double* cb = cen + (int64_t)b * (2 * p + 1);
  double* beta = beta_all + (((int64_t)b * npen + pen) * nlambda + l) * p;
  double s1 = 0.0, s2 = 0.0;
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const double v = beta[j] / cb[p + j];
    beta[j] = v;
    s1 = fma(cb[j], v, s1);
    if (shift) s2 = fma((double)shift[j], v, s2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) { red[0][w] = s1; red[1][w] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { t1 += red[0][i]; t2 += red[1][i]; }
    const double bp = intercept ? cb[2 * p] - t1 : 0.0;
    const int64_t o = ((int64_t)b * npen + pen) * nlambda + l;
    if (bprime) bprime[o] = bp;
    if (beta0 && b == 0)
      beta0[(int64_t)pen * nlambda + l] = intercept ? bp + (shift ? (double)shift[p] : 0.0) - t2 : 0.0;
  }
}

cudaError_t launch_unstandardize(double* beta_all, int B, int npen, int nlambda, int p,
                                 const double* cen, const float* shift, int intercept,
                                 double* bprime, double* beta0, cudaStream_t s) {
  unstandardize_kernel<<<dim3(nlambda, npen, B), 256, 0, s>>>(beta_all, npen, nlambda, p, cen, shift,
                                                              intercept, bprime, beta0);
  return cudaGetLastError();
}

}  // namespace oem

namespace oem {

// float32 copy with leading dimension ldg32 >= p; the padding columns are zero.
__global__ void convert_g_kernel(const double* __restrict__ G64, int64_t p, float* G32, int ldg32) {
  const int b = blockIdx.y;
  const int64_t pl = p * ldg32;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < pl;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ldg32, j = e % ldg32;
    G32[(int64_t)b * pl + e] = j < p ? (float)G64[b * p * p + i * p + j] : 0.f;
  }
}

cudaError_t launch_convert_g(const double* G64, int64_t p, int B, float* G32, int ldg32,
                             cudaStream_t s) {
  unsigned gx = (unsigned)((p * p + 255) / 256);
  if (gx > 2048) gx = 2048;
  convert_g_kernel<<<dim3(gx, B), 256, 0, s>>>(G64, p, G32, ldg32);
  return cudaGetLastError();
}

}  // namespace oem
