// Fold assembly (Section 3): reduce the Gram pass's chunk partials into
// per-fold raw sums of Z^T Z (float64), then form the full-data statistics
// X^T X / n, X^T y / n, y^T y / n and the leave-fold-out statistics by the
// paper's identity X_{-k}^T X_{-k} = sum_{c != k} X_c^T X_c.
#include "oem_internal.cuh"

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

// b = 0: full data / n; b = k+1: (sum - fold k) / (n - n_k).
__global__ void assemble_kernel(const double* __restrict__ Zg, int K, int q, int p, int ycols,
                                const int64_t* __restrict__ fold_off, int B, double* G64,
                                float* G32, int ldg32, double* c, double* N, double* cnt) {
  const int b = blockIdx.y;
  const int64_t n = fold_off[K] - fold_off[0];
  const int64_t nb = (b == 0) ? n : n - (fold_off[b] - fold_off[b - 1]);
  const double inv = nb > 0 ? 1.0 / (double)nb : 0.0;
  const int64_t pp = (int64_t)p * p, qq = (int64_t)q * q;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < pp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / p), j = (int)(e % p);
    const int64_t o = (int64_t)i * q + j;
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += Zg[k * qq + o];
    if (b > 0) s -= Zg[(b - 1) * qq + o];
    const double v = s * inv;
    if (G64) G64[b * pp + e] = v;
    if (G32) {
      float* row = G32 + (int64_t)b * p * ldg32 + (int64_t)i * ldg32;
      row[j] = (float)v;
      if (j == p - 1)  // zero the padding columns of the float32 copy
        for (int jj = p; jj < ldg32; ++jj) row[jj] = 0.f;
    }
    if (j == 0) {
      double sc = 0.0;
      for (int k = 0; k < K; ++k) sc += zc(Zg + k * qq, q, p, ycols, i);
      if (b > 0) sc -= zc(Zg + (b - 1) * qq, q, p, ycols, i);
      c[(int64_t)b * p + i] = sc * inv;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double sn = 0.0;
    for (int k = 0; k < K; ++k) sn += zn(Zg + k * qq, q, p, ycols);
    if (b > 0) sn -= zn(Zg + (b - 1) * qq, q, p, ycols);
    N[b] = sn * inv;
    cnt[b] = (double)nb;
  }
}

cudaError_t launch_assemble(const double* Zg, int K, int q, int p, int ycols,
                            const int64_t* fold_off, int with_leave_out, double* G64, float* G32,
                            int ldg32, double* c, double* N, double* cnt, cudaStream_t s) {
  const int B = with_leave_out ? K + 1 : 1;
  int64_t pp = (int64_t)p * p;
  unsigned gx = (unsigned)((pp + 255) / 256);
  if (gx > 2048) gx = 2048;
  assemble_kernel<<<dim3(gx, B), 256, 0, s>>>(Zg, K, q, p, ycols, fold_off, B, G64, G32, ldg32,
                                              c, N, cnt);
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
