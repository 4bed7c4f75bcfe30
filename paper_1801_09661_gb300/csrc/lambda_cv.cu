// Lambda grid (Section 5.1, lambda.min.ratio) and cross-validation scoring
// from fold statistics (Sections 3 and 5.4-5.5).
#include "oem_internal.cuh"

namespace oem {

// lambda_max: the smallest lambda at which beta = 0 is the fixed point. With
// beta = 0, u = c: lasso / MCP / SCAD keep beta_j = 0 iff |c_j| <= w_j lambda;
// the elastic net iff |c_j| <= alpha w_j lambda (alpha floored at 1e-3); the
// group lasso iff ||c_g|| <= c_k lambda. Zero weights are unpenalised.
__global__ void lambda_grid_kernel(const double* __restrict__ c, int p,
                                   const DevPenalty* __restrict__ pens, int nlambda, double ratio,
                                   double* __restrict__ lam) {
  __shared__ double red[32];
  const DevPenalty pen = pens[blockIdx.x];
  double m = 0.0;
  if (pen.kind == OEM_GROUP_LASSO || pen.kind == OEM_GROUP_MCP || pen.kind == OEM_GROUP_SCAD) {
    // groups are contiguous: a thread owns each group start. Group MCP /
    // SCAD update the norm with M / C, which vanish iff ||u_g|| <= c_k lambda.
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      if (j == 0 || pen.grp[j] != pen.grp[j - 1]) {
        const int g = pen.grp[j];
        double s = 0.0;
        for (int i = j; i < p && pen.grp[i] == g; ++i) s = fma(c[i], c[i], s);
        const double cg = pen.cg[g];
        if (cg > 0.0) m = fmax(m, sqrt(s) / cg);
      }
    }
  } else if (pen.kind == OEM_SPARSE_GROUP_LASSO) {
    // per group the smallest lambda with ||S(c_g, lambda tau w_g)|| <=
    // lambda (1 - tau) c_k, by bisection (the left side falls, the right
    // side grows with lambda)
    const double tau = pen.alpha64;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      if (!(j == 0 || pen.grp[j] != pen.grp[j - 1])) continue;
      const int g = pen.grp[j];
      int j1 = j;
      while (j1 < p && pen.grp[j1] == g) ++j1;
      const double ck = pen.cg[g];
      auto f = [&](double lam) {
        double s = 0.0;
        for (int i = j; i < j1; ++i) {
          const double w = pen.w64 ? pen.w64[i] : 1.0;
          const double t = fmax(fabs(c[i]) - lam * tau * w, 0.0);
          s = fma(t, t, s);
        }
        return sqrt(s) - lam * (1.0 - tau) * ck;
      };
      double hi = 0.0;
      if (tau > 0.0) {
        for (int i = j; i < j1; ++i) {
          const double w = pen.w64 ? pen.w64[i] : 1.0;
          if (w > 0.0) hi = fmax(hi, fabs(c[i]) / (tau * w));
        }
      } else {
        double s = 0.0;
        for (int i = j; i < j1; ++i) s = fma(c[i], c[i], s);
        hi = ck > 0.0 ? sqrt(s) / ck : 0.0;
      }
      hi = fmax(hi, 1e-300);
      for (int it = 0; it < 2100 && f(hi) > 0.0; ++it) hi *= 2.0;
      double lo = 0.0;
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (f(mid) > 0.0) lo = mid;
        else hi = mid;
      }
      m = fmax(m, hi);
    }
  } else {
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      const double w = pen.w64 ? pen.w64[j] : 1.0;
      if (w > 0.0) m = fmax(m, fabs(c[j]) / w);
    }
    if (pen.kind == OEM_ENET) m /= fmax(pen.alpha64, 1e-3);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    red[0] = t;
  }
  __syncthreads();
  const double lmax = red[0];
  for (int l = threadIdx.x; l < nlambda; l += blockDim.x) {
    const double t = nlambda > 1 ? (double)l / (double)(nlambda - 1) : 0.0;
    lam[(int64_t)blockIdx.x * nlambda + l] = (l == 0) ? lmax : lmax * pow(ratio, t);
  }
}

cudaError_t launch_lambda_grid(const double* c, int p, const DevPenalty* pens, int npen,
                               int nlambda, double ratio, double* lam, cudaStream_t s) {
  lambda_grid_kernel<<<npen, 256, 0, s>>>(c, p, pens, nlambda, ratio, lam);
  return cudaGetLastError();
}

// mse[pen][k][l] = (N_k - 2 beta^T c_k + beta^T G_k beta) / n_k with the raw
// fold sums of fold k and beta = the path leaving fold k out (Gram b = k+1).
// With an intercept (ocol >= 0) the coefficient vector is extended by the
// intercept bprime on the column of ones of Z (index ocol): the same quadratic
// form then gives ||y_k - bprime - X_k beta||^2 in the shifted coordinates.
__global__ void cv_mse_kernel(const double* __restrict__ Zg, int K, int q, int p, int ycols,
                              const int64_t* __restrict__ fold_off,
                              const double* __restrict__ beta_all, int npen, int nlambda,
                              double* __restrict__ mse, int ocol, const double* __restrict__ bprime) {
  __shared__ double red[32];
  __shared__ double bsh[2049];
  const int l = blockIdx.x, k = blockIdx.y, pen = blockIdx.z;
  const double* Z = Zg + (int64_t)k * q * q;
  const int64_t o = ((int64_t)(k + 1) * npen + pen) * nlambda + l;
  const double* beta = beta_all + o * p;
  const int pe = ocol >= 0 ? p + 1 : p;  // coefficients incl. the intercept
  const bool cached = pe <= 2049;
  if (cached) {
    for (int i = threadIdx.x; i < p; i += blockDim.x) bsh[i] = beta[i];
    if (ocol >= 0 && threadIdx.x == 0) bsh[p] = bprime[o];
  }
  __syncthreads();
  auto coef = [&](int i) { return cached ? bsh[i] : (i < p ? beta[i] : bprime[o]); };
  auto col = [&](int i) { return i < p ? i : ocol; };
  double s = 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < pe; i += nw) {
    const double bi = coef(i);
    if (bi == 0.0) continue;  // sparse paths: skip zero rows
    const int64_t ri = (int64_t)col(i) * q;
    double r = 0.0;
    for (int j = lane; j < pe; j += 32) r = fma(Z[ri + col(j)], coef(j), r);
    s = fma(bi, r, s);
    if (lane == 0) {
      double ci = 0.0;
      for (int t = 0; t < ycols; ++t) ci += Z[ri + p + t];
      s -= 2.0 * bi * ci;  // the linear term, added once per row
    }
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o2);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    double Nk = 0.0;
    for (int s2 = 0; s2 < ycols; ++s2)
      for (int t2 = 0; t2 < ycols; ++t2) Nk += Z[(int64_t)(p + s2) * q + p + t2];
    const double nk = (double)(fold_off[k + 1] - fold_off[k]);
    mse[((int64_t)pen * K + k) * nlambda + l] = nk > 0 ? (Nk + t) / nk : 0.0;
  }
}

// cvm, cvsd (sample sd over folds / sqrt(K)), lambda.min (ties to the larger
// lambda), lambda.1se (largest lambda within one cvsd of the minimum), and the
// best penalty (lowest cvm at its lambda.min).
__global__ void cv_select_kernel(const double* __restrict__ mse, int K, int npen, int nlambda,
                                 double* cvm, double* cvsd, int32_t* idx_min, int32_t* idx_1se,
                                 int32_t* best) {
  const int pen = threadIdx.x;
  if (pen < npen) {
    int imin = 0;
    double vmin = 0.0;
    for (int l = 0; l < nlambda; ++l) {
      double m = 0.0;
      for (int k = 0; k < K; ++k) m += mse[((int64_t)pen * K + k) * nlambda + l];
      m /= K;
      double v = 0.0;
      for (int k = 0; k < K; ++k) {
        const double t = mse[((int64_t)pen * K + k) * nlambda + l] - m;
        v = fma(t, t, v);
      }
      const double sd = K > 1 ? sqrt(v / (K - 1)) / sqrt((double)K) : 0.0;
      cvm[(int64_t)pen * nlambda + l] = m;
      cvsd[(int64_t)pen * nlambda + l] = sd;
      if (l == 0 || m < vmin) { vmin = m; imin = l; }
    }
    const double lim = vmin + cvsd[(int64_t)pen * nlambda + imin];
    int i1 = imin;
    for (int l = 0; l <= imin; ++l)
      if (cvm[(int64_t)pen * nlambda + l] <= lim) { i1 = l; break; }
    idx_min[pen] = imin;
    idx_1se[pen] = i1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int bp = 0;
    double bv = 0.0;
    for (int i = 0; i < npen; ++i) {
      const double v = cvm[(int64_t)i * nlambda + idx_min[i]];
      if (i == 0 || v < bv) { bv = v; bp = i; }
    }
    *best = bp;
  }
}

cudaError_t launch_cv_score(const double* Zg, int K, int q, int p, int ycols,
                            const int64_t* fold_off, const double* beta_all, int npen,
                            int nlambda, double* mse, double* cvm, double* cvsd,
                            int32_t* idx_min, int32_t* idx_1se, int32_t* best, cudaStream_t s,
                            int ocol, const double* bprime) {
  cv_mse_kernel<<<dim3(nlambda, K, npen), 256, 0, s>>>(Zg, K, q, p, ycols, fold_off, beta_all,
                                                       npen, nlambda, mse, ocol, bprime);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cv_select_kernel<<<1, 32, 0, s>>>(mse, K, npen, nlambda, cvm, cvsd, idx_min, idx_1se, best);
  return cudaGetLastError();
}

__global__ void copy_paths_kernel(const double* __restrict__ beta_all,
                                  const int32_t* __restrict__ it_all,
                                  const uint8_t* __restrict__ cv_all, int64_t nbeta, int64_t nl,
                                  double* beta, int32_t* iters, uint8_t* conv) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nbeta;
       e += (int64_t)gridDim.x * blockDim.x)
    beta[e] = beta_all[e];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nl;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (iters) iters[e] = it_all[e];
    if (conv) conv[e] = cv_all[e];
  }
}

cudaError_t launch_copy_paths(const double* beta_all, const int32_t* it_all, const uint8_t* cv_all,
                              int npen, int nlambda, int p, double* beta, int32_t* iters,
                              uint8_t* conv, unsigned* dstatus, cudaStream_t s) {
  (void)dstatus;
  const int64_t nl = (int64_t)npen * nlambda;
  copy_paths_kernel<<<256, 256, 0, s>>>(beta_all, it_all, cv_all, nl * p, nl, beta, iters, conv);
  return cudaGetLastError();
}

}  // namespace oem
