// The OEM constant d (Section 2.1): OEM converges for every d >= lambda_1(G)
// and fastest at d = lambda_1, which the paper computes by Lanczos. Here:
// float64 Lanczos (three-term recurrence, v_1 = 1/sqrt(p)) for a batch of
// Grams, then the largest Ritz value theta of the tridiagonal T_m and its
// residual norm r = beta_m |s_m|; d = theta + r bounds lambda_1 from above.
#include "oem_internal.cuh"

namespace oem {

constexpr int kLzMax = 128;  // longest recurrence kept per Gram

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int NT>
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = (threadIdx.x < NT / 32) ? red[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  return red[0];
}

// ||G_b||_F^2 partial sums (float32 arithmetic is plenty: it only scales the
// breakdown test) and v_1 = 1/sqrt(p).
__global__ void lz_init_kernel(const double* __restrict__ G, int64_t p, int64_t ldg,
                               int64_t strideG, LanczosWork w) {
  const int b = blockIdx.y;
  const double* Gb = G + b * strideG;
  float s = 0.f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < p * p;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float v = (float)Gb[(e / p) * ldg + (e % p)];
    s = fmaf(v, v, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&w.fro[b], (double)s);
  if (blockIdx.x == 0) {
    double* V = w.V + (int64_t)b * 3 * p;
    const double v0 = 1.0 / sqrt((double)p);
    for (int64_t i = threadIdx.x; i < p; i += blockDim.x) {
      V[i] = v0;          // slot 0: v_1
      V[2 * p + i] = 0.0; // slot 2: v_0 = 0
    }
    if (threadIdx.x == 0) w.mlen[b] = 0;
  }
}

// w = G v_j for all rows (one warp per row).
__global__ void lz_matvec_kernel(const double* __restrict__ G, int64_t p, int64_t ldg,
                                 int64_t strideG, LanczosWork w, int j) {
  const int b = blockIdx.y;
  if (w.mlen[b] != 0) return;  // finished (breakdown)
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5);
  if (row >= p) return;
  double* V = w.V + (int64_t)b * 3 * p;
  const double* v = V + (int64_t)(j % 3) * p;
  const double* g = G + b * strideG + row * ldg;
  double s = 0.0;
  for (int64_t c = lane; c < p; c += 32) s = fma(g[c], v[c], s);
  s = warp_sum(s);
  if (lane == 0) V[(int64_t)((j + 1) % 3) * p + row] = s;
}

// alpha_j = v_j . w; w -= alpha_j v_j + beta_{j-1} v_{j-1}; beta_j = ||w||;
// v_{j+1} = w / beta_j (stored in place of w).
__global__ void __launch_bounds__(1024) lz_update_kernel(int64_t p, LanczosWork w, int j, int steps) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  if (w.mlen[b] != 0) return;
  double* V = w.V + (int64_t)b * 3 * p;
  double* vc = V + (int64_t)(j % 3) * p;
  double* wv = V + (int64_t)((j + 1) % 3) * p;
  const double* vp = V + (int64_t)((j + 2) % 3) * p;
  const double bprev = (j > 0) ? w.beta[(int64_t)b * kLzMax + j - 1] : 0.0;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < p; i += blockDim.x) s = fma(vc[i], wv[i], s);
  const double a = block_sum<1024>(s, red);
  double s2 = 0.0;
  for (int64_t i = threadIdx.x; i < p; i += blockDim.x) {
    const double t = wv[i] - a * vc[i] - bprev * vp[i];
    wv[i] = t;
    s2 = fma(t, t, s2);
  }
  const double bn = sqrt(block_sum<1024>(s2, red));
  const double scale = sqrt(w.fro[b]);
  const bool stop = (bn <= 1e-13 * scale) || (j + 1 >= steps);
  if (!stop) {
    const double inv = 1.0 / bn;
    for (int64_t i = threadIdx.x; i < p; i += blockDim.x) wv[i] *= inv;
  }
  if (threadIdx.x == 0) {
    w.alpha[(int64_t)b * kLzMax + j] = a;
    w.beta[(int64_t)b * kLzMax + j] = bn;
    if (stop) w.mlen[b] = j + 1;
  }
}

// Number of eigenvalues of the symmetric tridiagonal (a, e) smaller than x:
// the sign changes along chi_0 = 1, chi_1, ..., chi_m, chi_k(x) = det(T_k - x I)
// (Sturm sequence), from the three-term recurrence
//   chi_k = (a_k - x) chi_{k-1} - e_{k-1}^2 chi_{k-2},
// which needs no division (float64 division is slow on this part). The pair
// (chi_{k-1}, chi_k) is rescaled by a power of two when it leaves
// [2^-400, 2^400], which keeps every sign; an exact zero takes the sign of its
// predecessor (the usual convention: a zero pivot counts as positive).
__device__ int sturm_below(const double* a, const double* e, int m, double x) {
  int cnt = 0;
  double c0 = 1.0, c1 = a[0] - x;
  if (c1 == 0.0) c1 = 0x1p-600;
  if (c1 < 0.0) ++cnt;
  for (int i = 1; i < m; ++i) {
    double c2 = fma(a[i] - x, c1, -(e[i - 1] * e[i - 1]) * c0);
    if (c2 == 0.0) c2 = copysign(0x1p-600, c1) * fmax(fabs(c1), 0x1p-400);
    if ((c2 < 0.0) != (c1 < 0.0)) ++cnt;
    c0 = c1;
    c1 = c2;
    const double mag = fmax(fabs(c0), fabs(c1));
    if (mag > 0x1p400) { c0 *= 0x1p-400; c1 *= 0x1p-400; }
    else if (mag < 0x1p-400) { c0 *= 0x1p400; c1 *= 0x1p400; }
  }
  return cnt;
}

__global__ void lz_finish_kernel(LanczosWork w, int steps, double* d) {
  const int b = blockIdx.x;
  (void)steps;
  const double fro = sqrt(w.fro[b]);
  const int m = w.mlen[b];
  if (fro == 0.0 || m <= 0) { d[b] = 1.0; return; }
  const double* a = w.alpha + (int64_t)b * kLzMax;
  const double* e = w.beta + (int64_t)b * kLzMax;  // e[0..m-2] off-diagonal; e[m-1] = beta_m
  if (m == 1) { d[b] = a[0] + e[0]; return; }
  // Gershgorin interval of T_m
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < m - 1 ? fabs(e[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  // Multisection for the largest eigenvalue theta: count(x) >= m <=> x > theta.
  // Each round the 32 lanes test 32 interior points and keep the sub-interval
  // where the count crosses m (the interval shrinks 33-fold per round).
  const int lane = threadIdx.x;
  for (int it = 0; it < 40; ++it) {
    const double wd = (hi - lo) / 33.0;
    const double x = lo + wd * (lane + 1);
    const bool above = (x < hi) && (x > lo) ? sturm_below(a, e, m, x) >= m : (x >= hi);
    const unsigned mask = __ballot_sync(0xffffffffu, above);
    const int first = mask ? __ffs(mask) - 1 : 32;  // first tested point above theta
    const double nlo = first == 0 ? lo : lo + wd * first;
    const double nhi = first == 32 ? hi : lo + wd * (first + 1);
    if (!(nhi - nlo < hi - lo)) break;  // no further progress in float64
    lo = nlo;
    hi = nhi;
  }
  if (lane != 0) return;
  const double theta = hi;
  // eigenvector of T_m for theta by inverse iteration with shift slightly
  // above theta (T - sigma I is then negative definite: no pivoting needed);
  // one reciprocal per row of the Thomas sweep
  const double sigma = theta + 1e-12 * fmax(fabs(theta), fro) + 1e-300;
  double x[kLzMax], cp[kLzMax], rp[kLzMax];
  {
    double den = a[0] - sigma;
    rp[0] = 1.0 / den;
    cp[0] = e[0] * rp[0];
    for (int i = 1; i < m; ++i) {
      den = (a[i] - sigma) - e[i - 1] * cp[i - 1];
      rp[i] = 1.0 / den;
      cp[i] = (i < m - 1) ? e[i] * rp[i] : 0.0;
    }
  }
  for (int i = 0; i < m; ++i) x[i] = 1.0;
  for (int rep = 0; rep < 2; ++rep) {
    // forward: dp_i = (x_i - e_{i-1} dp_{i-1}) / den_i, kept in x
    x[0] = x[0] * rp[0];
    for (int i = 1; i < m; ++i) x[i] = (x[i] - e[i - 1] * x[i - 1]) * rp[i];
    for (int i = m - 2; i >= 0; --i) x[i] = x[i] - cp[i] * x[i + 1];
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm = fma(x[i], x[i], nrm);
    const double inv = 1.0 / sqrt(nrm);
    for (int i = 0; i < m; ++i) x[i] *= inv;
  }
  const double r = fabs(e[m - 1] * x[m - 1]);
  d[b] = theta + r;
}

cudaError_t launch_lanczos(const double* G, int64_t p, int64_t ldg, int batch, int64_t strideG,
                           int steps, LanczosWork w, double* d, cudaStream_t s, int64_t* launches) {
  if (steps <= 0) steps = 64;
  if (steps > kLzMax) steps = kLzMax;
  if (steps > p) steps = (int)p;
  cudaError_t e = cudaMemsetAsync(w.fro, 0, sizeof(double) * batch, s);
  if (e != cudaSuccess) return e;
  {
    unsigned gx = (unsigned)((p * p + 255) / 256);
    if (gx > 64) gx = 64;
    lz_init_kernel<<<dim3(gx, batch), 256, 0, s>>>(G, p, ldg, strideG, w);
    ++*launches;
  }
  const int rows_per_blk = 8;
  const unsigned mgx = (unsigned)((p + rows_per_blk - 1) / rows_per_blk);
  for (int j = 0; j < steps; ++j) {
    lz_matvec_kernel<<<dim3(mgx, batch), rows_per_blk * 32, 0, s>>>(G, p, ldg, strideG, w, j);
    lz_update_kernel<<<batch, 1024, 0, s>>>(p, w, j, steps);
    *launches += 2;
  }
  lz_finish_kernel<<<batch, 32, 0, s>>>(w, steps, d);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace oem
