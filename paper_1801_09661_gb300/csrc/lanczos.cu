// The OEM constant d (Section 2.1): OEM converges for every d >= lambda_1(G)
// and fastest at d = lambda_1, which the paper computes by Lanczos. Here:
// float64 Lanczos (three-term recurrence, v_1 = 1/sqrt(p)) for a batch of
// Grams, then the largest Ritz value theta of the tridiagonal T_m and its
// residual norm r = beta_m |s_m|; d = theta + r bounds lambda_1 from above.
//
// All steps run in one cooperative launch: each Gram is served by a group of
// CTAs that own contiguous rows, with three group barriers per step (after the
// mat-vec and after the first Gram-Schmidt pass, for the projections
// v_i . w; after the second pass, for beta). The basis is reorthogonalised
// in full (classical Gram-Schmidt twice per step). The next mat-vec reads
// the unnormalised w of the last step and scales by 1 / beta; per-CTA
// partial sums are added in rank order (the same d on every run).
#include "oem_internal.cuh"

#include <algorithm>

namespace oem {


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ||G_b||_F^2 partial sums (float32 arithmetic is plenty: it only scales the
// breakdown test) and v_1 = 1/sqrt(p).
__global__ void lz_init_kernel(const double* __restrict__ G, int64_t p, int64_t ldg,
                               int64_t strideG, LanczosWork w, int steps) {
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
    double* V = w.V + (int64_t)b * (steps + 3) * p;
    const double v0 = 1.0 / sqrt((double)p);
    for (int64_t i = threadIdx.x; i < p; i += blockDim.x) {
      V[i] = v0;          // slot 0: v_0 (the start vector)
    }
    if (threadIdx.x == 0) w.mlen[b] = 0;
  }
}

constexpr int kLzThreads = 256;
constexpr int kLzGather = 64;  // CTAs per Gram at most
constexpr int kLzWarps = kLzThreads / 32;

// Sum of one value per thread of the CTA, in a fixed order (thread 0's
// result is the CTA's partial; every thread returns it).
__device__ double block_sum_fixed(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kLzWarps; ++i) t += red[i];
    red[kLzWarps] = t;
  }
  __syncthreads();
  t = red[kLzWarps];
  __syncthreads();
  return t;
}

// Steps 0 .. steps-1 for Gram b = b0 + blockIdx.x / GC; CTA rank owns rows
// [r0, r1). V slots (each p doubles): i = 0 .. steps hold v_i on the own
// rows (slot 0 starts as the full v_0 = 1/sqrt(p)); steps + 1 + (j & 1)
// holds w_j for all rows. Full reorthogonalisation by classical Gram-Schmidt
// applied twice: w' = w - sum_{i <= j} (v_i . w) v_i, then
// w'' = w' - sum_{i <= j} (v_i . w') v_i; alpha_j = v_j . w + v_j . w',
// beta_j = ||w''||. One group barrier after each of the three reductions.
__global__ void __launch_bounds__(kLzThreads) lz_steps_kernel(const double* __restrict__ G, int64_t p,
                                                             int64_t ldg, int64_t strideG, int steps,
                                                             LanczosWork w, int GC, int b0,
                                                             unsigned* dstatus) {
  extern __shared__ double src_s[];  // [p] the vector the mat-vec multiplies, then
                                     // [GC][j+1] the group's partials (gathered)
  double* gath = src_s + ((p + 1) & ~1LL);
  __shared__ double red[kLzWarps + 1];
  __shared__ double cs[kLzMax];      // projections of the current pass, i <= j
  const int b = b0 + (int)(blockIdx.x / GC), rank = (int)(blockIdx.x % GC);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t per = (p + GC - 1) / GC;
  const int64_t r0 = min(p, (int64_t)rank * per), r1 = min(p, r0 + per);
  const int R = (int)(r1 - r0);
  double* V = w.V + (int64_t)b * (steps + 3) * p;
  const double* Gb = G + b * strideG;
  unsigned* bar = w.bar + 2 * b;
  // partials per CTA: pass-1 projections [0, kLzMax), pass-2 projections
  // [kLzMax, 2 kLzMax), ||w''||^2 at 2 kLzMax
  double* part = w.part + (int64_t)b * kLzGroupMax * kLzPartStride;
  double* mine = part + (int64_t)rank * kLzPartStride;
  const double tol = 1e-13 * sqrt(w.fro[b]);
  unsigned gen = 0;
  double inv_prev = 1.0;
  for (int j = 0; j < steps; ++j) {
    double* vj = V + (int64_t)j * p;
    double* wj = V + (int64_t)(steps + 1 + (j & 1)) * p;
    const double* src = (j == 0) ? V : V + (int64_t)(steps + 1 + ((j + 1) & 1)) * p;
    const double scale = (j == 0) ? 1.0 : inv_prev;
    // ---- v_j = w''_{j-1} / beta_{j-1} (all rows into shared memory, own
    // rows kept), then w = G v_j on the own rows
    for (int64_t c = threadIdx.x; c < p; c += kLzThreads) src_s[c] = __ldcg(src + c) * scale;
    __syncthreads();
    if (j > 0)  // (v_0 is already in slot 0)
      for (int64_t row = r0 + threadIdx.x; row < r1; row += kLzThreads) vj[row] = src_s[row];
    for (int64_t row = r0 + warp; row < r1; row += kLzWarps) {
      const double* g = Gb + row * ldg;
      double acc = 0.0;
      for (int64_t c = lane; c < p; c += 32) acc = fma(g[c], src_s[c], acc);
      acc = warp_sum(acc);
      if (lane == 0) wj[row] = acc;
    }
    double alpha = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      __syncthreads();
      // partial projections v_i . w over the own rows, i <= j
      for (int i = threadIdx.x; i <= j; i += kLzThreads) {
        const double* vi = V + (int64_t)i * p;
        double t = 0.0;
        for (int64_t row = r0; row < r1; ++row) t = fma(vi[row], wj[row], t);
        mine[pass * kLzMax + i] = t;
      }
      if (!group_barrier(bar, (unsigned)GC, gen)) {
        if (threadIdx.x == 0) atomicOr(dstatus, kStatTimeout);
        return;
      }
      // gather all partials at once (independent loads), then add them per
      // projection in rank order
      const int nv = j + 1;
      for (int e = threadIdx.x; e < GC * nv; e += kLzThreads)
        gath[e] = __ldcg(part + (int64_t)(e / nv) * kLzPartStride + pass * kLzMax + e % nv);
      __syncthreads();
      for (int i = threadIdx.x; i < nv; i += kLzThreads) {
        double t = 0.0;
        for (int r = 0; r < GC; ++r) t += gath[r * nv + i];
        cs[i] = t;
      }
      __syncthreads();
      alpha += cs[j];
      // w <- w - sum_i (v_i . w) v_i on the own rows: 16 threads per row,
      // thread sub takes i = sub, sub + 16, ...; fixed shuffle tree
      for (int t0 = 0; t0 < R; t0 += kLzThreads / 16) {
        const int t = t0 + (int)(threadIdx.x >> 4), sub = (int)(threadIdx.x & 15);
        double v = 0.0;
        if (t < R)
          for (int i = sub; i < nv; i += 16) v = fma(cs[i], V[(int64_t)i * p + r0 + t], v);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (t < R && sub == 0) wj[r0 + t] -= v;
      }
    }
    double pb = 0.0;
    for (int t = threadIdx.x; t < R; t += kLzThreads) pb = fma(wj[r0 + t], wj[r0 + t], pb);
    const double pb_cta = block_sum_fixed(pb, red);
    if (threadIdx.x == 0) mine[2 * kLzMax] = pb_cta;
    if (!group_barrier(bar, (unsigned)GC, gen)) {
      if (threadIdx.x == 0) atomicOr(dstatus, kStatTimeout);
      return;
    }
    double bb = threadIdx.x < GC ? __ldcg(part + (int64_t)threadIdx.x * kLzPartStride + 2 * kLzMax) : 0.0;
    const double bn = sqrt(block_sum_fixed(bb, red));
    if (rank == 0 && threadIdx.x == 0) {
      w.alpha[(int64_t)b * kLzMax + j] = alpha;
      w.beta[(int64_t)b * kLzMax + j] = bn;
    }
    if (bn <= tol || j + 1 >= steps) {
      if (rank == 0 && threadIdx.x == 0) w.mlen[b] = j + 1;
      return;
    }
    inv_prev = 1.0 / bn;
    // the next step reads w'' (all rows, complete after the barrier) times
    // 1 / beta_j
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
__device__ int sturm_below(const double* a, const double* e2, int m, double x) {
  // e2[i] = e_i^2 (precomputed). Float64 work per step: one add, one
  // multiply, one fma; the sign test reads the sign bits, and the rescaling
  // test runs every 8 steps (a pair grows by at most (|a|+|x|+|e|)^8 between
  // tests, far inside the 2^+-400 window).
  int cnt = 0;
  double c0 = 1.0, c1 = a[0] - x;
  if (c1 == 0.0) c1 = 0x1p-600;
  cnt += __double2hiint(c1) < 0;
  for (int i = 1; i < m; ++i) {
    double c2 = fma(a[i] - x, c1, -e2[i - 1] * c0);
    if (c2 == 0.0) c2 = copysign(0x1p-600, c1) * fmax(fabs(c1), 0x1p-400);
    cnt += (__double2hiint(c2) ^ __double2hiint(c1)) < 0;
    c0 = c1;
    c1 = c2;
    if ((i & 7) == 0) {
      const int ex = max((__double2hiint(c0) >> 20) & 0x7FF, (__double2hiint(c1) >> 20) & 0x7FF);
      if (ex > 1023 + 400) { c0 *= 0x1p-400; c1 *= 0x1p-400; }
      else if (ex < 1023 - 400) { c0 *= 0x1p400; c1 *= 0x1p400; }
    }
  }
  return cnt;
}

// The same count in float32 (coarse phase of the multisection; float64
// arithmetic is slow on this part). Rescaling by 2^+-60.
__device__ int sturm_below_f32(const float* a, const float* e2, int m, float x) {
  int cnt = 0;
  float c0 = 1.f, c1 = a[0] - x;
  if (c1 == 0.f) c1 = 0x1p-100f;
  if (c1 < 0.f) ++cnt;
  for (int i = 1; i < m; ++i) {
    float c2 = fmaf(a[i] - x, c1, -e2[i - 1] * c0);
    if (c2 == 0.f) c2 = copysignf(0x1p-100f, c1) * fmaxf(fabsf(c1), 0x1p-60f);
    if ((c2 < 0.f) != (c1 < 0.f)) ++cnt;
    c0 = c1;
    c1 = c2;
    const float mag = fmaxf(fabsf(c0), fabsf(c1));
    if (mag > 0x1p60f) { c0 *= 0x1p-60f; c1 *= 0x1p-60f; }
    else if (mag < 0x1p-60f) { c0 *= 0x1p60f; c1 *= 0x1p60f; }
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
  // Coarse rounds in float32 down to a relative width of 1e-5, widened by a
  // margin and checked in float64; then float64 rounds.
  const int lane = threadIdx.x;
  __shared__ double ad[kLzMax], e2d[kLzMax];
  for (int i = lane; i < m; i += 32) {
    ad[i] = a[i];
    e2d[i] = e[i] * e[i];
  }
  __syncwarp();
  {
    __shared__ float af[kLzMax], e2f[kLzMax];
    for (int i = lane; i < m; i += 32) {
      af[i] = (float)a[i];
      e2f[i] = (float)(e[i] * e[i]);
    }
    __syncwarp();
    const float scale = (float)fmax(fabs(lo), fabs(hi));
    float flo = (float)lo, fhi = (float)hi;
    for (int it = 0; it < 8 && (fhi - flo) > 1e-5f * scale; ++it) {
      const float wd = (fhi - flo) / 33.f;
      const float x = flo + wd * (lane + 1);
      const bool above = (x < fhi) && (x > flo) ? sturm_below_f32(af, e2f, m, x) >= m : (x >= fhi);
      const unsigned mask = __ballot_sync(0xffffffffu, above);
      const int first = mask ? __ffs(mask) - 1 : 32;
      const float nlo = first == 0 ? flo : flo + wd * first;
      const float nhi = first == 32 ? fhi : flo + wd * (first + 1);
      if (!(nhi - nlo < fhi - flo)) break;
      flo = nlo;
      fhi = nhi;
    }
    // widen by 1e-4 of the scale and keep it only if float64 counts confirm it
    const double mg = 1e-4 * (double)scale + 1e-300;
    const double tlo = fmax(lo, (double)flo - mg), thi = fmin(hi, (double)fhi + mg);
    const bool ok_lo = lane == 0 ? sturm_below(ad, e2d, m, tlo) < m : true;
    const bool ok_hi = lane == 1 ? sturm_below(ad, e2d, m, thi) >= m : true;
    if (__all_sync(0xffffffffu, ok_lo && ok_hi)) { lo = tlo; hi = thi; }
  }
  for (int it = 0; it < 40; ++it) {
    const double wd = (hi - lo) / 33.0;
    const double x = lo + wd * (lane + 1);
    const bool above = (x < hi) && (x > lo) ? sturm_below(ad, e2d, m, x) >= m : (x >= hi);
    const unsigned mask = __ballot_sync(0xffffffffu, above);
    const int first = mask ? __ffs(mask) - 1 : 32;  // first tested point above theta
    const double nlo = first == 0 ? lo : lo + wd * first;
    const double nhi = first == 32 ? hi : lo + wd * (first + 1);
    if (!(nhi - nlo < hi - lo)) break;  // no further progress in float64
    lo = nlo;
    hi = nhi;
  }
  if (lane != 0) return;
  // full float64 resolution: the inverse iteration's shift below needs theta
  // to ~1e-15 to separate it from near-copies
  const double theta = hi;  // count(hi) >= m: hi >= theta
  // eigenvector of T_m for theta by inverse iteration with shift slightly
  // above theta (T - sigma I is then negative definite: no pivoting needed);
  // one reciprocal per row of the Thomas sweep. The shift must separate theta
  // from near-copies of it (the recurrence is not reorthogonalised), hence
  // float64 and a relative gap of 1e-12.
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
  // theta is resolved to the last bits of float64; the relative 1e-12 keeps
  // d above lambda_1 whatever the rounding in T_m
  d[b] = (theta + r) * (1.0 + 1e-12);
}

cudaError_t launch_lanczos(const double* G, int64_t p, int64_t ldg, int batch, int64_t strideG,
                           int steps, LanczosWork w, double* d, unsigned* dstatus, cudaStream_t s,
                           int64_t* launches) {
  steps = lanczos_steps_eff(steps, p);
  cudaError_t e = cudaMemsetAsync(w.fro, 0, sizeof(double) * batch, s);
  if (e != cudaSuccess) return e;
  {
    unsigned gx = (unsigned)((p * p + 255) / 256);
    if (gx > 64) gx = 64;
    lz_init_kernel<<<dim3(gx, batch), 256, 0, s>>>(G, p, ldg, strideG, w, steps);
    ++*launches;
  }
  // one cooperative launch per batch slice whose CTA groups fit on the device
  int dev = 0, sms = kNumSMsHint, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // shared memory: the vector (p, rounded to even) + the gathered partials
  const size_t smem = ((size_t)((p + 1) & ~1LL) + (size_t)kLzGather * kLzMax) * sizeof(double);
  e = cudaFuncSetAttribute(lz_steps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lz_steps_kernel, kLzThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int cap = per_sm * sms;
  e = cudaMemsetAsync(w.bar, 0, sizeof(unsigned) * 2 * batch, s);
  if (e != cudaSuccess) return e;
  // about 16 rows per CTA (two per warp), at most kLzGather CTAs per Gram:
  // fewer CTAs make the group barriers and sums cheaper
  const int want = (int)std::min<int64_t>(kLzGather, std::max<int64_t>(1, (p + 15) / 16));
  for (int b0 = 0; b0 < batch;) {
    const int nb = std::min(batch - b0, cap);
    const int GC = std::max(1, std::min(want, std::min(sms, cap) / nb));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nb * GC));
    cfg.blockDim = dim3(kLzThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident, or no launch
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, lz_steps_kernel, G, p, ldg, strideG, steps, w, GC, b0, dstatus);
    if (e != cudaSuccess) return e;
    ++*launches;
    b0 += nb;
  }
  lz_finish_kernel<<<batch, 32, 0, s>>>(w, steps, d);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace oem
