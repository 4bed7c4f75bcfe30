// The OEM constant d (Section 2.1): OEM converges for every d >= lambda_1(G)
// and fastest at d = lambda_1, which the paper computes by Lanczos. Here:
// Lanczos (three-term recurrence, v_1 = 1/sqrt(p), full reorthogonalisation)
// for a batch of Grams, then the largest Ritz value theta of the tridiagonal
// T_m and its residual norm r = beta_m |s_m|; d = theta + r bounds lambda_1
// from above.
//
// One thread-block cluster per Gram runs all its steps in one launch: the
// CTAs own contiguous rows, reduce through distributed shared memory and
// meet at three cluster barriers per step (after the partial projections of
// each Gram-Schmidt pass, and after the exchange of w''). All arithmetic is
// double-float (pairs of float32, about 48 significant bits) on the float32
// pipe: float64 runs at 1/64 of float32 on this part, with long latencies.
// Cluster partial sums are added in rank order (the same d on every run).
#include "oem_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace oem {

namespace cg = cooperative_groups;


// ------------------------------------------------------------ double-float
// A value is a float2 (hi, lo) with |lo| <= ulp(hi) / 2: about 48 significant
// bits from float32 arithmetic (float64 arithmetic runs at 1/64 of float32 on
// this part, with long latencies). TwoSum and TwoProduct are the error-free
// transformations of Knuth and of Dekker (with a fused multiply-add).
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 df_quick(float a, float b) {  // |a| >= |b| or a == 0
  const float s = a + b;
  return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 df_add(float2 x, float2 y) {
  const float2 s = df_two_sum(x.x, y.x);
  const float2 t = df_two_sum(x.y, y.y);
  float2 u = df_quick(s.x, s.y + t.x);
  return df_quick(u.x, u.y + t.y);
}
__device__ __forceinline__ float2 df_neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
  const float p = x.x * y.x;
  float e = fmaf(x.x, y.x, -p);
  e = fmaf(x.x, y.y, e);
  e = fmaf(x.y, y.x, e);
  return df_quick(p, e);
}
__device__ __forceinline__ float2 df_scale(float2 x, float s) { return make_float2(x.x * s, x.y * s); }  // s a power of two
// running dot product: (h, l) += x * y, renormalised by the caller at the end
__device__ __forceinline__ void df_dot_acc(float& h, float& l, float2 x, float2 y) {
  const float p = x.x * y.x;
  const float pe = fmaf(x.x, y.x, -p);
  const float cr = fmaf(x.x, y.y, x.y * y.x);
  const float s = h + p;
  const float bb = s - h;
  l += ((h - (s - bb)) + (p - bb)) + (pe + cr);
  h = s;
}
__device__ __forceinline__ float2 df_norm(float h, float l) { return df_two_sum(h, l); }
// (h, l) += (h2, l2) without renormalising (for reduction trees)
__device__ __forceinline__ void df_acc_add(float& h, float& l, float h2, float l2) {
  const float2 s = df_two_sum(h, h2);
  h = s.x;
  l += l2 + s.y;
}
// (h, l) summed over the lanes of an aligned group of W lanes (xor tree)
template <int W>
__device__ __forceinline__ void df_group_sum(float& h, float& l) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
    df_acc_add(h, l, h2, l2);
  }
}
// 1 / x and sqrt(x): float32 estimate, one Newton step in double-float
__device__ __forceinline__ float2 df_rcp(float2 x) {
  const float r = 1.f / x.x;
  const float2 e = df_add(make_float2(1.f, 0.f), df_neg(df_mul(x, make_float2(r, 0.f))));
  return df_quick(r, r * e.x);
}
__device__ __forceinline__ float2 df_sqrt(float2 x) {
  if (!(x.x > 0.f)) return make_float2(0.f, 0.f);
  const float r = sqrtf(x.x);
  const float2 e = df_add(x, df_neg(df_mul(make_float2(r, 0.f), make_float2(r, 0.f))));
  return df_quick(r, e.x * (0.5f / r));
}
__device__ __forceinline__ float2 df_from(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// Power of two s with s * max|G_b| in [0.5, 1): every double-float value of
// the recurrence stays far inside the float32 range.
__device__ __forceinline__ float lz_scale(float gmax) {
  if (!(gmax > 0.f) || !isfinite(gmax)) return 1.f;
  int e;
  frexpf(gmax, &e);  // gmax = m 2^e, m in [0.5, 1)
  return ldexpf(1.f, -e);
}

// (hi, lo) float32 copy of G_b and max |G_b| (atomicMax on the bits of a
// non-negative float: the same value whatever the order).
__global__ void lz_split_kernel(const double* __restrict__ G, int64_t p, int64_t ldg, int64_t strideG,
                                LanczosWork w) {
  const int b = blockIdx.y;
  const double* Gb = G + b * strideG;
  float2* out = w.Gs + (int64_t)b * p * p;
  float mx = 0.f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < p * p;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = df_from(Gb[(e / p) * ldg + (e % p)]);
    out[e] = v;
    mx = fmaxf(mx, fabsf(v.x));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned*>(w.gmax) + b, __float_as_uint(mx));
}

// Sum of one double-float per thread of the CTA in a fixed order; every
// thread returns it.
__device__ float2 block_sum_df(float vh, float vl, float2* red) {
  df_group_sum<32>(vh, vl);
  const int wp = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[wp] = df_norm(vh, vl);
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t = red[0];
    for (int i = 1; i < kLzThreads / 32; ++i) t = df_add(t, red[i]);
    red[kLzThreads / 32] = t;
  }
  __syncthreads();
  const float2 t = red[kLzThreads / 32];
  __syncthreads();
  return t;
}

// Steps 0 .. steps-1 of the Lanczos recurrence for Gram b = blockIdx.x / C,
// run by one thread-block cluster of C CTAs in double-float arithmetic on
// the scaled matrix s G_b. CTA rank owns rows [rank per, +per); it holds the
// whole current vector X, its rows of G_b, of the basis V and of w. Per step:
//   v_j = X / beta_{j-1}; w = s G_b v_j on the own rows;
//   two classical Gram-Schmidt passes w <- w - sum_{i <= j} (v_i . w) v_i,
//   each projection summed over the cluster: every CTA stores its partial
//   into a slot of every peer (DSMEM), a cluster barrier, then each CTA adds
//   the C slots in rank order;
//   the CTAs store their rows of w'' into every peer's X together with their
//   partial ||w''||^2, a cluster barrier, beta_j = ||w''|| (the same on every
//   CTA).
// alpha_j = v_j . w + v_j . w'. Three cluster barriers per step.
__global__ void __launch_bounds__(kLzThreads, 1) lz_cluster_kernel(int64_t p, int steps, LanczosWork w, LzPlan L) {
  extern __shared__ __align__(16) unsigned char lz_smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = L.C;
  const int rank = (int)cluster.block_rank();
  const int b = (int)(blockIdx.x / C);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* X = reinterpret_cast<float2*>(lz_smem + L.off_X);
  float2* P1 = reinterpret_cast<float2*>(lz_smem + L.off_P1);
  float2* P2 = reinterpret_cast<float2*>(lz_smem + L.off_P2);
  float2* Bq = reinterpret_cast<float2*>(lz_smem + L.off_B);
  float2* W = reinterpret_cast<float2*>(lz_smem + L.off_W);
  __shared__ float2 red[kLzThreads / 32 + 1];
  __shared__ float2 cs[kLzMax];
  const int64_t r0 = min(p, (int64_t)rank * L.per), r1 = min(p, r0 + L.per);
  const int R = (int)(r1 - r0);
  // basis rows: V(i, t) = vb[i * vs + t]
  float2* vb = L.vsm ? reinterpret_cast<float2*>(lz_smem + L.off_V)
                     : reinterpret_cast<float2*>(w.V + (int64_t)b * (steps + 3) * p) + r0;
  const int64_t vs = L.vsm ? L.vstride : p;
  const float2* Gr = w.Gs + (int64_t)b * p * p + r0 * p;  // own rows of G_b, row stride p
  if (L.gsm) {
    float2* Gsm = reinterpret_cast<float2*>(lz_smem + L.off_G);
    const float4* src = reinterpret_cast<const float4*>(Gr);
    float4* dst = reinterpret_cast<float4*>(Gsm);
    const int64_t n2 = (int64_t)R * p;  // float2 elements
    if ((((int64_t)b * p * p + r0 * p) & 1) == 0) {  // 16-byte aligned start: copy in float4
      for (int64_t e = threadIdx.x; e < n2 / 2; e += kLzThreads) dst[e] = __ldg(src + e);
      if ((n2 & 1) && threadIdx.x == 0) Gsm[n2 - 1] = Gr[n2 - 1];
    } else {
      for (int64_t e = threadIdx.x; e < n2; e += kLzThreads) Gsm[e] = Gr[e];
    }
    Gr = Gsm;
  }
  const float s = lz_scale(w.gmax[b]);
  // ||s G_b||_F^2 over the own rows, summed over the cluster in rank order
  {
    float fh = 0.f, fl = 0.f;
    for (int64_t e = threadIdx.x; e < (int64_t)R * p; e += kLzThreads) {
      const float2 g = df_scale(Gr[e], s);
      df_dot_acc(fh, fl, g, g);
    }
    const float2 f = block_sum_df(fh, fl, red);
    if (threadIdx.x < C) cluster.map_shared_rank(Bq, (int)threadIdx.x)[rank] = f;
  }
  {
    const float2 v0 = df_from(1.0 / sqrt((double)p));
    for (int64_t c = threadIdx.x; c < p; c += kLzThreads) X[c] = v0;
  }
  cluster.sync();  // every CTA initialised (and its ||G||_F^2 part delivered)
  float2 fro2 = Bq[0];
  for (int k = 1; k < C; ++k) fro2 = df_add(fro2, Bq[k]);
  if (rank == 0 && threadIdx.x == 0) {
    w.fro[b] = (double)fro2.x + (double)fro2.y;
    w.mlen[b] = 0;
  }
  const float tol = 1e-13f * sqrtf(fro2.x);
  float2 scale = make_float2(1.f, 0.f);  // v_j = X * scale
  for (int j = 0; j < steps; ++j) {
    // ---- v_j (all rows) and its own rows in V
    for (int64_t c = threadIdx.x; c < p; c += kLzThreads) X[c] = df_mul(X[c], scale);
    __syncthreads();
    for (int t = threadIdx.x; t < R; t += kLzThreads) vb[(int64_t)j * vs + t] = X[r0 + t];
    // ---- w = s G v_j on the own rows (a warp per row, two interleaved sums per lane)
    for (int t = warp; t < R; t += kLzThreads / 32) {
      const float2* g = Gr + (int64_t)t * p;
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
      int c = lane;
      for (; c + 32 < p; c += 64) {
        df_dot_acc(h0, l0, g[c], X[c]);
        df_dot_acc(h1, l1, g[c + 32], X[c + 32]);
      }
      if (c < p) df_dot_acc(h0, l0, g[c], X[c]);
      df_acc_add(h0, l0, h1, l1);
      df_group_sum<32>(h0, l0);
      if (lane == 0) W[t] = df_scale(df_norm(h0, l0), s);
    }
    float2 alpha = make_float2(0.f, 0.f);
    const int nv = j + 1;
    for (int pass = 0; pass < 2; ++pass) {
      float2* Pb = pass ? P2 : P1;
      __syncthreads();
      // partial projections v_i . w over the own rows (8 threads per i), into
      // slot `rank` of every CTA
      for (int i0 = 0; i0 < nv; i0 += kLzThreads / 8) {
        const int i = i0 + (int)(threadIdx.x >> 3), sub = (int)(threadIdx.x & 7);
        float h = 0.f, l = 0.f;
        if (i < nv)
          for (int u = sub; u < R; u += 8) df_dot_acc(h, l, vb[(int64_t)i * vs + u], W[u]);
        df_group_sum<8>(h, l);
        if (i < nv && sub < C) cluster.map_shared_rank(Pb, sub)[rank * kLzMax + i] = df_norm(h, l);
        if (i < nv && C > 8 && sub + 8 < C) cluster.map_shared_rank(Pb, sub + 8)[rank * kLzMax + i] = df_norm(h, l);
      }
      cluster.sync();
      for (int i = threadIdx.x; i < nv; i += kLzThreads) {
        float2 t = Pb[i];
        for (int k = 1; k < C; ++k) t = df_add(t, Pb[k * kLzMax + i]);
        cs[i] = t;
      }
      __syncthreads();
      alpha = df_add(alpha, cs[j]);
      // w <- w - sum_i (v_i . w) v_i on the own rows: 16 threads per row,
      // thread sub takes i = sub, sub + 16, ...; fixed shuffle tree
      for (int t0 = 0; t0 < R; t0 += kLzThreads / 16) {
        const int t = t0 + (int)(threadIdx.x >> 4), sub = (int)(threadIdx.x & 15);
        float h = 0.f, l = 0.f;
        if (t < R)
          for (int i = sub; i < nv; i += 16) df_dot_acc(h, l, cs[i], vb[(int64_t)i * vs + t]);
        df_group_sum<16>(h, l);
        if (t < R && sub == 0) W[t] = df_add(W[t], df_neg(df_norm(h, l)));
      }
    }
    __syncthreads();
    // ---- ||w''||^2 partial; w'' rows and the partial into every CTA
    float bh = 0.f, bl = 0.f;
    for (int t = threadIdx.x; t < R; t += kLzThreads) df_dot_acc(bh, bl, W[t], W[t]);
    const float2 pb_cta = block_sum_df(bh, bl, red);
    for (int e = threadIdx.x; e < C * R; e += kLzThreads) {
      const int k = e / R, t = e % R;
      cluster.map_shared_rank(X, k)[r0 + t] = W[t];
    }
    if (threadIdx.x < C) cluster.map_shared_rank(Bq, (int)threadIdx.x)[rank] = pb_cta;
    cluster.sync();
    float2 bq = Bq[0];
    for (int k = 1; k < C; ++k) bq = df_add(bq, Bq[k]);
    const float2 bn = df_sqrt(bq);
    if (rank == 0 && threadIdx.x == 0) {
      w.alpha[(int64_t)b * kLzMax + j] = alpha;
      w.beta[(int64_t)b * kLzMax + j] = bn;
    }
    if (bn.x <= tol || j + 1 >= steps) {
      if (rank == 0 && threadIdx.x == 0) w.mlen[b] = j + 1;
      break;
    }
    scale = df_rcp(bn);
  }
  cluster.sync();  // no CTA leaves while a peer could still address its shared memory
}

// Number of eigenvalues of the symmetric tridiagonal (a, e) smaller than x:
// the sign changes along chi_0 = 1, chi_1, ..., chi_m, chi_k(x) = det(T_k - x I)
// (Sturm sequence), from the three-term recurrence
//   chi_k = (a_k - x) chi_{k-1} - e_{k-1}^2 chi_{k-2},
// which needs no division. The pair (chi_{k-1}, chi_k) is rescaled by a power
// of two when it leaves [2^-60, 2^60], which keeps every sign; an exact zero
// takes the sign of its predecessor (the usual convention: a zero pivot
// counts as positive). Float32 (coarse phase) and double-float versions.
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
__device__ int sturm_below_df(const float2* a, const float2* e2, int m, float2 x) {
  int cnt = 0;
  const float2 nx = df_neg(x);
  float2 c0 = make_float2(1.f, 0.f), c1 = df_add(a[0], nx);
  if (c1.x == 0.f) c1 = make_float2(0x1p-100f, 0.f);
  if (c1.x < 0.f) ++cnt;
  for (int i = 1; i < m; ++i) {
    float2 c2 = df_add(df_mul(df_add(a[i], nx), c1), df_neg(df_mul(e2[i - 1], c0)));
    if (c2.x == 0.f) c2 = make_float2(copysignf(0x1p-100f, c1.x) * fmaxf(fabsf(c1.x), 0x1p-60f), 0.f);
    if ((c2.x < 0.f) != (c1.x < 0.f)) ++cnt;
    c0 = c1;
    c1 = c2;
    const float mag = fmaxf(fabsf(c0.x), fabsf(c1.x));
    if (mag > 0x1p60f) { c0 = df_scale(c0, 0x1p-60f); c1 = df_scale(c1, 0x1p-60f); }
    else if (mag < 0x1p-60f) { c0 = df_scale(c0, 0x1p60f); c1 = df_scale(c1, 0x1p60f); }
  }
  return cnt;
}

// theta = the largest eigenvalue of T_m (scaled), its unit eigenvector s and
// d = (theta + beta_m |s_m|) (1 + 1e-12) / scale. One warp per Gram.
__global__ void lz_finish_kernel(LanczosWork w, double* d) {
  const int b = blockIdx.x;
  const int lane = threadIdx.x;
  const float sc = lz_scale(w.gmax[b]);
  const float fro = sqrtf((float)w.fro[b]);
  const int m = w.mlen[b];
  if (fro == 0.f || m <= 0) { if (lane == 0) d[b] = 1.0; return; }
  const float2* a = w.alpha + (int64_t)b * kLzMax;
  const float2* e = w.beta + (int64_t)b * kLzMax;  // e[0..m-2] off-diagonal; e[m-1] = beta_m
  if (m == 1) {
    if (lane == 0) d[b] = (((double)a[0].x + (double)a[0].y) + ((double)e[0].x + (double)e[0].y)) / (double)sc;
    return;
  }
  __shared__ float2 ad[kLzMax], e2d[kLzMax];
  __shared__ float af[kLzMax], e2f[kLzMax];
  for (int i = lane; i < m; i += 32) {
    ad[i] = a[i];
    e2d[i] = df_mul(e[i], e[i]);
    af[i] = a[i].x;
    e2f[i] = e[i].x * e[i].x;
  }
  __syncwarp();
  // Gershgorin interval of T_m, widened by a relative 1e-6
  float lo = 3.4e38f, hi = -3.4e38f;
  for (int i = lane; i < m; i += 32) {
    const float r = (i > 0 ? fabsf(e[i - 1].x) : 0.f) + (i < m - 1 ? fabsf(e[i].x) : 0.f);
    lo = fminf(lo, a[i].x - r);
    hi = fmaxf(hi, a[i].x + r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const float scale = fmaxf(fabsf(lo), fabsf(hi));
  lo -= 1e-6f * scale;
  hi += 1e-6f * scale;
  // Multisection for the largest eigenvalue theta: count(x) >= m <=> x > theta.
  // Each round the 32 lanes test 32 interior points and keep the sub-interval
  // where the count crosses m (the interval shrinks 33-fold per round):
  // float32 rounds down to a relative width of 1e-5, the bracket widened and
  // checked in double-float, then double-float rounds.
  float flo = lo, fhi = hi;
  for (int it = 0; it < 12 && (fhi - flo) > 1e-5f * scale; ++it) {
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
  float2 dlo = make_float2(lo, 0.f), dhi = make_float2(hi, 0.f);
  {
    const float mg = 1e-4f * scale;
    const float2 tlo = make_float2(fmaxf(lo, flo - mg), 0.f), thi = make_float2(fminf(hi, fhi + mg), 0.f);
    const bool ok_lo = lane == 0 ? sturm_below_df(ad, e2d, m, tlo) < m : true;
    const bool ok_hi = lane == 1 ? sturm_below_df(ad, e2d, m, thi) >= m : true;
    if (__all_sync(0xffffffffu, ok_lo && ok_hi)) { dlo = tlo; dhi = thi; }
  }
  for (int it = 0; it < 16; ++it) {
    const float2 wd = df_scale(df_add(dhi, df_neg(dlo)), 1.f / 32.f);  // 32 equal parts; lanes test 31 points
    const float2 x = df_add(dlo, df_mul(wd, make_float2((float)(lane + 1), 0.f)));
    const bool above = lane < 31 ? sturm_below_df(ad, e2d, m, x) >= m : true;
    const unsigned mask = __ballot_sync(0xffffffffu, above);
    const int first = __ffs(mask) - 1;  // first tested point above theta (lane 31 stands for dhi)
    const float2 nlo = first == 0 ? dlo : df_add(dlo, df_mul(wd, make_float2((float)first, 0.f)));
    const float2 nhi = first == 31 ? dhi : df_add(dlo, df_mul(wd, make_float2((float)(first + 1), 0.f)));
    const float2 wnew = df_add(nhi, df_neg(nlo)), wold = df_add(dhi, df_neg(dlo));
    if (!(wnew.x < wold.x) || wnew.x <= 1e-14f * scale) { dlo = nlo; dhi = nhi; break; }
    dlo = nlo;
    dhi = nhi;
  }
  if (lane != 0) return;
  const float2 theta = dhi;  // count(dhi) >= m: dhi >= theta
  // eigenvector of T_m for theta by inverse iteration with shift slightly
  // above theta (T - sigma I is then negative definite: no pivoting needed)
  const float2 sigma = df_add(theta, make_float2(1e-12f * fmaxf(fabsf(theta.x), fro), 0.f));
  float2 x[kLzMax], cp[kLzMax], rp[kLzMax];
  {
    float2 den = df_add(ad[0], df_neg(sigma));
    rp[0] = df_rcp(den);
    cp[0] = df_mul(e[0], rp[0]);
    for (int i = 1; i < m; ++i) {
      den = df_add(df_add(ad[i], df_neg(sigma)), df_neg(df_mul(e[i - 1], cp[i - 1])));
      rp[i] = df_rcp(den);
      cp[i] = (i < m - 1) ? df_mul(e[i], rp[i]) : make_float2(0.f, 0.f);
    }
  }
  for (int i = 0; i < m; ++i) x[i] = make_float2(1.f, 0.f);
  for (int rep = 0; rep < 2; ++rep) {
    x[0] = df_mul(x[0], rp[0]);
    for (int i = 1; i < m; ++i) x[i] = df_mul(df_add(x[i], df_neg(df_mul(e[i - 1], x[i - 1]))), rp[i]);
    for (int i = m - 2; i >= 0; --i) x[i] = df_add(x[i], df_neg(df_mul(cp[i], x[i + 1])));
    float h = 0.f, l = 0.f;
    for (int i = 0; i < m; ++i) df_dot_acc(h, l, x[i], x[i]);
    const float2 inv = df_rcp(df_sqrt(df_norm(h, l)));
    for (int i = 0; i < m; ++i) x[i] = df_mul(x[i], inv);
  }
  const float2 r = df_mul(e[m - 1], x[m - 1]);
  const double th = (double)theta.x + (double)theta.y;
  const double rr = fabs((double)r.x + (double)r.y);
  // theta is resolved to about 2^-46 of the spectrum; the relative 1e-12
  // keeps d above lambda_1 whatever the rounding
  d[b] = (th + rr) * (1.0 + 1e-12) / (double)sc;
}

cudaError_t launch_lanczos(const double* G, int64_t p, int64_t ldg, int batch, int64_t strideG,
                           int steps, LanczosWork w, double* d, unsigned* dstatus, cudaStream_t s,
                           int64_t* launches) {
  (void)dstatus;
  steps = lanczos_steps_eff(steps, p);
  cudaError_t e = cudaMemsetAsync(w.gmax, 0, sizeof(float) * batch, s);
  if (e != cudaSuccess) return e;
  {
    const unsigned gx = (unsigned)std::min<int64_t>(1024, (p * p + 255) / 256);
    lz_split_kernel<<<dim3(gx, batch), 256, 0, s>>>(G, p, ldg, strideG, w);
    ++*launches;
  }
  // one cluster per Gram; 16 CTAs when the device can hold such a cluster
  e = cudaFuncSetAttribute(lz_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kLzThreads);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int C = lanczos_cluster(p);
  LzPlan L{};
  for (;;) {
    L = lanczos_plan(p, steps, C);
    attr[0].val.clusterDim.x = (unsigned)C;
    cfg.gridDim = dim3((unsigned)C);
    cfg.dynamicSmemBytes = L.smem;
    e = cudaFuncSetAttribute(lz_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, lz_cluster_kernel, &cfg) == cudaSuccess && nclusters > 0) break;
    cudaGetLastError();
    if (C == 1) return cudaErrorInvalidConfiguration;
    C /= 2;
  }
  cfg.gridDim = dim3((unsigned)(batch * C));
  e = cudaLaunchKernelEx(&cfg, lz_cluster_kernel, p, steps, w, L);
  if (e != cudaSuccess) return e;
  ++*launches;
  lz_finish_kernel<<<batch, 32, 0, s>>>(w, d);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace oem
