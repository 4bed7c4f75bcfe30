// The OEM iteration (Section 2.1 Step 2, Section 2.2 updates) for every
// (Gram, penalty) instance, warm-started along each instance's lambda grid.
//
// Per instance and iteration: u = c + d beta - G beta; beta <- threshold(u).
// The code carries u itself and updates it by the change of beta,
//   u_{t+1} = u_t + d (beta_{t+1} - beta_t) - G (beta_{t+1} - beta_t),
// which is the same quantity; the mat-vec then acts on a vector that shrinks
// as the iteration converges, so float32 products stay accurate, and u is
// kept as a float32 (hi, lo) pair so its rounding does not accumulate.
//
// One thread-block cluster per Gram. CTA r of the cluster owns rows
// [slice[r], slice[r+1]) of G (the leading rows resident in shared memory)
// and of every instance's u and beta. Each iteration it forms its rows of
// G * dbeta for all instances of the Gram at once (G is read once for all
// of them), thresholds, and writes its slice of the new dbeta into the shared
// memory of every CTA of the cluster (DSMEM), together with its partial
// max|dbeta| and max|beta|; one cluster barrier per iteration. Every CTA then
// takes the same convergence decisions from the same partials.
#include "oem_internal.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace oem {

constexpr int kIterThreads = 256;
constexpr int kIterWarps = kIterThreads / 32;
constexpr int kMaxCluster = 16;

int oem_iter_mpad(int npen) { return npen <= 1 ? 1 : npen <= 2 ? 2 : npen <= 4 ? 4 : 8; }

template <typename T>
__device__ __forceinline__ T dev_copysign(T a, T b) { return copysign(a, b); }

// Scalar updates of Section 2.2 (Eqs. lasso, net, mcp, scad); wl = w_j lambda.
template <typename T>
__device__ __forceinline__ T thr_scalar(int kind, T u, T wl, T alpha, T gamma, T d) {
  const T au = fabs(u);
  if (kind == OEM_LASSO) {
    const T s = au - wl;
    return s > T(0) ? dev_copysign(s / d, u) : T(0);
  }
  if (kind == OEM_ENET) {
    const T s = au - wl * alpha;
    return s > T(0) ? dev_copysign(s / (d + wl * (T(1) - alpha)), u) : T(0);
  }
  if (kind == OEM_MCP) {
    if (au <= wl * gamma * d) {
      const T s = au - wl;
      return s > T(0) ? dev_copysign(gamma * s / (gamma * d - T(1)), u) : T(0);
    }
    return u / d;
  }
  // SCAD
  if (au <= (d + T(1)) * wl) {
    const T s = au - wl;
    return s > T(0) ? dev_copysign(s / d, u) : T(0);
  }
  if (au <= wl * gamma * d)
    return dev_copysign(((gamma - T(1)) * au - wl * gamma) / ((gamma - T(1)) * d - T(1)), u);
  return u / d;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_f(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Load the M entries of column j of the dbeta buffer ([p][M] layout).
template <typename T, int M>
__device__ __forceinline__ void load_col(const T* __restrict__ D, int j, T (&v)[M]) {
  const T* s = D + (size_t)j * M;
  if constexpr (sizeof(T) == 4 && M % 4 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 4) {
      const float4 t = *reinterpret_cast<const float4*>(s + k);
      v[k] = t.x; v[k + 1] = t.y; v[k + 2] = t.z; v[k + 3] = t.w;
    }
  } else if constexpr (sizeof(T) == 4 && M == 2) {
    const float2 t = *reinterpret_cast<const float2*>(s);
    v[0] = t.x; v[1] = t.y;
  } else if constexpr (sizeof(T) == 8 && M % 2 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 2) {
      const double2 t = *reinterpret_cast<const double2*>(s + k);
      v[k] = t.x; v[k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < M; ++k) v[k] = s[k];
  }
}

template <typename T, int M>
__device__ __forceinline__ void store_col(T* __restrict__ dst, const T* __restrict__ src) {
  if constexpr (sizeof(T) == 4 && M % 4 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 4)
      *reinterpret_cast<float4*>(dst + k) = *reinterpret_cast<const float4*>(src + k);
  } else if constexpr (sizeof(T) == 8 && M % 2 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 2)
      *reinterpret_cast<double2*>(dst + k) = *reinterpret_cast<const double2*>(src + k);
  } else {
#pragma unroll
    for (int k = 0; k < M; ++k) dst[k] = src[k];
  }
}

// Shared-memory carve-up (offsets in bytes, each 16-byte aligned).
struct IterSmem {
  size_t dbuf, uhi, ulo, beta, w, v, gn, cgr, glen, st, red, lred, state, gs, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline IterSmem iter_smem_layout(int p, int M, int maxR, int C, int tsz,
                                                     int smem_rows, int ldgs) {
  IterSmem L;
  size_t o = 0;
  L.dbuf = o;  o = al16(o + (size_t)2 * p * M * tsz);
  L.uhi = o;   o = al16(o + (size_t)M * maxR * tsz);
  L.ulo = o;   o = al16(o + (size_t)M * maxR * tsz);
  L.beta = o;  o = al16(o + (size_t)M * maxR * tsz);
  L.w = o;     o = al16(o + (size_t)M * maxR * tsz);
  L.v = o;     o = al16(o + (size_t)M * maxR * tsz);
  L.gn = o;    o = al16(o + (size_t)M * maxR * tsz);
  L.cgr = o;   o = al16(o + (size_t)M * maxR * tsz);
  L.glen = o;  o = al16(o + (size_t)M * maxR * 4);
  L.st = o;    o = al16(o + (size_t)maxR * M * tsz);
  L.red = o;   o = al16(o + (size_t)2 * kMaxCluster * M * 2 * tsz);
  L.lred = o;  o = al16(o + (size_t)kIterWarps * M * 2 * tsz);
  L.state = o; o = al16(o + 256);
  L.gs = o;    o = al16(o + (size_t)smem_rows * ldgs * tsz);
  L.total = o;
  (void)C;
  return L;
}

struct IterState {
  int lidx[8];      // current lambda index
  int its[8];       // iterations at the current lambda
  int done[8];
  int rec[8];       // lambda index recorded this iteration (-1 none)
  int all_done;
  int skip_mv;      // every dbeta of the last iteration was zero
  int has_group;
  float pad;
};

template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e) {
  s = a + b;
  const T bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <typename T, int M>
__global__ void __launch_bounds__(kIterThreads, 1) oem_iter_kernel(IterArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = a.C;
  const int rank = (int)cluster.block_rank();
  const int b = blockIdx.x / C;
  const int p = a.p, L = a.nlambda, m = a.npen, maxR = a.max_rows;
  const int i0 = a.slice[rank], R = a.slice[rank + 1] - i0;
  const int ldgs = (p + 3) & ~3;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr bool kF32 = sizeof(T) == 4;

  extern __shared__ __align__(16) unsigned char smem[];
  const IterSmem Ls = iter_smem_layout(p, M, maxR, C, (int)sizeof(T), a.smem_rows, ldgs);
  T* Dbuf = reinterpret_cast<T*>(smem + Ls.dbuf);
  T* uhi = reinterpret_cast<T*>(smem + Ls.uhi);
  T* ulo = reinterpret_cast<T*>(smem + Ls.ulo);
  T* bet = reinterpret_cast<T*>(smem + Ls.beta);
  T* wv = reinterpret_cast<T*>(smem + Ls.w);
  T* vb = reinterpret_cast<T*>(smem + Ls.v);
  T* gn = reinterpret_cast<T*>(smem + Ls.gn);
  T* cgr = reinterpret_cast<T*>(smem + Ls.cgr);
  int* glen = reinterpret_cast<int*>(smem + Ls.glen);
  T* st = reinterpret_cast<T*>(smem + Ls.st);
  T* red = reinterpret_cast<T*>(smem + Ls.red);
  T* lred = reinterpret_cast<T*>(smem + Ls.lred);
  IterState* S = reinterpret_cast<IterState*>(smem + Ls.state);
  T* Gs = reinterpret_cast<T*>(smem + Ls.gs);

  const T* Gglob = kF32 ? reinterpret_cast<const T*>(a.G32 + (size_t)b * p * a.ldg)
                        : reinterpret_cast<const T*>(a.G64 + (size_t)b * p * p);
  const int ldgg = kF32 ? a.ldg : p;
  const double* cb = a.c + (size_t)b * p;
  const T dgram = (T)a.d[b];

  // per-instance parameters (registers, identical in every thread)
  int kind[M];
  T alpha[M], gamma[M], dk[M], lamv[M];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    if (k < m) {
      const DevPenalty& pen = a.pens[k];
      kind[k] = pen.kind;
      alpha[k] = kF32 ? (T)pen.alpha : (T)pen.alpha64;
      gamma[k] = kF32 ? (T)pen.gamma : (T)pen.gamma64;
      T de = dgram;
      if (pen.kind == OEM_MCP) de = fmax(de, (T)(1.01 / pen.gamma64));
      if (pen.kind == OEM_SCAD) de = fmax(de, (T)(1.01 / (pen.gamma64 - 1.0)));
      dk[k] = de;
      lamv[k] = (T)a.lam[(size_t)k * L];
    } else {
      kind[k] = OEM_LASSO; alpha[k] = T(1); gamma[k] = T(3); dk[k] = T(1); lamv[k] = T(0);
    }
  }

  // ---- initialise: beta = 0, u = c (hi/lo), weights, groups, G rows
  for (int e = tid; e < M * maxR; e += kIterThreads) {
    const int k = e / maxR, i = e % maxR;
    T hi = T(0), lo = T(0), wt = T(1), cgv = T(0);
    int gl = 0;
    if (k < m && i < R) {
      const double cv = cb[i0 + i];
      hi = (T)cv;
      lo = (T)(cv - (double)hi);
      const DevPenalty& pen = a.pens[k];
      if (kF32) { if (pen.w32) wt = (T)pen.w32[i0 + i]; }
      else { if (pen.w64) wt = (T)pen.w64[i0 + i]; }
      if (pen.kind == OEM_GROUP_LASSO) {
        const int g = pen.grp[i0 + i];
        cgv = (T)pen.cg[g];
        if (i == 0 || pen.grp[i0 + i - 1] != g) {
          int len = 1;
          while (i + len < R && pen.grp[i0 + i + len] == g) ++len;
          gl = len;
        }
      }
    }
    uhi[e] = hi; ulo[e] = lo; bet[e] = T(0); wv[e] = wt; cgr[e] = cgv; glen[e] = gl;
    gn[e] = T(0); vb[e] = T(0);
  }
  for (int e = tid; e < 2 * p * M; e += kIterThreads) Dbuf[e] = T(0);
  for (int e = tid; e < a.smem_rows * ldgs; e += kIterThreads) {
    const int i = e / ldgs, j = e % ldgs;
    Gs[e] = (i < R && j < p) ? Gglob[(size_t)(i0 + i) * ldgg + j] : T(0);
  }
  if (tid == 0) {
    for (int k = 0; k < 8; ++k) {
      S->lidx[k] = 0; S->its[k] = 0; S->done[k] = (k >= m); S->rec[k] = -1;
    }
    S->all_done = (m == 0);
    S->skip_mv = 1;
    int hg = 0;
    for (int k = 0; k < m; ++k) hg |= (a.pens[k].kind == OEM_GROUP_LASSO);
    S->has_group = hg;
  }
  cluster.sync();  // every CTA initialised before any DSMEM write

  int cur = 0;
  const T tol = (T)a.tol;
  for (;;) {
    const int nxt = cur ^ 1;
    const T* Dc = Dbuf + (size_t)cur * p * M;
    // ---- phase 1: v = G_slice * dbeta (all instances at once)
    if (!S->skip_mv) {
      for (int ib = warp * 2; ib < R; ib += kIterWarps * 2) {
        const int ib1 = (ib + 1 < R) ? ib + 1 : ib;
        const T* g0 = (ib < a.smem_rows) ? Gs + (size_t)ib * ldgs : Gglob + (size_t)(i0 + ib) * ldgg;
        const T* g1 = (ib1 < a.smem_rows) ? Gs + (size_t)ib1 * ldgs : Gglob + (size_t)(i0 + ib1) * ldgg;
        T acc0[M], acc1[M];
#pragma unroll
        for (int k = 0; k < M; ++k) { acc0[k] = T(0); acc1[k] = T(0); }
        for (int j = lane; j < p; j += 32) {
          T dv[M];
          load_col<T, M>(Dc, j, dv);
          const T ga = g0[j], gb = g1[j];
#pragma unroll
          for (int k = 0; k < M; ++k) { acc0[k] = fma(ga, dv[k], acc0[k]); acc1[k] = fma(gb, dv[k], acc1[k]); }
        }
#pragma unroll
        for (int k = 0; k < M; ++k) { acc0[k] = warp_sum_f(acc0[k]); acc1[k] = warp_sum_f(acc1[k]); }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < M; ++k) {
            vb[k * maxR + ib] = acc0[k];
            if (ib1 != ib) vb[k * maxR + ib1] = acc1[k];
          }
        }
      }
      __syncthreads();
      // ---- phase 2a: u += d dbeta - G dbeta (compensated)
      for (int e = tid; e < M * R; e += kIterThreads) {
        const int k = e / R, i = e % R;
        const int idx = k * maxR + i;
        const T incr = fma(dk[k], Dc[(size_t)(i0 + i) * M + k], -vb[idx]);
        if (kF32) {
          T s, er;
          two_sum(uhi[idx], incr, s, er);
          const T lo = ulo[idx] + er;
          const T hi = s + lo;
          ulo[idx] = lo - (hi - s);
          uhi[idx] = hi;
        } else {
          uhi[idx] += incr;
        }
      }
      __syncthreads();
    }
    // ---- phase 2b: group norms ||u_g|| (groups never straddle slices)
    if (S->has_group) {
      for (int e = tid; e < M * R; e += kIterThreads) {
        const int k = e / R, i = e % R;
        const int idx = k * maxR + i;
        const int len = glen[idx];
        if (len > 0) {
          T s = T(0);
          for (int t = 0; t < len; ++t) s = fma(uhi[idx + t], uhi[idx + t], s);
          s = sqrt(s);
          for (int t = 0; t < len; ++t) gn[idx + t] = s;
        }
      }
      __syncthreads();
    }
    // ---- phase 2c: threshold, dbeta, local maxima
    T mx_d[M], mx_b[M];
#pragma unroll
    for (int k = 0; k < M; ++k) { mx_d[k] = T(0); mx_b[k] = T(0); }
    for (int e = tid; e < M * R; e += kIterThreads) {
      const int k = e / R, i = e % R;
      const int idx = k * maxR + i;
      T dn = T(0);
      // registers are indexed by a runtime k: select through an unrolled loop
#pragma unroll
      for (int kk = 0; kk < M; ++kk) {
        if (kk == k && !S->done[kk]) {
          const T u = uhi[idx];
          T bn;
          if (kind[kk] == OEM_GROUP_LASSO) {
            const T nr = gn[idx];
            const T f = nr > T(0) ? T(1) - cgr[idx] * lamv[kk] / nr : T(0);
            bn = f > T(0) ? u / dk[kk] * f : T(0);
          } else {
            bn = thr_scalar<T>(kind[kk], u, wv[idx] * lamv[kk], alpha[kk], gamma[kk], dk[kk]);
          }
          dn = bn - bet[idx];
          bet[idx] = bn;
          mx_d[kk] = fmax(mx_d[kk], fabs(dn));
          mx_b[kk] = fmax(mx_b[kk], fabs(bn));
        } else if (kk == k) {
          mx_b[kk] = fmax(mx_b[kk], fabs(bet[idx]));
        }
      }
      st[(size_t)i * M + k] = dn;
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
      mx_d[k] = warp_max(mx_d[k]);
      mx_b[k] = warp_max(mx_b[k]);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < M; ++k) {
        lred[(warp * M + k) * 2] = mx_d[k];
        lred[(warp * M + k) * 2 + 1] = mx_b[k];
      }
    }
    __syncthreads();
    // ---- phase 2d: DSMEM all-gather of the dbeta slice and the partial maxima
    for (int e = tid; e < C * R; e += kIterThreads) {
      const int r = e / R, i = e % R;
      T* dst = cluster.map_shared_rank(Dbuf + (size_t)nxt * p * M + (size_t)(i0 + i) * M, r);
      store_col<T, M>(dst, st + (size_t)i * M);
    }
    if (tid < C * M) {
      const int r = tid / M, k = tid % M;
      T md = T(0), mb = T(0);
      for (int w = 0; w < kIterWarps; ++w) {
        md = fmax(md, lred[(w * M + k) * 2]);
        mb = fmax(mb, lred[(w * M + k) * 2 + 1]);
      }
      T* dst = cluster.map_shared_rank(red + ((size_t)(nxt * kMaxCluster + rank) * M + k) * 2, r);
      dst[0] = md;
      dst[1] = mb;
    }
    cluster.sync();
    // ---- phase 3: convergence decisions (identical in every CTA)
    if (tid == 0) {
      int all = 1, anyd = 0;
      for (int k = 0; k < m; ++k) {
        S->rec[k] = -1;
        if (S->done[k]) continue;
        T md = T(0), mb = T(0);
        for (int r = 0; r < C; ++r) {
          md = fmax(md, red[((size_t)(nxt * kMaxCluster + r) * M + k) * 2]);
          mb = fmax(mb, red[((size_t)(nxt * kMaxCluster + r) * M + k) * 2 + 1]);
        }
        if (md > T(0)) anyd = 1;
        const int it = ++S->its[k];
        const bool conv = md <= tol * fmax(T(1), mb);
        if (conv || it >= a.max_iter) {
          const int l = S->lidx[k];
          S->rec[k] = l;
          if (rank == 0) {
            const size_t o = ((size_t)b * m + k) * L + l;
            a.iters[o] = it;
            a.conv[o] = conv ? 1 : 0;
            if (!conv) atomicOr(a.dstatus, kStatNotConv);
          }
          S->its[k] = 0;
          S->lidx[k] = l + 1;
          if (l + 1 >= L) S->done[k] = 1;
        }
        all &= S->done[k];
      }
      S->all_done = all;
      S->skip_mv = !anyd;
    }
    __syncthreads();
    // record solved lambdas (own rows) and move to the next lambda
#pragma unroll
    for (int k = 0; k < M; ++k) {
      if (k < m) {
        const int l = S->rec[k];
        if (l >= 0) {
          double* out = a.beta + (((size_t)b * m + k) * L + l) * p + i0;
          for (int i = tid; i < R; i += kIterThreads) out[i] = (double)bet[k * maxR + i];
          if (l + 1 < L) lamv[k] = (T)a.lam[(size_t)k * L + l + 1];
        }
      }
    }
    const int fin = S->all_done;
    __syncthreads();
    if (fin) break;
    cur = nxt;
  }
  cluster.sync();  // no CTA leaves while a peer could still address its shared memory
}

size_t oem_iter_smem_fixed(int p, int npen, int max_rows, int C, int precision) {
  const int M = oem_iter_mpad(npen);
  const int tsz = precision == OEM_ITER_F64 ? 8 : 4;
  return iter_smem_layout(p, M, max_rows, C, tsz, 0, (p + 3) & ~3).total;
}

size_t oem_iter_smem_per_row(int p, int precision) {
  const int tsz = precision == OEM_ITER_F64 ? 8 : 4;
  return (size_t)((p + 3) & ~3) * tsz;
}

template <typename T, int M>
static cudaError_t launch_t(const IterArgs& a, size_t smem, cudaStream_t s, bool query, int* out) {
  auto kfn = oem_iter_kernel<T, M>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.B * a.C));
  cfg.blockDim = dim3(kIterThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query) {
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kfn, &cfg);
    *out = (e == cudaSuccess) ? n : 0;
    return e;
  }
  return cudaLaunchKernelEx(&cfg, kfn, a);
}

template <typename T>
static cudaError_t dispatch_m(const IterArgs& a, size_t smem, cudaStream_t s, bool q, int* out) {
  switch (oem_iter_mpad(a.npen)) {
    case 1: return launch_t<T, 1>(a, smem, s, q, out);
    case 2: return launch_t<T, 2>(a, smem, s, q, out);
    case 4: return launch_t<T, 4>(a, smem, s, q, out);
    default: return launch_t<T, 8>(a, smem, s, q, out);
  }
}

int oem_iter_max_cluster(const IterArgs& a0, size_t smem, int C) {
  IterArgs a = a0;
  a.C = C;
  int n = 0;
  cudaError_t e = (a.precision == OEM_ITER_F64) ? dispatch_m<double>(a, smem, 0, true, &n)
                                                : dispatch_m<float>(a, smem, 0, true, &n);
  if (e != cudaSuccess) { cudaGetLastError(); return 0; }
  return n;
}

cudaError_t launch_oem_iter(const IterArgs& a, size_t smem, cudaStream_t s) {
  if (a.precision == OEM_ITER_F64) return dispatch_m<double>(a, smem, s, false, nullptr);
  return dispatch_m<float>(a, smem, s, false, nullptr);
}

}  // namespace oem
