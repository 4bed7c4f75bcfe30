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
// Replicated update. A task (a Gram with M of its instances; tasks of one
// launch may differ in p) runs on C CTAs: one thread-block cluster (C <= 16)
// or, in grid mode, C CTAs of a cooperative launch. CTA r owns the mat-vec
// rows [slice[r], slice[r+1]) of G, but every CTA keeps u, beta and dbeta of
// ALL p rows and applies the thresholds to all of them. One iteration:
//   A. every CTA forms y_i = (G dbeta)_i of its rows for the M instances and
//      sends them to every CTA of the task (cluster: st.async stores into
//      each peer's shared memory, counted on the receiver's mbarrier; float64
//      iteration: DSMEM stores and a cluster barrier; grid mode: 64-bit words
//      in global memory that carry the exchange number in their high half,
//      so a reader polls for exactly the words it needs);
//   B. every thread updates u of its elements by d dbeta - y (float32 TwoSum);
//   C. the thresholds give beta and the new dbeta (group norms between two
//      block barriers for group penalties);
//   D. max|dbeta| and max|beta| per instance by a block reduction: every CTA
//      holds all rows, so its block maxima are the task's maxima and every
//      CTA takes the same convergence decisions with no second exchange.
// The mat-vec keeps its G rows in registers where they fit, else in shared
// memory, else reads them from L2. For p <= 1024 each warp owns rows and runs
// over all columns (lane l reads columns 4l .. 4l+3, + 128, ...; one
// reduce-scatter per row group); for larger p each warp owns 128-column
// segments of all the CTA's rows and the segment sums are added in segment
// order. Either way the order of every sum depends on p only, so every layout
// (cluster size, grid mode, instances per task) gives the same bits. A launch
// may stop after a loop budget and save its state (serving), to be resumed by
// a later launch. Every wait is bounded (IterLaunch::wait_cycles): on expiry
// the kernel sets the timeout status bit and returns.
#include "oem_internal.cuh"
#include "iter_common.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace oem {

int oem_iter_mpad(int npen) { return npen <= 1 ? 1 : npen <= 2 ? 2 : npen <= 4 ? 4 : 8; }


// 512 threads: one G row per warp held in registers (long rows); else 256.
__host__ __device__ constexpr int rep_threads(bool longrow) { return longrow ? 512 : 256; }
constexpr int kRepMaxWarps = 16;

// Shared-memory carve-up (byte offsets, 16-byte aligned).
struct RepSmem {
  size_t db, yb, uh, ul, be, gn, cg, gl, sl, sn, lred, xbar, gs, total;
};
// Group slots per instance: whole groups packed into 32-lane slots (groups
// of at most 32 rows; at least half a slot is used, so p / 16 + 2 slots).
__host__ __device__ inline int rep_gslots(int p) { return p / 16 + 2; }
__host__ __device__ inline RepSmem rep_smem_layout(int p, int M, int tsz, bool grid, bool groups,
                                                   int smem_rows) {
  const int ldgs = (p + 3) & ~3;
  const int NW = kRepMaxWarps;
  const size_t pm = (size_t)p * M;
  RepSmem L;
  size_t o = 0;
  L.db = o;   o = al16(o + 2 * (size_t)ldgs * M * tsz);           // dbeta, two parities
  L.yb = o;   o = al16(o + 2 * (size_t)ldgs * M * tsz);           // G dbeta received, two parities
  L.uh = o;   o = al16(o + pm * tsz);
  L.ul = o;   o = al16(o + pm * tsz);
  L.be = o;   o = al16(o + pm * tsz);
  L.gn = o;   o = al16(o + (groups ? pm * tsz : 0));              // group norm per element
  L.cg = o;   o = al16(o + (groups ? pm * tsz : 0));              // group weight per element
  L.gl = o;   o = al16(o + (groups ? pm * 4 : 0));                // group length at group starts
  L.sl = o;   o = al16(o + (groups ? (size_t)M * rep_gslots(p) * 32 * 4 : 0));  // group slots
  L.sn = o;   o = al16(o + (groups ? (size_t)(M + 1) * 4 : 0));   // slots per instance, long-group flag
  L.lred = o; o = al16(o + (size_t)2 * NW * 2 * M * 4);
  L.xbar = o; o = al16(o + 32);                                   // two mbarriers, timeout flag
  L.gs = o;   o = al16(o + (size_t)smem_rows * ldgs * tsz);
  L.total = o;
  return L;
}

template <typename T, int M, int NT, bool kGrid, int RG, bool kLong>
__global__ void __launch_bounds__(NT, 1) oem_iter_kernel(IterLaunch P) {
  constexpr int NW = NT / 32;
  constexpr bool kF32 = sizeof(T) == 4;
  constexpr bool kAsync = kF32 && !kGrid;
  static_assert(NT % M == 0 && 32 % M == 0, "instances per lane layout");
  // elements per thread whose state lives in registers (the wide mat-vec's
  // G rows take most of the 128 registers a thread has at 512 threads)
  constexpr int kRepJR = kLong ? 2 : 4;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = P.C;
  const int rank = kGrid ? (int)(blockIdx.x % C) : (int)cluster.block_rank();
  const IterTask& tk = P.tasks[blockIdx.x / C];
  const int p = tk.p, L = tk.L, m = tk.npen;
  const int i0 = kGrid ? tk.gslice[rank] : tk.slice[rank];
  const int R = (kGrid ? tk.gslice[rank + 1] : tk.slice[rank + 1]) - i0;
  const int ldgs = (p + 3) & ~3, smem_rows = tk.smem_rows;
  const int PM = p * M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long wait_lim = P.wait_cycles > 0 ? P.wait_cycles : 4000000000LL;

  extern __shared__ __align__(16) unsigned char smem[];
  const RepSmem Ls = rep_smem_layout(p, M, (int)sizeof(T), kGrid, P.groups != 0, smem_rows);
  T* const Dbuf = reinterpret_cast<T*>(smem + Ls.db);
  T* const Ybuf = reinterpret_cast<T*>(smem + Ls.yb);   // [2][ldgs][M]
  T* const uhs = reinterpret_cast<T*>(smem + Ls.uh);
  T* const uls = reinterpret_cast<T*>(smem + Ls.ul);
  T* const bes = reinterpret_cast<T*>(smem + Ls.be);
  T* const gns = reinterpret_cast<T*>(smem + Ls.gn);
  T* const cgs = reinterpret_cast<T*>(smem + Ls.cg);
  int* const gls = reinterpret_cast<int*>(smem + Ls.gl);
  uint32_t* const gsl = reinterpret_cast<uint32_t*>(smem + Ls.sl);  // [M][gsm][32]: row | start << 16 | end << 21
  int* const gsn = reinterpret_cast<int*>(smem + Ls.sn);            // [M] slots, [M] any group > 32 rows
  volatile int* const long_grp = gsn + M;
  const int gsm = rep_gslots(p);
  float* const lred = reinterpret_cast<float*>(smem + Ls.lred);  // [2][NW][2M] (room for 16 warps)
  const uint32_t xbar0 = xs_u32(smem + Ls.xbar);                 // mbarriers of Ybuf parities 0 / 1
  T* const Gs = reinterpret_cast<T*>(smem + Ls.gs);
  unsigned long long* const xw = reinterpret_cast<unsigned long long*>(tk.xD);  // grid: [2][PM][W]
  const T* Gglob = kF32 ? reinterpret_cast<const T*>(tk.G32) : reinterpret_cast<const T*>(tk.G64);
  const int ldgg = kF32 ? tk.ldg : p;
  const T dgram = (T)tk.d[0];

  // ---- per-instance parameters and control state (identical in every thread)
  int kind[M], lidx[M], its[M], done[M];
  T alpha[M], gamma[M], dk[M], lamv[M];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    lidx[k] = 0; its[k] = 0; done[k] = 1;
    kind[k] = OEM_LASSO; alpha[k] = T(1); gamma[k] = T(3); dk[k] = T(1); lamv[k] = T(0);
    if (k < m) {
      const DevPenalty& pen = tk.pens[k];
      kind[k] = pen.kind;
      alpha[k] = kF32 ? (T)pen.alpha : (T)pen.alpha64;
      gamma[k] = kF32 ? (T)pen.gamma : (T)pen.gamma64;
      T de = dgram;
      if (pen.kind == OEM_MCP || pen.kind == OEM_GROUP_MCP) de = fmax(de, (T)(1.01 / pen.gamma64));
      if (pen.kind == OEM_SCAD || pen.kind == OEM_GROUP_SCAD) de = fmax(de, (T)(1.01 / (pen.gamma64 - 1.0)));
      dk[k] = de;
      done[k] = 0;
      if (tk.resume) {
        lidx[k] = tk.st_ctl[k * 4 + 0];
        its[k] = tk.st_ctl[k * 4 + 1];
        done[k] = tk.st_ctl[k * 4 + 2];
      }
      if (!done[k]) lamv[k] = (T)tk.lam[(size_t)k * L + lidx[k]];
    }
  }
  bool has_group = false;
  for (int k = 0; k < m; ++k) has_group |= (tk.pens[k].kind >= OEM_GROUP_LASSO);

  // ---- this thread's elements e = tid + NT j: row e / M, instance kq = tid % M
  const int kq = tid % M;
  const bool my_inst = kq < m;
  int my_kind = OEM_LASSO;
  T my_alpha = T(1), my_gamma = T(3), my_d = T(1), my_lam = T(0);
  int my_done = 1;
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (k == kq) {
      my_kind = kind[k]; my_alpha = alpha[k]; my_gamma = gamma[k]; my_d = dk[k];
      my_lam = lamv[k]; my_done = done[k];
    }
  const float* w32 = my_inst ? tk.pens[kq].w32 : nullptr;
  const double* w64 = my_inst ? tk.pens[kq].w64 : nullptr;
  auto weight = [&](int i) -> T {
    if constexpr (kF32) return w32 ? (T)w32[i] : T(1);
    else return w64 ? (T)w64[i] : T(1);
  };
  const int nJ = (PM + NT - 1) / NT;
  T r_uh[kRepJR], r_ul[kRepJR], r_b[kRepJR], r_w[kRepJR], r_dn[kRepJR];

  // ---- initialise u, beta (every row), weights, group arrays, dbeta, G rows
  for (int j = 0; j < nJ; ++j) {
    const int e = tid + NT * j;
    if (e >= PM) break;
    const int i = e / M;
    T hi = T(0), lo = T(0), b0 = T(0);
    if (my_inst) {
      if (tk.resume) {
        const size_t o = (size_t)kq * p + i;
        hi = (T)tk.st_u[2 * o];
        lo = (T)tk.st_u[2 * o + 1];
        b0 = (T)tk.st_beta[o];
      } else {
        const double cv = tk.c[i];
        hi = (T)cv;
        lo = (T)(cv - (double)hi);
      }
    }
    uhs[e] = hi; uls[e] = lo; bes[e] = b0;
#pragma unroll
    for (int q = 0; q < kRepJR; ++q)
      if (q == j) { r_uh[q] = hi; r_ul[q] = lo; r_b[q] = b0; r_w[q] = weight(i); r_dn[q] = T(0); }
  }
  if (P.groups) {
    for (int e2 = tid; e2 < PM; e2 += NT) {
      const int k = e2 / p, i = e2 % p;
      T cgv = T(0);
      int gl = 0;
      if (k < m && tk.pens[k].kind >= OEM_GROUP_LASSO) {
        const DevPenalty& pen = tk.pens[k];
        const int g = pen.grp[i];
        cgv = (T)pen.cg[g];
        if (i == 0 || pen.grp[i - 1] != g) {
          int len = 1;
          while (i + len < p && pen.grp[i + len] == g) ++len;
          gl = len;
        }
      }
      cgs[e2] = cgv; gls[e2] = gl; gns[e2] = T(0);
    }
    for (int e3 = tid; e3 < M * gsm * 32; e3 += NT) gsl[e3] = 0xFFFFFFFFu;
    if (tid == 0) *long_grp = 0;
    __syncthreads();
    // pack each group instance's groups, in order, into 32-lane slots
    if (lane == 0 && warp < M) {
      const int k = warp;
      int sl = 0, used = 0, lng = 0;
      if (k < m && tk.pens[k].kind >= OEM_GROUP_LASSO) {
        for (int i = 0; i < p;) {
          const int len = max(1, gls[k * p + i]);
          if (len > 32) { lng = 1; break; }
          if (used + len > 32) { ++sl; used = 0; }
          if (sl >= gsm) { lng = 1; break; }  // cannot happen for groups <= 32 rows
          for (int q = 0; q < len; ++q)
            gsl[((size_t)k * gsm + sl) * 32 + used + q] =
                (uint32_t)(i + q) | ((uint32_t)used << 16) | ((uint32_t)(used + len - 1) << 21);
          used += len;
          i += len;
        }
        if (used) ++sl;
      }
      gsn[k] = sl;
      if (lng) atomicOr((int*)long_grp, 1);
    }
  }
  for (int e = tid; e < 2 * ldgs * M; e += NT) Dbuf[e] = T(0);
  if (kAsync && tid == 0) {
    xs_init_n(xbar0, NW);
    xs_init_n(xbar0 + 8, NW);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = tid; e < smem_rows * ldgs; e += NT) {
    const int i = e / ldgs, j = e % ldgs;
    Gs[e] = (i < R && j < p) ? Gglob[(size_t)(i0 + i) * ldgg + j] : T(0);
  }

  // ---- mat-vec roles: warp w owns rows [wlo, whi) of the CTA's slice; a
  // row group is RG rows (V = RG M sums); after the reduction lane l holds
  // the sum of value v = l / S, S = 32 / V: row rsub = v / M of the group and
  // instance kv = v % M (the first lane of each group of S acts). Lane l runs
  // over columns 4l .. 4l+3, + 128, ... and the lanes' sums meet in one
  // butterfly, for every p and every layout.
  constexpr int V = RG * M, S = 32 / V;
  static_assert(V == 1 || V == 2 || V == 4 || V == 8 || V == 16, "row group");
  const int vq = lane / S, rsub = vq / M, kv = vq % M;
  const bool even = (lane % S) == 0;
  int wlo = 0, whi = 0;
  {
    const int per = (R + NW - 1) / NW;
    wlo = min(R, warp * per);
    whi = min(R, wlo + per);
  }
  // Float32 G rows in registers when a warp holds one row group: lane l
  // holds columns 4l .. 4l+3 + 128 s of each row, s < kGS (p <= 512 with
  // 256 threads; one row per warp and p <= 2048 with 512). Same products in
  // the same order as from shared memory.
  constexpr int kGS = kLong ? 16 : 4;
  constexpr bool kGregT = kF32 && RG <= 4;
  const bool greg_on = kGregT && (whi - wlo) <= RG && p <= 128 * kGS;
  float4 greg[kGregT ? RG : 1][kGregT ? kGS : 1];
  auto grow = [&](int ib) -> const T* {  // local row ib of this CTA's slice
    return ib < smem_rows ? Gs + (size_t)ib * ldgs : Gglob + (size_t)(i0 + ib) * ldgg;
  };
  __syncthreads();
  if constexpr (kGregT) {
#pragma unroll
    for (int r = 0; r < RG; ++r)
#pragma unroll
      for (int sx = 0; sx < kGS; ++sx) {
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        const int j4 = lane * 4 + 128 * sx;
        if (greg_on && r < whi - wlo && j4 < p) g = *reinterpret_cast<const float4*>(grow(wlo + r) + j4);
        greg[r][sx] = g;
      }
  }
  if constexpr (!kGrid) cluster.sync();  // every CTA initialised before any DSMEM access

  const T tol = (T)P.tol;
  int skip_mv = 1;  // dbeta of the previous iteration is all zero (y = 0)
  int all_done = 1;
  for (int k = 0; k < m; ++k) all_done &= done[k];
  unsigned xc = 0;  // exchanges done (grid-mode tags are xc + 1)
  int64_t loops = 0;
  int t = 0;
  bool final_pass = false;  // one more mat-vec and u update before saving the state
  bool fail = false;
  while (!all_done || final_pass) {
    const T* Dp = Dbuf + (size_t)((t & 1) ^ 1) * ldgs * M;  // dbeta of the last iteration
    T* Dn = Dbuf + (size_t)(t & 1) * ldgs * M;              // dbeta of this one
    const bool got_y = !skip_mv;
    const unsigned b = xc & 1;
    const unsigned tag = xc + 1;
    // the tag a reader waits for (test_stall: one that is never written)
    const unsigned want_tag = tag + ((P.test_stall && xc == 0) ? 1u : 0u);
    T* Yb = Ybuf + (size_t)b * ldgs * M;  // parities 16-byte aligned
    if (got_y) {
      // ---- A. y = G dbeta for this CTA's rows, delivered to every CTA
      auto deliver = [&](int il, int k, T y) {  // local row il, instance k
        const int e = (i0 + il) * M + k;
        if constexpr (kGrid) {
          if constexpr (kF32) {
            st_tag1(xw + (size_t)b * PM + e, tag_word(__float_as_uint(y), tag));
          } else {
            const unsigned long long bits = (unsigned long long)__double_as_longlong(y);
            st_tag2(xw + ((size_t)b * PM + e) * 2, tag_word((uint32_t)bits, tag),
                    tag_word((uint32_t)(bits >> 32), tag));
          }
        } else if constexpr (kF32) {
          Yb[e] = y;
        } else {
          for (int r = 0; r < C; ++r) cluster.map_shared_rank(Yb, r)[e] = y;
        }
      };
      {
        for (int gb = wlo; gb < whi; gb += RG) {
          const int nv = min(RG, whi - gb);
          T acc[V];
#pragma unroll
          for (int q = 0; q < V; ++q) acc[q] = T(0);
          if constexpr (kF32) {
            auto step4 = [&](int j4, auto gload) {
              float dv[4][M];
#pragma unroll
              for (int q = 0; q < M; ++q) {
                const int u = (j4 * M >> 2) + q;
                const float4 tq = *reinterpret_cast<const float4*>(Dp + ((u ^ ((u >> 3) & (M - 1))) << 2));
                const float tv[4] = {tq.x, tq.y, tq.z, tq.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) dv[(q * 4 + e) / M][(q * 4 + e) % M] = tv[e];
              }
#pragma unroll
              for (int r = 0; r < RG; ++r) {
                const float4 g4 = gload(r);
                const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                  for (int k = 0; k < M; ++k) acc[r * M + k] = fma(gv[c], dv[c][k], acc[r * M + k]);
              }
            };
            if (kGregT && greg_on) {
#pragma unroll
              for (int sx = 0; sx < kGS; ++sx) {
                const int j4 = lane * 4 + 128 * sx;
                if (j4 < p) step4(j4, [&](int r) { return greg[kGregT ? r : 0][kGregT ? sx : 0]; });
              }
            } else {
              const T* gr[RG];
#pragma unroll
              for (int r = 0; r < RG; ++r) gr[r] = grow(gb + min(r, nv - 1));
              for (int j4 = lane * 4; j4 < p; j4 += 128)
                step4(j4, [&](int r) {
                  return r < nv ? *reinterpret_cast<const float4*>(gr[r] + j4) : make_float4(0.f, 0.f, 0.f, 0.f);
                });
            }
          } else {
            const T* gr[RG];
#pragma unroll
            for (int r = 0; r < RG; ++r) gr[r] = grow(gb + min(r, nv - 1));
#pragma unroll 4
            for (int j = lane; j < p; j += 32) {
              T dv[M];
              load_col<T, M>(Dp, j, dv);
#pragma unroll
              for (int r = 0; r < RG; ++r) {
                const T g = r < nv ? gr[r][j] : T(0);
#pragma unroll
                for (int k = 0; k < M; ++k) acc[r * M + k] = fma(g, dv[k], acc[r * M + k]);
              }
            }
          }
          const T y = reduce_scatter_any<V>(acc, lane);
          if (even && gb + rsub < whi) deliver(gb + rsub, kv, y);
        }
        if constexpr (kAsync) {
          // this warp's words to every peer: a 16-byte unit inside the warp's
          // rows as one float4 store, a unit shared with a neighbour warp word
          // by word (i0 M is a multiple of 4: units are aligned)
          __syncwarp();
          const int f0 = (i0 + wlo) * M, f1 = (i0 + whi) * M;
          const int u0 = f0 >> 2, nu = f1 > f0 ? ((f1 + 3) >> 2) - u0 : 0;
          const uint32_t bar = xbar0 + 8 * b;
          for (int e = lane; e < nu * (C - 1); e += 32) {
            const int u = u0 + e / (C - 1);
            int r = e % (C - 1);
            r += (r >= rank);
            const float* src = Yb + 4 * u;
            const uint32_t ra = xs_map(xs_u32(src), r), rb = xs_map(bar, r);
            if (4 * u >= f0 && 4 * u + 4 <= f1) {
              xs_st4(ra, *reinterpret_cast<const float4*>(src), rb);
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (4 * u + q >= f0 && 4 * u + q < f1) xs_st1(ra + 4 * q, __float_as_uint(src[q]), rb);
            }
          }
        }
      }
      // ---- wait for every CTA's y
      if constexpr (kAsync) {
        __syncwarp();
        const uint32_t bar = xbar0 + 8 * b;
        if (lane == 0) {
          // test_stall: four bytes more than the peers send
          if (warp == 0) xs_arm(bar, (uint32_t)((p - R) * M * 4) + ((P.test_stall && xc == 0) ? 4u : 0u));
          else xs_arrive(bar);
        }
        const uint32_t par = (xc >> 1) & 1u;
        bool ok = xs_try(bar, par);
        if (!ok) {
          const long long t0 = clock64();
          while (!(ok = xs_try(bar, par)))
            if (clock64() - t0 > wait_lim) break;
        }
        if (!ok) fail = true;
      } else if constexpr (!kGrid) {
        cluster.sync();
      }
      ++xc;
    }

    // ---- B, C. u update, thresholds, dbeta and maxima for this thread's elements
    // y of element e (grid mode: polled until its tag is this exchange's)
    // grid mode: y of this thread's elements from global memory -- the loads
    // of a batch of elements in flight at once, the stale ones again (after a
    // short pause, to spare L2 the spinning) until their tag is this
    // exchange's; register elements' values go to yr, the others to this
    // thread's own slots of Yb (cluster mode: already in Yb)
    T yr[kRepJR];
#pragma unroll
    for (int j = 0; j < kRepJR; ++j) yr[j] = T(0);
    if (got_y) {
      if constexpr (kGrid) {
        constexpr int kB = kLong ? 4 : 8;
        long long t0 = 0;
        bool started = false;
        for (int j0 = 0; j0 < nJ && !fail; j0 += kB) {
          unsigned long long w0[kB], w1[kB];
          unsigned pend = 0;
#pragma unroll
          for (int q = 0; q < kB; ++q)
            if (j0 + q < nJ && tid + NT * (j0 + q) < PM) pend |= 1u << q;
          while (pend) {
#pragma unroll
            for (int q = 0; q < kB; ++q) {
              const size_t e = (size_t)tid + (size_t)NT * (j0 + q);
              if ((pend >> q) & 1u) {
                if constexpr (kF32) w0[q] = ld_tag1(xw + (size_t)b * PM + e);
                else ld_tag2(xw + ((size_t)b * PM + e) * 2, w0[q], w1[q]);
              }
            }
#pragma unroll
            for (int q = 0; q < kB; ++q) {
              if (!((pend >> q) & 1u)) continue;
              const int e = tid + NT * (j0 + q);
              bool hit;
              T v;
              if constexpr (kF32) {
                hit = (unsigned)(w0[q] >> 32) == want_tag;
                v = __uint_as_float((uint32_t)w0[q]);
              } else {
                hit = (unsigned)(w0[q] >> 32) == want_tag && (unsigned)(w1[q] >> 32) == want_tag;
                v = __longlong_as_double((long long)(((w1[q] & 0xffffffffull) << 32) | (w0[q] & 0xffffffffull)));
              }
              if (hit) {
                if (j0 == 0 && q < kRepJR) yr[q < kRepJR ? q : 0] = v;
                else Yb[e] = v;
                pend &= ~(1u << q);
              }
            }
            if (!pend) break;
            if (!started) {
              t0 = clock64();
              started = true;
            } else if (clock64() - t0 > wait_lim) {
              fail = true;
              break;
            }
            __nanosleep(64);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < kRepJR; ++j) {
          const int e = tid + NT * j;
          if (e < PM) yr[j] = Yb[e];
        }
      }
    }
    const bool upd = got_y && my_inst;
    // u <- u + (d dbeta - y), TwoSum in float32
    auto u_update = [&](T& uh, T& ul, T dnp, T y) {
      if (!upd) return;
      const T incr = fma(my_d, dnp, -y);
      // an instance whose dbeta was zero (y == 0 exactly) keeps its u bit
      // for bit, however the instances are grouped into tasks
      if (incr == T(0)) return;
      if constexpr (kF32) {
        const T h = uh;
        const T s1 = h + incr, bb = s1 - h;
        const T e = (h - (s1 - bb)) + (incr - bb);
        const T lo = ul + e;
        const T hi2 = s1 + lo;
        ul = lo - (hi2 - s1);
        uh = hi2;
      } else {
        uh += incr;
      }
    };
    T lmd = T(0), lmb = T(0);  // this thread's running max |dbeta|, |beta| (instance kq)
    T gmd[M], gmb[M];          // group tasks: per instance
#pragma unroll
    for (int k = 0; k < M; ++k) { gmd[k] = T(0); gmb[k] = T(0); }
    auto gmax = [&](int k, T dn, T bn) {
#pragma unroll
      for (int kk = 0; kk < M; ++kk)
        if (kk == k) { gmd[kk] = fmax(gmd[kk], fabs(dn)); gmb[kk] = fmax(gmb[kk], fabs(bn)); }
    };
    if (final_pass) {
      // the pending dbeta applied to u, for a resumed launch to continue from
#pragma unroll
      for (int j = 0; j < kRepJR; ++j) {
        const int e = tid + NT * j;
        if (e < PM) {
          u_update(r_uh[j], r_ul[j], has_group ? Dp[dpos<T, M>(e / M, kq)] : r_dn[j], yr[j]);
          uhs[e] = r_uh[j];
          uls[e] = r_ul[j];
        }
      }
      for (int j = kRepJR; j < nJ; ++j) {
        const int e = tid + NT * j;
        if (e >= PM) break;
        T uh = uhs[e], ul = uls[e];
        u_update(uh, ul, Dp[dpos<T, M>(e / M, kq)], got_y ? Yb[e] : T(0));
        uhs[e] = uh; uls[e] = ul;
      }
      break;
    }
    if (!has_group) {
      auto scalar_step = [&](T& uh, T& ul, T& bv, T wt, T dnp, T y) -> T {
        u_update(uh, ul, dnp, y);
        T dn = T(0);
        if (my_inst) {
          if (!my_done) {
            const T bn = thr_scalar<T>(my_kind, uh, wt * my_lam, my_alpha, my_gamma, my_d);
            dn = bn - bv;
            bv = bn;
            lmd = fmax(lmd, fabs(dn));
            lmb = fmax(lmb, fabs(bn));
          } else {
            lmb = fmax(lmb, fabs(bv));
          }
        }
        return dn;
      };
#pragma unroll
      for (int j = 0; j < kRepJR; ++j) {
        const int e = tid + NT * j;
        if (e < PM) {
          const T dn = scalar_step(r_uh[j], r_ul[j], r_b[j], r_w[j], r_dn[j], yr[j]);
          r_dn[j] = dn;
          Dn[dpos<T, M>(e / M, kq)] = dn;
        }
      }
      for (int j = kRepJR; j < nJ; ++j) {
        const int e = tid + NT * j;
        if (e >= PM) break;
        const int i = e / M;
        T uh = uhs[e], ul = uls[e], bv = bes[e];
        const T dn = scalar_step(uh, ul, bv, weight(i), Dp[dpos<T, M>(i, kq)], got_y ? Yb[e] : T(0));
        uhs[e] = uh; uls[e] = ul; bes[e] = bv;
        Dn[dpos<T, M>(i, kq)] = dn;
      }
    } else {
      // Group tasks keep beta and dbeta in shared memory (the group step
      // writes them by group, not by thread); u stays in this thread's
      // registers and its shared copy feeds the norms.
      // ---- C1. u update of every element; scalar instances of the task are
      // thresholded here too
      auto c1 = [&](T& uh, T& ul, int e, T y) {
        const int i = e / M;
        u_update(uh, ul, Dp[dpos<T, M>(i, kq)], y);
        uhs[e] = uh;
        if (my_inst && my_kind < OEM_GROUP_LASSO) {
          const T bv = bes[e];
          T dn = T(0);
          if (!my_done) {
            const T bn = thr_scalar<T>(my_kind, uh, weight(i) * my_lam, my_alpha, my_gamma, my_d);
            dn = bn - bv;
            bes[e] = bn;
            gmax(kq, dn, bn);
          } else {
            gmax(kq, T(0), bv);
          }
          Dn[dpos<T, M>(i, kq)] = dn;
        }
      };
#pragma unroll
      for (int j = 0; j < kRepJR; ++j) {
        const int e = tid + NT * j;
        if (e < PM) c1(r_uh[j], r_ul[j], e, yr[j]);
      }
      for (int j = kRepJR; j < nJ; ++j) {
        const int e = tid + NT * j;
        if (e >= PM) break;
        T uh = uhs[e], ul = uls[e];
        c1(uh, ul, e, got_y ? Yb[e] : T(0));
        uls[e] = ul;
      }
      __syncthreads();
      if (!*long_grp) {
        // ---- C2. one warp per slot of whole groups (Section 2.2: Eqs.
        // glasso, gmcp, gscad, sglasso need ||u_g||, or ||v_g|| with
        // v = S(u, w lambda tau) / d): the squares summed by a segmented
        // warp scan over each group's lanes, then every lane's update
        for (int k = 0; k < M; ++k) {
          if (k >= m) break;
          int kd = OEM_LASSO;
          T lamk = T(0), alk = T(1), gak = T(3), dkk = T(1);
          int dnk = 1;
#pragma unroll
          for (int kk = 0; kk < M; ++kk)
            if (kk == k) { kd = kind[kk]; lamk = lamv[kk]; alk = alpha[kk]; gak = gamma[kk]; dkk = dk[kk]; dnk = done[kk]; }
          if (kd < OEM_GROUP_LASSO) continue;
          const float* w32k = tk.pens[k].w32;
          const double* w64k = tk.pens[k].w64;
          for (int sl = warp; sl < gsn[k]; sl += NW) {
            const uint32_t info = gsl[((size_t)k * gsm + sl) * 32 + lane];
            const bool valid = info != 0xFFFFFFFFu;
            const int i = (int)(info & 0xFFFFu);
            const int st = valid ? (int)((info >> 16) & 31u) : lane;
            const int en = valid ? (int)((info >> 21) & 31u) : lane;
            const int e = i * M + k;
            const T u = valid ? uhs[e] : T(0);
            T wt = T(1);
            if constexpr (kF32) { if (valid && w32k) wt = (T)w32k[i]; }
            else { if (valid && w64k) wt = (T)w64k[i]; }
            T v = u;
            if (kd == OEM_SPARSE_GROUP_LASSO) v = fmax(fabs(u) - wt * lamk * alk, T(0)) / dkk;
            T sc = v * v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const T tq = __shfl_up_sync(0xffffffffu, sc, o);
              if (lane - o >= st) sc += tq;
            }
            const T nrm = sqrt(__shfl_sync(0xffffffffu, sc, en));
            if (!valid) continue;
            const T bv = bes[e];
            if (dnk) {
              Dn[dpos<T, M>(i, k)] = T(0);
              gmax(k, T(0), bv);
              continue;
            }
            const T cgv = cgs[(size_t)k * p + i];
            T bn;
            if (kd == OEM_GROUP_LASSO) {
              const T f = nrm > T(0) ? T(1) - cgv * lamk / nrm : T(0);
              bn = f > T(0) ? u / dkk * f : T(0);
            } else if (kd == OEM_GROUP_MCP || kd == OEM_GROUP_SCAD) {
              // Eqs. gmcp / gscad: the scalar rule on the norm, u's direction
              const T bnorm = nrm > T(0) ? thr_scalar<T>(kd == OEM_GROUP_MCP ? OEM_MCP : OEM_SCAD, nrm,
                                                         cgv * lamk, alk, gak, dkk)
                                         : T(0);
              bn = nrm > T(0) ? u * (bnorm / nrm) : T(0);
            } else {
              // reading of Eq. sglasso: the group step shrinks v by c_k lambda (1 - tau) / d
              const T vv = copysign(v, u);
              const T f = nrm > T(0) ? T(1) - cgv * lamk * (T(1) - alk) / (dkk * nrm) : T(0);
              bn = f > T(0) ? vv * f : T(0);
            }
            const T dn = bn - bv;
            bes[e] = bn;
            Dn[dpos<T, M>(i, k)] = dn;
            gmax(k, dn, bn);
          }
        }
      } else {
        // ---- groups longer than a warp: norms by one thread per group,
        // then every element's update
        for (int e2 = tid; e2 < PM; e2 += NT) {
          const int len = gls[e2];
          if (len == 0) continue;
          const int k = e2 / p, i = e2 % p;
          int kd = OEM_LASSO;
          T lt = T(0), dd = T(1);
#pragma unroll
          for (int kk = 0; kk < M; ++kk)
            if (kk == k) { kd = kind[kk]; lt = lamv[kk] * alpha[kk]; dd = dk[kk]; }
          const float* gw32 = kd == OEM_SPARSE_GROUP_LASSO ? tk.pens[k].w32 : nullptr;
          const double* gw64 = kd == OEM_SPARSE_GROUP_LASSO ? tk.pens[k].w64 : nullptr;
          T s2 = T(0);
          for (int q = 0; q < len; ++q) {
            const T u = uhs[(i + q) * M + k];
            if (kd == OEM_SPARSE_GROUP_LASSO) {
              T wq = T(1);
              if constexpr (kF32) { if (gw32) wq = (T)gw32[i + q]; }
              else { if (gw64) wq = (T)gw64[i + q]; }
              const T v = fmax(fabs(u) - wq * lt, T(0)) / dd;
              s2 = fma(v, v, s2);
            } else {
              s2 = fma(u, u, s2);
            }
          }
          s2 = sqrt(s2);
          for (int q = 0; q < len; ++q) gns[e2 + q] = s2;
        }
        __syncthreads();
        for (int j = 0; j < nJ; ++j) {
          const int e = tid + NT * j;
          if (e >= PM) break;
          if (!my_inst || my_kind < OEM_GROUP_LASSO) continue;
          const int i = e / M, g2 = kq * p + i;
          const T bv = bes[e];
          if (my_done) {
            Dn[dpos<T, M>(i, kq)] = T(0);
            gmax(kq, T(0), bv);
            continue;
          }
          const T u = uhs[e], nrm = gns[g2], cgv = cgs[g2];
          T bn;
          if (my_kind == OEM_GROUP_LASSO) {
            const T f = nrm > T(0) ? T(1) - cgv * my_lam / nrm : T(0);
            bn = f > T(0) ? u / my_d * f : T(0);
          } else if (my_kind == OEM_GROUP_MCP || my_kind == OEM_GROUP_SCAD) {
            const T bnorm = nrm > T(0) ? thr_scalar<T>(my_kind == OEM_GROUP_MCP ? OEM_MCP : OEM_SCAD, nrm,
                                                       cgv * my_lam, my_alpha, my_gamma, my_d)
                                       : T(0);
            bn = nrm > T(0) ? u * (bnorm / nrm) : T(0);
          } else {
            const T v = copysign(fmax(fabs(u) - weight(i) * my_lam * my_alpha, T(0)) / my_d, u);
            const T f = nrm > T(0) ? T(1) - cgv * my_lam * (T(1) - my_alpha) / (my_d * nrm) : T(0);
            bn = f > T(0) ? v * f : T(0);
          }
          const T dn = bn - bv;
          bes[e] = bn;
          Dn[dpos<T, M>(i, kq)] = dn;
          gmax(kq, dn, bn);
        }
      }
    }
    // ---- D. block maxima per instance: every CTA holds all rows, so these
    // are the task's maxima
    if (has_group) {
      float* lr = lred + (size_t)(t & 1) * NW * 2 * M;
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const T a1 = warp_max(gmd[k]), a2 = warp_max(gmb[k]);
        if (lane == 0) {
          lr[(warp * M + k) * 2] = to_red(a1);
          lr[(warp * M + k) * 2 + 1] = to_red(a2);
        }
      }
    } else {
#pragma unroll
      for (int o = M; o < 32; o <<= 1) {
        lmd = fmax(lmd, __shfl_xor_sync(0xffffffffu, lmd, o));
        lmb = fmax(lmb, __shfl_xor_sync(0xffffffffu, lmb, o));
      }
      float* lr = lred + (size_t)(t & 1) * NW * 2 * M;
      if (lane < M) {
        lr[(warp * M + lane) * 2] = to_red(lmd);
        lr[(warp * M + lane) * 2 + 1] = to_red(lmb);
      }
    }
    if (__syncthreads_or(fail ? 1 : 0)) {
      fail = true;
      break;
    }
    float mx[2 * M];
    {
      const float* lr = lred + (size_t)(t & 1) * NW * 2 * M;
      constexpr int E = 2 * M;
      float v = 0.f;
      for (int e = lane; e < NW * E; e += 32) v = fmax(v, lr[e]);  // e % E == lane % E
#pragma unroll
      for (int o = E; o < 32; o <<= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
#pragma unroll
      for (int q = 0; q < E; ++q) mx[q] = __shfl_sync(0xffffffffu, v, q);
    }
    // ---- decisions (every thread, same data, same result)
    int anyd = 0;
    all_done = 1;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      if (k >= m || done[k]) continue;
      const T md = (T)mx[2 * k], mb = (T)mx[2 * k + 1];
      if (md > T(0)) anyd = 1;
      const int it = ++its[k];
      const bool conv = md <= tol * fmax(T(1), mb);
      if (conv || it >= P.max_iter) {
        const int l = lidx[k];
        if (rank == 0 && tid == 0) {
          const size_t o = (size_t)k * L + l;
          tk.iters[o] = it;
          tk.conv[o] = conv ? 1 : 0;
          if (!conv) atomicOr(P.dstatus, kStatNotConv);
        }
        if (k == kq) {  // this CTA writes the rows of its slice
          double* out = tk.beta + ((size_t)k * L + l) * p;
#pragma unroll
          for (int j = 0; j < kRepJR; ++j) {
            const int e = tid + NT * j, i = e / M;
            if (e < PM && i >= i0 && i < i0 + R) out[i] = (double)(has_group ? bes[e] : r_b[j]);
          }
          for (int j = kRepJR; j < nJ; ++j) {
            const int e = tid + NT * j, i = e / M;
            if (e >= PM) break;
            if (i >= i0 && i < i0 + R) out[i] = (double)bes[e];
          }
        }
        its[k] = 0;
        lidx[k] = l + 1;
        if (l + 1 >= L) done[k] = 1;
        else lamv[k] = (T)tk.lam[(size_t)k * L + l + 1];
      }
      all_done &= done[k];
    }
    skip_mv = !anyd;
#pragma unroll
    for (int k = 0; k < M; ++k)
      if (k == kq) { my_lam = lamv[k]; my_done = done[k]; }
    ++t;
    ++loops;
    if (!all_done && P.max_loops > 0 && loops >= P.max_loops) {
      if (tk.st_u && !skip_mv) final_pass = true;
      else break;
    }
  }
  if (__syncthreads_or(fail ? 1 : 0) && tid == 0) atomicOr(P.dstatus, kStatTimeout);
  // ---- save the state for a later launch (serving): each CTA its slice
  if (tk.st_u) {
#pragma unroll
    for (int j = 0; j < kRepJR; ++j) {
      const int e = tid + NT * j, i = e / M;
      if (e < PM) {
        uhs[e] = r_uh[j];
        uls[e] = r_ul[j];
        if (!has_group) bes[e] = r_b[j];
      }
      (void)i;
    }
    for (int j = 0; j < nJ; ++j) {
      const int e = tid + NT * j, i = e / M;
      if (e >= PM) break;
      if (my_inst && i >= i0 && i < i0 + R) {
        const size_t o = (size_t)kq * p + i;
        tk.st_u[2 * o] = (double)uhs[e];
        tk.st_u[2 * o + 1] = (double)uls[e];
        tk.st_beta[o] = (double)bes[e];
      }
    }
    if (rank == 0 && tid == 0) {
      for (int k = 0; k < m; ++k) {
        tk.st_ctl[k * 4 + 0] = lidx[k];
        tk.st_ctl[k * 4 + 1] = its[k];
        tk.st_ctl[k * 4 + 2] = done[k];
      }
      int fin = 1;
      for (int k = 0; k < m; ++k) fin &= done[k];
      tk.st_ctl[32] = fin;
    }
  }
  if (tk.fin_out && rank == 0 && tid == 0) *tk.fin_out = all_done;
  if constexpr (!kGrid)
    cluster.sync();  // no CTA leaves while a peer could still address its shared memory
}

size_t oem_iter_smem_fixed(int p, int M, int max_rows, int precision, bool grid, bool groups) {
  const int tsz = precision == OEM_ITER_F64 ? 8 : 4;
  (void)max_rows;
  return rep_smem_layout(p, oem_iter_mpad(M), tsz, grid, groups, 0).total;
}

size_t oem_iter_smem_per_row(int p, int precision) {
  const int tsz = precision == OEM_ITER_F64 ? 8 : 4;
  return (size_t)((p + 3) & ~3) * tsz;
}

size_t oem_iter_xbuf_bytes(int p, int M, int precision) {
  const int W = precision == OEM_ITER_F64 ? 2 : 1;
  return (2 * (size_t)p * oem_iter_mpad(M) * W * 8 + 255) & ~(size_t)255;
}

template <typename T, int M, bool kGrid, int RG, bool kLong>
static cudaError_t launch_t(const IterLaunch& P, cudaStream_t s, bool query, int* out) {
  constexpr int NT = rep_threads(kLong);
  auto kfn = oem_iter_kernel<T, M, NT, kGrid, RG, kLong>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(P.ntasks * P.C));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = P.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if constexpr (kGrid) {
    if (query) {
      int n = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kfn, NT, P.smem);
      *out = (e == cudaSuccess) ? n : 0;
      return e;
    }
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident, or no launch
    attr[0].val.cooperative = 1;
  } else {
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query) {
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kfn, &cfg);
    *out = (e == cudaSuccess) ? n : 0;
    return e;
  }
  return cudaLaunchKernelEx(&cfg, kfn, P);
}

// Row group: 16 / M rows, or 4 when no warp owns more than 4 rows (the
// instances then fill fewer sums per lane and no load is wasted); long rows
// (IterLaunch::wide, float32, at most 2 instances per task): 512 threads,
// one row per warp.
template <typename T, int M, bool kGrid>
static cudaError_t dispatch_w(const IterLaunch& P, cudaStream_t s, bool q, int* out) {
  if constexpr (sizeof(T) == 4 && M <= 2) {
    if (P.wide) return launch_t<T, M, kGrid, 1, true>(P, s, q, out);
  }
  constexpr int RGF = 16 / M;
  if constexpr (RGF > 4) {
    constexpr int NW = rep_threads(false) / 32;
    if ((P.max_rows + NW - 1) / NW <= 4) return launch_t<T, M, kGrid, 4, false>(P, s, q, out);
  }
  return launch_t<T, M, kGrid, RGF, false>(P, s, q, out);
}
template <typename T, int M>
static cudaError_t dispatch_g(const IterLaunch& P, cudaStream_t s, bool q, int* out) {
  return P.grid ? dispatch_w<T, M, true>(P, s, q, out) : dispatch_w<T, M, false>(P, s, q, out);
}
template <typename T>
static cudaError_t dispatch_m(const IterLaunch& P, cudaStream_t s, bool q, int* out) {
  switch (P.M) {
    case 1: return dispatch_g<T, 1>(P, s, q, out);
    case 2: return dispatch_g<T, 2>(P, s, q, out);
    case 4: return dispatch_g<T, 4>(P, s, q, out);
    default: return dispatch_g<T, 8>(P, s, q, out);
  }
}

int oem_iter_max_cluster(const IterLaunch& P0) {
  IterLaunch P = P0;
  int n = 0;
  cudaError_t e = (P.precision == OEM_ITER_F64) ? dispatch_m<double>(P, 0, true, &n)
                                                : dispatch_m<float>(P, 0, true, &n);
  if (e != cudaSuccess) { cudaGetLastError(); return 0; }
  return n;
}

cudaError_t launch_oem_iter(const IterLaunch& P, cudaStream_t s) {
  if (P.precision == OEM_ITER_F64) return dispatch_m<double>(P, s, false, nullptr);
  return dispatch_m<float>(P, s, false, nullptr);
}

}  // namespace oem
