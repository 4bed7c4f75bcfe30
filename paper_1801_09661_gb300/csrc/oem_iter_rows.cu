// The OEM iteration (Section 2.1 Step 2, Section 2.2 updates) for every
// (Gram, penalty) instance, warm-started along each instance's lambda grid:
// the row-owned kernel, used where the replicated kernel of oem_iter.cu does
// not fit (p above kIterRepMaxP: u, beta and dbeta of all rows would not fit
// in one CTA's shared memory).
//
// Per instance and iteration: u = c + d beta - G beta; beta <- threshold(u).
// The code carries u itself and updates it by the change of beta,
//   u_{t+1} = u_t + d (beta_{t+1} - beta_t) - G (beta_{t+1} - beta_t),
// which is the same quantity; the mat-vec then acts on a vector that shrinks
// as the iteration converges, so float32 products stay accurate, and u is
// kept as a float32 (hi, lo) pair so its rounding does not accumulate.
//
// One thread-block cluster per task (a Gram with its instances; tasks of one
// launch may differ in p). CTA r of the cluster owns rows [slice[r],
// slice[r+1]) of G, u and beta; inside the CTA every warp owns a contiguous
// block of those rows (aligned to group starts for the group penalties).
// Float32 iteration, per iteration and warp (lane = row):
//   1. y_i = (G dbeta)_i for every instance over the list of 16-column
//      blocks of dbeta that hold a nonzero value, in increasing column order
//      with one accumulator per column of each 4-column unit (a zero unit is
//      skipped: it would add exact zeros), so the sums depend on the nonzero
//      units only and every layout gives the same bits; G's blocks come from
//      a cache in shared memory, filled from L2 by the first mat-vec that
//      needs them (blocks beyond its slots are read from L2 each time); then
//      the u update and, without groups, the threshold;
//   2. for group penalties, windows of 32 rows that start at a group start
//      and hold whole groups: the group norms by segmented warp scans, then
//      the group steps;
//   3. its dbeta rows and its own maxima (max|dbeta|, max|beta| per
//      instance) go to every CTA of the cluster as st.async stores counted
//      on the receiver's mbarrier for that buffer, then the warp arrives on
//      its own CTA's barrier (warp 0 arms it with every byte the peers send);
//   4. every warp waits (bounded) for the bytes addressed to its CTA, builds
//      its words of the next buffer's block list (giving cache slots to
//      blocks that are new), and warp 0 takes the maxima over the C x 8
//      warps' entries; one block barrier, then every thread takes the same
//      convergence decisions from the same values.
// Float64 iteration: a warp forms (G dbeta)_i RG rows at a time (lane l
// takes columns l, l + 32, ...; one reduce-scatter per row group) from the
// rows resident in shared memory or from L2; plain DSMEM stores, a DSMEM
// atomic max of the CTA's maxima into every CTA's slot (order-preserving
// 32-bit images) and one cluster barrier per iteration. A launch may stop
// after a loop budget and save its state (serving), to be resumed by a later
// launch.
//
// Grid mode (the slices of one cluster, at most 16 SMs, cannot keep the
// Gram's blocks in shared memory, but those of C > 16 CTAs can): the C CTAs
// of a task are an ordinary group of a cooperative launch, one per SM. Each
// iteration a CTA writes its rows of the new dbeta and its maxima to global
// memory as 64-bit words tagged with the exchange number, and polls (bounded)
// for every CTA's words of this exchange; the arithmetic is the same as in
// cluster mode.
#include "oem_internal.cuh"
#include "iter_common.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace oem {


// Threads per CTA. Every warp reads the whole dbeta once per group of its
// rows, so more warps than needed to spread a CTA's rows only add
// shared-memory traffic.
template <typename T, int M>
constexpr int iter_threads() { return 256; }

// Shared-memory carve-up (byte offsets, 16-byte aligned). The dbeta buffers
// have ldd rows (iter_ldd); rows p.. stay zero. Float64: the Gram
// region holds the first smem_rows rows of the CTA's slice of G. Float32:
// it holds the column-block cache: ucache slots, each one block of 16
// columns (four 16-byte units) of every row of the slice ([slot][unit][row]);
// nzl[b] lists the column blocks of dbeta buffer b that hold a nonzero value
// of some instance, in increasing order (entry: the block, and its slot's
// offset in float4 | nonzero units << 26 | state << 30, state 0 cached, 1 to
// be filled by the mat-vec that reads it, 2 without a slot), the blocks of
// word s (blocks 32 s .. 32 s + 31) at entries 32 s + k, nzc[b][s] of them; cbit[s] has bit l set when block
// 32 s + l has been given a slot (or refused one); smap[k] is block k's slot
// (-1: none).
struct IterSmem {
  size_t dbuf, uhi, ulo, beta, w, cgr, glen, st, lred, red, xbar, xslot, xred, nzc, nzl, cbit, smap, gs, total;
};
constexpr int kIterMaxWarps = 16;
constexpr int kRowsWarps = 8;  // warps of the row-owned kernel (256 threads)
__host__ __device__ inline int iter_units(int p) { return (p + 3) >> 2; }     // 4 columns
__host__ __device__ inline int iter_blocks(int p) { return (p + 15) >> 4; }    // 16 columns
__host__ __device__ inline int iter_block_words(int p) { return (iter_blocks(p) + 31) >> 5; }
__host__ __device__ inline int iter_list_len(int p) { return 32 * iter_block_words(p); }
constexpr int kMaxBlockSlots = 32767;  // slot + 1 takes 15 bits of a list entry
// Rows of a dbeta buffer: float32 whole 16-column blocks, float64 4 rows.
__host__ __device__ inline int iter_ldd(int p, int tsz) { return tsz == 4 ? (p + 15) & ~15 : (p + 3) & ~3; }
__host__ __device__ inline IterSmem iter_smem_layout(int p, int M, int maxR, int tsz, int smem_rows,
                                                     int ucache = 0) {
  const int ldgs = (p + 3) & ~3, ldd = iter_ldd(p, tsz);
  const int nbk = iter_blocks(p), nwd = iter_block_words(p);
  const bool f32 = tsz == 4;
  IterSmem L;
  size_t o = 0;
  L.dbuf = o;  o = al16(o + (size_t)2 * ldd * M * tsz);
  L.uhi = o;   o = al16(o + (size_t)M * maxR * tsz);
  L.ulo = o;   o = al16(o + (size_t)M * maxR * tsz);
  L.beta = o;  o = al16(o + (size_t)M * maxR * tsz);
  L.w = o;     o = al16(o + (size_t)M * maxR * tsz);
  L.cgr = o;   o = al16(o + (size_t)M * maxR * tsz);
  L.glen = o;  o = al16(o + (size_t)M * maxR * 4);
  L.st = o;    o = al16(o + (size_t)maxR * M * tsz);
  L.lred = o;  o = al16(o + (size_t)kIterMaxWarps * M * 2 * 4);
  L.red = o;   o = al16(o + (size_t)3 * M * 2 * 4);
  L.xbar = o;  o = al16(o + 2 * 8);
  L.xslot = o; o = al16(o + (size_t)2 * 16 * kRowsWarps * M * 2 * 4);
  L.xred = o;  o = al16(o + (size_t)(M * 2 + 1) * 4);
  L.nzc = o;   o = al16(o + (f32 ? (size_t)(2 * nwd + 1) * 4 : 0));
  L.nzl = o;   o = al16(o + (f32 ? (size_t)2 * iter_list_len(p) * 8 : 0));
  L.cbit = o;  o = al16(o + (f32 ? (size_t)nwd * 4 : 0));
  L.smap = o;  o = al16(o + (f32 ? (size_t)nbk * 2 : 0));
  L.gs = o;
  o = al16(o + (f32 ? (size_t)ucache * maxR * 64 : (size_t)smem_rows * ldgs * tsz));
  L.total = o;
  return L;
}

template <typename T, int M, int NT, bool kGrid, int RG>
__global__ void __launch_bounds__(NT, 1) oem_iter_rows_kernel(IterLaunch P) {
  constexpr int NW = NT / 32;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = P.C;
  const int rank = kGrid ? (int)(blockIdx.x % C) : (int)cluster.block_rank();
  const IterTask& tk = P.tasks[blockIdx.x / C];
  const int p = tk.p, L = tk.L, m = tk.npen, maxR = tk.max_rows;
  const int i0 = kGrid ? tk.gslice[rank] : tk.slice[rank];
  const int R = (kGrid ? tk.gslice[rank + 1] : tk.slice[rank + 1]) - i0;
  // grid mode exchange buffer (zeroed before the launch): [2][p M W] tagged
  // words of dbeta, [2][C][2M] tagged words of the CTAs' maxima, then the
  // two words of the start barrier
  constexpr int W = sizeof(T) / 4;
  unsigned long long* const xw = reinterpret_cast<unsigned long long*>(tk.xD);
  unsigned long long* const xm = xw + (size_t)2 * tk.p * M * W;
  unsigned* const xbarg = reinterpret_cast<unsigned*>(xm + (size_t)2 * P.C * 2 * M);
  unsigned bar_gen = 0;
  const long long wait_lim = P.wait_cycles > 0 ? P.wait_cycles : 4000000000LL;
  const int ldgs = (p + 3) & ~3, smem_rows = tk.smem_rows;
  const int ldd = iter_ldd(p, (int)sizeof(T));  // rows of a dbeta buffer
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr bool kF32 = sizeof(T) == 4;

  extern __shared__ __align__(16) unsigned char smem[];
  const int ucs = kF32 ? tk.ucache : 0;  // column-block cache slots
  const IterSmem Ls = iter_smem_layout(p, M, maxR, (int)sizeof(T), tk.smem_rows, ucs);
  T* Dbuf = reinterpret_cast<T*>(smem + Ls.dbuf);
  T* uhi = reinterpret_cast<T*>(smem + Ls.uhi);
  T* ulo = reinterpret_cast<T*>(smem + Ls.ulo);
  T* bet = reinterpret_cast<T*>(smem + Ls.beta);
  T* wv = reinterpret_cast<T*>(smem + Ls.w);
  T* cgr = reinterpret_cast<T*>(smem + Ls.cgr);
  int* glen = reinterpret_cast<int*>(smem + Ls.glen);
  T* st = reinterpret_cast<T*>(smem + Ls.st);
  float* lred = reinterpret_cast<float*>(smem + Ls.lred);  // [warp][2M] block table
  unsigned int* red = reinterpret_cast<unsigned int*>(smem + Ls.red);  // [3][2M] slots
  T* Gs = reinterpret_cast<T*>(smem + Ls.gs);
  const int nwd = iter_block_words(p);  // words of the block bitmaps
  const int nll = iter_list_len(p);
  int* nzc = reinterpret_cast<int*>(smem + Ls.nzc);              // [2][nwd], then the slots given
  uint2* nzl = reinterpret_cast<uint2*>(smem + Ls.nzl);          // [2][nll]
  unsigned* cbit = reinterpret_cast<unsigned*>(smem + Ls.cbit);  // [nwd]
  short* smap = reinterpret_cast<short*>(smem + Ls.smap);        // [blocks]
  float4* ucache = reinterpret_cast<float4*>(smem + Ls.gs);      // [ucs][4][maxR]
  constexpr bool kAsync = kF32 && !kGrid;
  const uint32_t xbar0 = xs_u32(smem + Ls.xbar);  // mbarriers of dbeta buffers 0 / 1
  unsigned int* xslot = reinterpret_cast<unsigned int*>(smem + Ls.xslot);  // [2][C][NW][2M]
  unsigned int* xred = reinterpret_cast<unsigned int*>(smem + Ls.xred);    // [2M], then the timeout flag
  volatile unsigned int* xfail = xred + 2 * M;
  const T* Gglob = kF32 ? reinterpret_cast<const T*>(tk.G32) : reinterpret_cast<const T*>(tk.G64);
  const int ldgg = kF32 ? tk.ldg : p;
  const double* cb = tk.c;
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
      if (pen.kind == OEM_SCAD || pen.kind == OEM_GROUP_SCAD)
        de = fmax(de, (T)(1.01 / (pen.gamma64 - 1.0)));
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

  // ---- this warp's contiguous row block, aligned to allowed boundaries
  int wlo, whi;
  {
    const int per = (R + NW - 1) / NW;
    auto bound = [&](int wi) {
      if (wi <= 0) return 0;
      if (wi >= NW) return R;
      int b = min(R, wi * per);
      if (tk.allowed) while (b < R && !tk.allowed[i0 + b]) ++b;
      return b;
    };
    wlo = bound(warp);
    whi = max(wlo, bound(warp + 1));
  }
  // the mat-vec and u-update rows: float32 (one row per lane) and float64
  // without group penalties the warp's block above; float64 with them an
  // even split (group-aligned blocks would leave most warps idle), the group
  // norms and thresholds then on [wlo, whi) after a block barrier
  int mlo = wlo, mhi = whi;
  if (!kF32 && has_group) {
    const int per = (R + NW - 1) / NW;
    mlo = min(R, warp * per);
    mhi = min(R, mlo + per);
  }

  // ---- initialise u, beta, weights, groups, the G rows kept in shared memory
  for (int e = tid; e < M * maxR; e += NT) {
    const int k = e / maxR, i = e % maxR;
    T hi = T(0), lo = T(0), wt = T(1), cgv = T(0), b0 = T(0);
    int gl = 0;
    if (k < m && i < R) {
      const DevPenalty& pen = tk.pens[k];
      if (tk.resume) {
        const size_t o = (size_t)k * p + i0 + i;
        hi = (T)tk.st_u[2 * o];
        lo = (T)tk.st_u[2 * o + 1];
        b0 = (T)tk.st_beta[o];
      } else {
        const double cv = cb[i0 + i];
        hi = (T)cv;
        lo = (T)(cv - (double)hi);
      }
      if (kF32) { if (pen.w32) wt = (T)pen.w32[i0 + i]; }
      else { if (pen.w64) wt = (T)pen.w64[i0 + i]; }
      if (pen.kind >= OEM_GROUP_LASSO) {
        const int g = pen.grp[i0 + i];
        cgv = (T)pen.cg[g];
        if (i == 0 || pen.grp[i0 + i - 1] != g) {
          int len = 1;
          while (i + len < R && pen.grp[i0 + i + len] == g) ++len;
          gl = len;
        }
      }
    }
    uhi[e] = hi; ulo[e] = lo; bet[e] = b0; wv[e] = wt; cgr[e] = cgv; glen[e] = gl;
  }
  for (int e = tid; e < 2 * ldd * M; e += NT) Dbuf[e] = T(0);
  for (int e = tid; e < maxR * M; e += NT) st[e] = T(0);  // padded instances keep dbeta = 0
  for (int e = tid; e < 3 * M * 2; e += NT) red[e] = 0u;
  static_assert(NT / 32 == kRowsWarps, "warps of the row-owned kernel");
  if (kAsync && tid == 0) {
    // one arrival per warp and phase (warp 0's carries the expected bytes)
    xs_init_n(xbar0, NW);
    xs_init_n(xbar0 + 8, NW);
    *xfail = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if constexpr (kF32) {
    for (int e = tid; e < iter_blocks(p); e += NT) smap[e] = -1;
    for (int e = tid; e < nwd; e += NT) cbit[e] = 0u;
    for (int e = tid; e < 2 * nwd + 1; e += NT) nzc[e] = 0;
  } else {
    for (int e = tid; e < smem_rows * ldgs; e += NT) {
      const int i = e / ldgs, j = e % ldgs;
      Gs[e] = (i < R && j < p) ? Gglob[(size_t)(i0 + i) * ldgg + j] : T(0);
    }
  }
  if constexpr (kGrid) {
    if (!group_barrier(xbarg, (unsigned)C, bar_gen, wait_lim)) {
      if (tid == 0) atomicOr(P.dstatus, kStatTimeout);
      return;
    }
  } else {
    cluster.sync();  // every CTA initialised before any DSMEM access
  }

  // Float64 lane roles in the row-group mat-vec: a group is RG rows (V = RG M sums);
  // after the reduce-scatter lane l holds the sum of value v = l / S,
  // S = 32 / V, i.e. row rsub = v / M of the group and instance kq = v % M
  // (the first lane of each group of S acts).
  constexpr int V = RG * M, S = 32 / V;
  static_assert(V == 4 || V == 8 || V == 16, "row group");
  const int vq = lane / S, rsub = vq / M, kq = vq % M;
  const bool even = (lane % S) == 0;
  int my_kind = OEM_LASSO;
  T my_alpha = T(1), my_gamma = T(3), my_d = T(1), my_lam = T(0);
  int my_done = 1;
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (k == kq) {
      my_kind = kind[k]; my_alpha = alpha[k]; my_gamma = gamma[k]; my_d = dk[k];
      my_lam = lamv[k]; my_done = done[k];
    }
  const bool my_inst = kq < m;

  const T tol = (T)P.tol;
  // Float32 mat-vec of local rows [r0, r0 + 32) (lane = row i = r0 + lane,
  // active when in): y_i = (G dbeta)_i for every instance over the 16-column
  // blocks whose dbeta has a nonzero value (the list of buffer Db), in
  // increasing column order, one accumulator per column within each 4-column
  // unit; the caller adds (a0 + a1) + (a2 + a3). A zero unit adds exact
  // zeros (fma(g, 0, a) = a for finite g), so the sums are those of every
  // nonzero unit in increasing order, whatever the layout. G from the
  // block's cache slot, filled from L2 by the first mat-vec that needs it;
  // blocks without a slot are read from L2 each time.
  const int nu_all = iter_units(p);
  auto rows_matvec = [&](int r0, bool in, const T* Db, int b, float (&a)[M][4]) {
    const int i = r0 + lane;
    const int ii = in ? i : r0;  // a lane past the slice reads a valid row, unused
    const float* grow = reinterpret_cast<const float*>(Gglob) + (size_t)(i0 + ii) * ldgg;
    const float* Dbf = reinterpret_cast<const float*>(Db);
    // dbeta of block kb: units 4 kb + j, instances q
    auto load_dv = [&](int kb, float (&dv)[4][4][M]) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < M; ++q) {
          const int uu = (4 * kb + j) * M + q;
          const float4 tq = *reinterpret_cast<const float4*>(Dbf + ((uu ^ ((uu >> 3) & (M - 1))) << 2));
          const float tv[4] = {tq.x, tq.y, tq.z, tq.w};
#pragma unroll
          for (int c = 0; c < 4; ++c) dv[j][(q * 4 + c) / M][(q * 4 + c) % M] = tv[c];
        }
    };
    auto fma_block = [&](const float4 (&g)[4], const float (&dv)[4][4][M]) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float gv[4] = {g[j].x, g[j].y, g[j].z, g[j].w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < M; ++k) a[k][c] = fma(gv[c], dv[j][c][k], a[k][c]);
      }
    };
    // any entry: cached, to be filled from L2 (units past p give zeros), or
    // without a slot (read from L2)
    auto block_any = [&](uint2 e) {
      const int kb = (int)e.x;
      const unsigned st2 = e.y >> 30, off = e.y & 0x3FFFFFFu;
      float dv[4][4][M];
      load_dv(kb, dv);
      float4 g[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int u = 4 * kb + j;
        float4* cp = ucache + off + (size_t)j * maxR + ii;
        if (st2 == 0u) {
          g[j] = *cp;
        } else {
          g[j] = u < nu_all ? *reinterpret_cast<const float4*>(grow + 4 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
          if (st2 == 1u && in) *cp = g[j];
        }
      }
      fma_block(g, dv);
    };
    constexpr int UB = M <= 2 ? 2 : 1;  // cached blocks whose loads are in flight together
    for (int sw = 0; sw < nwd; ++sw) {
    const uint2* lst = nzl + (size_t)b * nll + 32 * sw;
    const int cnt = nzc[b * nwd + sw];
    int q = 0;
    if constexpr (UB == 2) {
      for (; q + 2 <= cnt; q += 2) {
        const uint4 e2 = *reinterpret_cast<const uint4*>(lst + q);
        if (((e2.y | e2.w) >> 30) == 0u) {
          // two cached blocks; a unit whose dbeta is zero for every
          // instance (flag clear) is neither loaded nor added: its terms are
          // exact zeros
          float dv[2][4][4][M];
          float4 g[2][4];
          const unsigned ey[2] = {e2.y, e2.w}, ex[2] = {e2.x, e2.z};
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const bool on = (ey[h] >> (26 + j)) & 1u;
              g[h][j] = on ? ucache[(ey[h] & 0x3FFFFFFu) + (size_t)j * maxR + ii] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int q = 0; q < M; ++q) {
                const int uu = (4 * (int)ex[h] + j) * M + q;
                const float4 tq = on ? *reinterpret_cast<const float4*>(Dbf + ((uu ^ ((uu >> 3) & (M - 1))) << 2))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                const float tv[4] = {tq.x, tq.y, tq.z, tq.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) dv[h][j][(q * 4 + c) / M][(q * 4 + c) % M] = tv[c];
              }
            }
          fma_block(g[0], dv[0]);
          fma_block(g[1], dv[1]);
        } else {
          block_any(make_uint2(e2.x, e2.y));
          block_any(make_uint2(e2.z, e2.w));
        }
      }
    }
    for (; q < cnt; ++q) block_any(lst[q]);
    }
  };
  // Float32, one warp: word sw of the list of 16-column blocks of dbeta
  // buffer b with a nonzero value (every CTA's rows have arrived), giving a
  // cache slot to each block that is nonzero for the first time (while
  // slots last; its entry is marked to be filled by the mat-vec that reads
  // it). Which block gets which slot does not change any result.
  int* const nslot = nzc + 2 * nwd;  // slots given so far
  auto build_word = [&](int b, int sw) {
    const float* Db = reinterpret_cast<const float*>(Dbuf) + (size_t)b * ldd * M;
    const int kb = 32 * sw + lane;
    unsigned fl = 0u;  // the block's nonzero 4-column units
    int slv = -1;
    if (kb < iter_blocks(p)) {
      // whole blocks: buffer rows past p are zero
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t o = 0u;
#pragma unroll
        for (int q = 0; q < M; ++q) {
          const int uu = (4 * kb + j) * M + q;
          const float4 v = *reinterpret_cast<const float4*>(Db + ((uu ^ ((uu >> 3) & (M - 1))) << 2));
          o |= __float_as_uint(v.x) | __float_as_uint(v.y) | __float_as_uint(v.z) | __float_as_uint(v.w);
        }
        fl |= ((o & 0x7fffffffu) != 0u ? 1u : 0u) << j;
      }
      slv = smap[kb];
    }
    const unsigned cb = cbit[sw];
    const unsigned bits = __ballot_sync(0xffffffffu, fl != 0u);
    const unsigned nb = bits & ~cb;
    const unsigned lt = (1u << lane) - 1u;
    unsigned state = slv >= 0 ? 0u : 2u;
    if (nb) {  // blocks nonzero for the first time
      int base = 0;
      if (lane == 0) base = atomicAdd(nslot, __popc(nb));
      base = __shfl_sync(0xffffffffu, base, 0);
      const int sl = base + __popc(nb & lt);
      if (((nb >> lane) & 1u) && sl < ucs) {
        smap[kb] = (short)sl;
        slv = sl;
        state = 1u;
      }
      if (lane == 0) cbit[sw] = cb | nb;
    }
    if ((bits >> lane) & 1u)
      nzl[(size_t)b * nll + 32 * sw + __popc(bits & lt)] =
          make_uint2((unsigned)kb, (unsigned)(slv >= 0 ? slv * 4 * maxR : 0) | (fl << 26) | (state << 30));
    if (lane == 0) nzc[b * nwd + sw] = __popc(bits);
  };
  int skip_mv = 1;      // dbeta of the previous iteration is all zero
  int all_done = 1;
  for (int k = 0; k < m; ++k) all_done &= done[k];
  int64_t loops = 0;
  int t = 0;
  while (!all_done) {
    const int cur = t & 1, nxt = cur ^ 1;
    const T* Dc = Dbuf + (size_t)cur * ldd * M;
    const int nr = whi - wlo;
    T lmd = T(0), lmb = T(0);  // float64: this lane's running max |dbeta|, |beta| (instance kq)
    T mx_d[M], mx_b[M];        // float32 (and group steps): per instance, this lane's rows
#pragma unroll
    for (int k = 0; k < M; ++k) { mx_d[k] = T(0); mx_b[k] = T(0); }
    if constexpr (kF32) {
      // ---- 1. one row per lane, rows [wlo, whi) in chunks of 32: y = G dbeta
      // for every instance, the u update and, without groups, the threshold
      for (int r0 = wlo; r0 < whi; r0 += 32) {
        const int i = r0 + lane;
        const bool in = i < whi;
        float a[M][4];
#pragma unroll
        for (int k = 0; k < M; ++k)
#pragma unroll
          for (int c = 0; c < 4; ++c) a[k][c] = 0.f;
        if (!skip_mv) rows_matvec(r0, in, Dc, cur, a);
        if (in) {
#pragma unroll
          for (int k = 0; k < M; ++k) {
            if (k >= m) {
              st[(size_t)i * M + k] = T(0);
              continue;
            }
            const int idx = k * maxR + i;
            if (!skip_mv) {
              const T y = (a[k][0] + a[k][1]) + (a[k][2] + a[k][3]);
              const T incr = fma(dk[k], Dc[dpos<T, M>(i0 + i, k)], -y);
              // an instance whose dbeta was zero (y == 0 exactly) keeps its
              // u bit for bit, however the instances are grouped into tasks
              if (incr != T(0)) {
                const T h = uhi[idx];
                const T s1 = h + incr, bb = s1 - h;
                const T e = (h - (s1 - bb)) + (incr - bb);
                const T lo = ulo[idx] + e;
                const T hi2 = s1 + lo;
                ulo[idx] = lo - (hi2 - s1);
                uhi[idx] = hi2;
              }
            }
            if (!has_group) {
              T dn = T(0);
              if (!done[k]) {
                const T bn = thr_scalar<T>(kind[k], uhi[idx], wv[idx] * lamv[k], alpha[k], gamma[k], dk[k]);
                dn = bn - bet[idx];
                bet[idx] = bn;
                mx_d[k] = fmax(mx_d[k], fabs(dn));
                mx_b[k] = fmax(mx_b[k], fabs(bn));
              } else {
                mx_b[k] = fmax(mx_b[k], fabs(bet[idx]));
              }
              st[(size_t)i * M + k] = dn;
            }
          }
        }
      }
      __syncwarp();  // the group steps read u of the warp's own rows
    } else {
      // ---- 1. float64, per group of RG rows: y = G dbeta for all instances
      // (one pass over dbeta for the group; lane l takes columns l, l + 32,
      // ...; one reduce-scatter), u update and, without groups, the threshold
      for (int gb = mlo; gb < mhi; gb += RG) {
        const int nv = min(RG, mhi - gb);
        T y = T(0);
        if (!skip_mv) {
          T acc[V];
#pragma unroll
          for (int q = 0; q < V; ++q) acc[q] = T(0);
          const T* gr[RG];
#pragma unroll
          for (int r = 0; r < RG; ++r) {
            const int ib = gb + min(r, nv - 1);
            gr[r] = ib < smem_rows ? Gs + (size_t)ib * ldgs : Gglob + (size_t)(i0 + ib) * ldgg;
          }
#pragma unroll 4
          for (int j = lane; j < p; j += 32) {
            T dv[M];
            load_col<T, M>(Dc, j, dv);
#pragma unroll
            for (int r = 0; r < RG; ++r) {
              const T g = r < nv ? gr[r][j] : T(0);
#pragma unroll
              for (int k = 0; k < M; ++k) acc[r * M + k] = fma(g, dv[k], acc[r * M + k]);
            }
          }
          y = reduce_scatter<V>(acc, lane);
        }
        const int i = gb + rsub;  // this lane's row (local index)
        if (even && i < mhi) {
          const int idx = kq * maxR + i;
          if (my_inst && !skip_mv) {
            const T incr = fma(my_d, Dc[dpos<T, M>(i0 + i, kq)], -y);
            if (incr != T(0)) uhi[idx] += incr;
          }
          if (!has_group) {
            T dn = T(0);
            if (my_inst) {
              if (!my_done) {
                const T bn = thr_scalar<T>(my_kind, uhi[idx], wv[idx] * my_lam, my_alpha, my_gamma, my_d);
                dn = bn - bet[idx];
                bet[idx] = bn;
                lmd = fmax(lmd, fabs(dn));
                lmb = fmax(lmb, fabs(bn));
              } else {
                lmb = fmax(lmb, fabs(bet[idx]));
              }
            }
            st[(size_t)i * M + kq] = dn;
          }
        }
      }
      if (has_group) __syncthreads();  // every row's u before the group norms
      else __syncwarp();
    }
    if (has_group) {
      // ---- 2. thresholds of the warp's rows [wlo, whi) (group-aligned):
      // per group instance, windows of 32 rows that start at a group start
      // and hold whole groups; ||u_g|| (or ||v_g||, v = S(u, w lambda tau) / d,
      // for the sparse group lasso) by a segmented scan over each group's
      // lanes, whose summation tree depends on the group's length only, so
      // every layout gives the same bits. A group longer than 32 rows is
      // summed in row order by one lane.
#pragma unroll
      for (int k = 0; k < M; ++k) {
        if (k >= m) continue;
        const int kd = kind[k], dnk = done[k];
        const T lamk = lamv[k], alk = alpha[k], gak = gamma[k], dkk = dk[k];
        auto record = [&](int idx, int i, T bn) {
          const T dn = bn - bet[idx];
          bet[idx] = bn;
          mx_d[k] = fmax(mx_d[k], fabs(dn));
          mx_b[k] = fmax(mx_b[k], fabs(bn));
          st[(size_t)i * M + k] = dn;
        };
        auto keep = [&](int idx, int i) {
          mx_b[k] = fmax(mx_b[k], fabs(bet[idx]));
          st[(size_t)i * M + k] = T(0);
        };
        if (kd < OEM_GROUP_LASSO) {  // a scalar instance of a group task
          for (int i = wlo + lane; i < whi; i += 32) {
            const int idx = k * maxR + i;
            if (dnk) keep(idx, i);
            else record(idx, i, thr_scalar<T>(kd, uhi[idx], wv[idx] * lamk, alk, gak, dkk));
          }
          continue;
        }
        // Section 2.2, Eqs. glasso, gmcp, gscad, sglasso
        auto group_step = [&](int idx, int i, T u, T nrm) {
          if (dnk) { keep(idx, i); return; }
          const T cgv = cgr[idx];
          T bn;
          if (kd == OEM_GROUP_LASSO) {
            const T f = nrm > T(0) ? T(1) - cgv * lamk / nrm : T(0);
            bn = f > T(0) ? u / dkk * f : T(0);
          } else if (kd == OEM_GROUP_MCP || kd == OEM_GROUP_SCAD) {
            // the scalar rule on the norm, u's direction
            const T bnorm = nrm > T(0) ? thr_scalar<T>(kd == OEM_GROUP_MCP ? OEM_MCP : OEM_SCAD, nrm,
                                                       cgv * lamk, alk, gak, dkk)
                                       : T(0);
            bn = nrm > T(0) ? u * (bnorm / nrm) : T(0);
          } else {
            // reading of Eq. sglasso: the group step shrinks v by
            // c_k lambda (1 - tau) / d
            const T v = copysign(fmax(fabs(u) - wv[idx] * lamk * alk, T(0)) / dkk, u);
            const T f = nrm > T(0) ? T(1) - cgv * lamk * (T(1) - alk) / (dkk * nrm) : T(0);
            bn = f > T(0) ? v * f : T(0);
          }
          record(idx, i, bn);
        };
        auto vterm = [&](int idx, T u) {
          return kd == OEM_SPARSE_GROUP_LASSO ? fmax(fabs(u) - wv[idx] * lamk * alk, T(0)) / dkk : u;
        };
        int r0 = wlo;
        while (r0 < whi) {
          const int i = r0 + lane;
          const bool in = i < whi;
          const int idx = k * maxR + (in ? i : r0);
          const int len = in ? glen[idx] : 0;
          const unsigned starts = __ballot_sync(0xffffffffu, len > 0);  // lane 0 is a start
          const int mys = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));
          const int myend = mys + __shfl_sync(0xffffffffu, len, mys) - 1;
          const bool fits = in && myend < 32;
          const unsigned nf = __ballot_sync(0xffffffffu, in && !fits);
          if (nf & 1u) {
            // the window's first group is longer than 32 rows
            const int len0 = __shfl_sync(0xffffffffu, len, 0);
            T s2 = T(0);
            if (lane == 0) {
              for (int q = 0; q < len0; ++q) {
                const T v = vterm(idx + q, uhi[idx + q]);
                s2 = fma(v, v, s2);
              }
              s2 = sqrt(s2);
            }
            s2 = __shfl_sync(0xffffffffu, s2, 0);
            for (int q = lane; q < len0; q += 32) {
              const int i2 = r0 + q, id2 = k * maxR + i2;
              group_step(id2, i2, uhi[id2], s2);
            }
            r0 += len0;
            continue;
          }
          const T u = fits ? uhi[idx] : T(0);
          const T v = fits ? vterm(idx, u) : T(0);
          T sc = v * v;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const T tq = __shfl_up_sync(0xffffffffu, sc, o);
            if (lane - o >= mys) sc += tq;
          }
          const T nrm = sqrt(__shfl_sync(0xffffffffu, sc, fits ? myend : lane));
          if (fits) group_step(idx, i, u, nrm);
          r0 += nf ? __ffs(nf) - 1 : 32;
        }
      }
      if constexpr (!kF32) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const T a1 = warp_max(mx_d[k]), a2 = warp_max(mx_b[k]);
          if (k == kq) { lmd = a1; lmb = a2; }
        }
      }
      __syncwarp();
    }
    // ---- 3. DSMEM: dbeta rows to every CTA, maxima into every CTA's slot
    {
      if constexpr (kF32) {
        // by 16-byte units of the buffer: a unit inside the warp's rows goes
        // as one float4 store, a unit shared with a neighbour warp element by
        // element (i0 is a multiple of 4, so st is unit-aligned)
        const int f0 = (i0 + wlo) * M, f1 = (i0 + whi) * M;
        const int u0 = f0 >> 2, nu = ((f1 + 3) >> 2) - u0;
        T* Dn = Dbuf + (size_t)nxt * ldd * M;
        const int CC = C;
        if constexpr (kGrid) {
          // this warp's dbeta words, tagged with the iteration number
          for (int e = f0 + lane; e < f1; e += 32)
            st_tag1(xw + (size_t)nxt * p * M + e, tag_word(__float_as_uint(st[e - i0 * M]), (uint32_t)t + 1u));
        } else if constexpr (kAsync) {
          const uint32_t bar = xbar0 + 8 * nxt;
          for (int e = lane; e < nu * C; e += 32) {
            const int u = u0 + e / C, r = e % C;
            float* dl = Dn + ((u ^ ((u >> 3) & (M - 1))) << 2);
            const float* src = st + (4 * u - i0 * M);
            const bool whole = 4 * u >= f0 && 4 * u + 4 <= f1;
            if (r == rank) {
              if (whole) {
                *reinterpret_cast<float4*>(dl) = *reinterpret_cast<const float4*>(src);
              } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  if (4 * u + q >= f0 && 4 * u + q < f1) dl[q] = src[q];
              }
            } else {
              const uint32_t ra = xs_map(xs_u32(dl), r), rb = xs_map(bar, r);
              if (whole) {
                xs_st4(ra, *reinterpret_cast<const float4*>(src), rb);
              } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  if (4 * u + q >= f0 && 4 * u + q < f1) xs_st1(ra + 4 * q, __float_as_uint(src[q]), rb);
              }
            }
          }
        } else {
          for (int e = lane; e < nu * CC; e += 32) {
            const int u = u0 + e / CC, r = e % CC;
            float* dst = cluster.map_shared_rank(Dn, r) + ((u ^ ((u >> 3) & (M - 1))) << 2);
            const float* src = st + (4 * u - i0 * M);
            if (4 * u >= f0 && 4 * u + 4 <= f1) {
              *reinterpret_cast<float4*>(dst) = *reinterpret_cast<const float4*>(src);
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (4 * u + q >= f0 && 4 * u + q < f1) dst[q] = src[q];
            }
          }
        }
      } else if constexpr (kGrid) {
        for (int e = (i0 + wlo) * M + lane; e < (i0 + whi) * M; e += 32) {
          const unsigned long long bits = (unsigned long long)__double_as_longlong((double)st[e - i0 * M]);
          st_tag2(xw + ((size_t)nxt * p * M + e) * 2, tag_word((uint32_t)bits, (uint32_t)t + 1u),
                  tag_word((uint32_t)(bits >> 32), (uint32_t)t + 1u));
        }
      } else {
        T* Dn = Dbuf + (size_t)nxt * ldd * M;
        for (int e = lane; e < nr * C; e += 32) {
          const int i = wlo + e / C, r = e % C;
          store_row<T, M>(cluster.map_shared_rank(Dn, r), i0 + i, st + (size_t)i * M);
        }
      }
      if constexpr (kAsync) {
        // the warp's maxima per instance into entry [nxt][rank][warp] of
        // every CTA (st.async counted on the peers' barriers); then the
        // warp's arrival on this CTA's barrier, after its own stores (warp 0
        // arms it with every byte the peers send)
        constexpr int E = 2 * M;
        const uint32_t bar = xbar0 + 8 * nxt;
        unsigned int* slw = xslot + (((size_t)nxt * 16 + rank) * NW + warp) * E;
        float mv[E];
#pragma unroll
        for (int k = 0; k < M; ++k) {
          mv[2 * k] = to_red(warp_max(mx_d[k]));
          mv[2 * k + 1] = to_red(warp_max(mx_b[k]));
        }
        for (int e = lane; e < C * E; e += 32) {
          const int r = e / E, q = e % E;
          float val = 0.f;
#pragma unroll
          for (int qq = 0; qq < E; ++qq)
            if (qq == q) val = mv[qq];
          if (r == rank) slw[q] = __float_as_uint(val);
          else xs_st1(xs_map(xs_u32(slw + q), r), __float_as_uint(val), xs_map(bar, r));
        }
        __syncwarp();
        if (lane == 0) {
          // test_stall: four bytes more than the peers send, so the first
          // wait of the launch must run out
          if (warp == 0)
            xs_arm(bar, (uint32_t)(((p - R) * M + (C - 1) * NW * E) * 4) + ((P.test_stall && t == 0) ? 4u : 0u));
          else xs_arrive(bar);
        }
      } else if constexpr (kF32) {
        // the warp's maxima per instance into the block table
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const T a1 = warp_max(mx_d[k]), a2 = warp_max(mx_b[k]);
          if (lane == 0) {
            lred[(warp * M + k) * 2] = to_red(a1);
            lred[(warp * M + k) * 2 + 1] = to_red(a2);
          }
        }
      } else {
        // instance kq's warp maxima end in lane S kq (lanes of one instance
        // differ in the row bits 32 / RG .. 16 of the lane index)
#pragma unroll
        for (int o = 32 / RG; o < 32; o <<= 1) {
          lmd = fmax(lmd, __shfl_xor_sync(0xffffffffu, lmd, o));
          lmb = fmax(lmb, __shfl_xor_sync(0xffffffffu, lmb, o));
        }
        if (even && rsub == 0) {
          lred[(warp * M + kq) * 2] = to_red(lmd);
          lred[(warp * M + kq) * 2 + 1] = to_red(lmb);
        }
      }
    }
    // ---- 3b. (without the asynchronous exchange) warp 0: the block's maxima
    // into slot t % 3 of every CTA (the slot is zeroed after its decisions,
    // two iterations before its reuse)
    if constexpr (!kAsync) __syncthreads();
    if (!kAsync && warp == 0) {
      constexpr int E = 2 * M;  // values per slot
      float v = 0.f;
      if (lane < E)
        for (int w = 0; w < NW; ++w) v = fmax(v, lred[w * E + lane]);
      if constexpr (kGrid) {
        if (lane < E)
          st_tag1(xm + ((size_t)nxt * C + rank) * E + lane, tag_word(__float_as_uint(v), (uint32_t)t + 1u));
      } else {
        unsigned int* slot = red + (size_t)(t % 3) * E;
        for (int base = 0; base < C * E; base += 32) {
          const int e = base + lane, q = e % E;
          const float val = __shfl_sync(0xffffffffu, v, q);
          if (e < C * E && val > 0.f)
            atomicMax(cluster.map_shared_rank(slot + q, e / E), __float_as_uint(val));
        }
      }
    }
    if constexpr (kGrid) {
      // every CTA's dbeta words into this CTA's next buffer, and every CTA's
      // maxima into slot t % 3: loads of a batch in flight at once, the stale
      // ones again after a short pause until their tag is this iteration's
      // test_stall: the first exchange waits for a tag that nobody writes
      const uint32_t want = (uint32_t)t + 1u + ((P.test_stall && t == 0) ? 1u : 0u);
      T* Dn = Dbuf + (size_t)nxt * ldd * M;
      const int nw = p * M, nm = C * 2 * M;
      bool bad = false;
      long long w0c = 0;
      bool started = false;
      constexpr int kB = 8;
      for (int base = tid; base < nw + nm && !bad; base += NT * kB) {
        unsigned long long a0[kB], a1[kB];
        unsigned pend = 0;
#pragma unroll
        for (int q = 0; q < kB; ++q)
          if (base + q * NT < nw + nm) pend |= 1u << q;
        while (pend) {
#pragma unroll
          for (int q = 0; q < kB; ++q) {
            if (!((pend >> q) & 1u)) continue;
            const int e = base + q * NT;
            if (e < nw) {
              if constexpr (sizeof(T) == 4) a0[q] = ld_tag1(xw + (size_t)nxt * nw + e);
              else ld_tag2(xw + ((size_t)nxt * nw + e) * 2, a0[q], a1[q]);
            } else {
              a0[q] = ld_tag1(xm + (size_t)nxt * nm + (e - nw));
            }
          }
#pragma unroll
          for (int q = 0; q < kB; ++q) {
            if (!((pend >> q) & 1u)) continue;
            const int e = base + q * NT;
            bool hit = (uint32_t)(a0[q] >> 32) == want;
            if constexpr (sizeof(T) == 8) { if (e < nw) hit = hit && (uint32_t)(a1[q] >> 32) == want; }
            if (!hit) continue;
            if (e < nw) {
              T v;
              if constexpr (sizeof(T) == 4) v = __uint_as_float((uint32_t)a0[q]);
              else v = __longlong_as_double((long long)(((a1[q] & 0xffffffffull) << 32) | (a0[q] & 0xffffffffull)));
              Dn[dpos<T, M>(e / M, e % M)] = v;
            } else {
              const uint32_t bits = (uint32_t)a0[q];
              if (bits) atomicMax(red + (size_t)(t % 3) * M * 2 + (e - nw) % (2 * M), bits);
            }
            pend &= ~(1u << q);
          }
          if (!pend) break;
          if (!started) {
            w0c = clock64();
            started = true;
          } else if (clock64() - w0c > wait_lim) {
            bad = true;
            break;
          }
          __nanosleep(64);
        }
      }
      if (__syncthreads_or(bad ? 1 : 0)) {
        if (tid == 0) atomicOr(P.dstatus, kStatTimeout);
        break;
      }
      if constexpr (kF32) {
        for (int sw = warp; sw < nwd; sw += NW) build_word(nxt, sw);
        __syncthreads();
      }
    } else if constexpr (kAsync) {
      // every warp waits (bounded) for the bytes addressed to this CTA, then
      // builds its words of the list; warp 0 takes the maxima over the C
      // entries into xred
      {
        constexpr int E = 2 * M;
        const uint32_t bar = xbar0 + 8 * nxt;
        const uint32_t par = (uint32_t)((t >> 1) & 1);
        bool ok = xs_try(bar, par);
        if (!ok) {
          const long long t0 = clock64();
          while (!(ok = xs_try(bar, par)))
            if (clock64() - t0 > wait_lim) break;
        }
        ok = __all_sync(0xffffffffu, ok);
        if (ok)
          for (int sw = warp; sw < nwd; sw += NW) build_word(nxt, sw);
        if (warp == 0) {
          const unsigned int* sl = xslot + (size_t)nxt * 16 * NW * E;
          unsigned int mx = 0u;
          for (int e = lane; e < C * NW * E; e += 32) mx = max(mx, sl[e]);
          for (int o = E; o < 32; o <<= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          if (lane < E) xred[lane] = mx;
        }
        if (lane == 0 && !ok) *xfail = 1u;
      }
      __syncthreads();
      if (*xfail) {
        if (tid == 0) atomicOr(P.dstatus, kStatTimeout);
        break;
      }
    } else {
      cluster.sync();
    }
    // ---- 4. decisions (every thread, same data, same result)
    {
      const unsigned int* slot = kAsync ? xred : red + (size_t)(t % 3) * M * 2;
      int anyd = 0;
      all_done = 1;
#pragma unroll
      for (int k = 0; k < M; ++k) {
        if (k >= m || done[k]) continue;
        const T md = (T)from_red(slot[2 * k]), mb = (T)from_red(slot[2 * k + 1]);
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
          double* out = tk.beta + ((size_t)k * L + l) * p + i0;
          for (int i = wlo + lane; i < whi; i += 32) out[i] = (double)bet[k * maxR + i];
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
      if (tid < M * 2) {
        red[(size_t)((t + 2) % 3) * M * 2 + tid] = 0u;
      }
    }
    ++t;
    ++loops;
    if (P.max_loops > 0 && loops >= P.max_loops) break;
  }
  __syncwarp();
  // ---- save the state for a later launch (serving): apply the pending dbeta
  if (tk.st_u) {
    if (!all_done && !skip_mv) {
      const T* Dc = Dbuf + (size_t)(t & 1) * ldd * M;
      // the same sums as the loop's mat-vec, so that a resumed path is the
      // same as an uninterrupted one
      if constexpr (kF32) {
        for (int r0 = wlo; r0 < whi; r0 += 32) {
          const int i = r0 + lane;
          const bool in = i < whi;
          float a[M][4];
#pragma unroll
          for (int k = 0; k < M; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) a[k][c] = 0.f;
          rows_matvec(r0, in, Dc, t & 1, a);
          if (!in) continue;
#pragma unroll
          for (int k = 0; k < M; ++k) {
            if (k >= m) continue;
            const int idx = k * maxR + i;
            const T y = (a[k][0] + a[k][1]) + (a[k][2] + a[k][3]);
            const T incr = fma(dk[k], Dc[dpos<T, M>(i0 + i, k)], -y);
            if (incr != T(0)) {
              const T h = uhi[idx];
              const T s1 = h + incr, bb = s1 - h;
              const T e = (h - (s1 - bb)) + (incr - bb);
              const T lo = ulo[idx] + e;
              const T hi2 = s1 + lo;
              ulo[idx] = lo - (hi2 - s1);
              uhi[idx] = hi2;
            }
          }
        }
      } else {
        for (int ib = wlo; ib < whi; ++ib) {
          const T* g0 = (ib < smem_rows) ? Gs + (size_t)ib * ldgs : Gglob + (size_t)(i0 + ib) * ldgg;
          T acc[M];
#pragma unroll
          for (int k = 0; k < M; ++k) acc[k] = T(0);
          for (int j = lane; j < p; j += 32) {
            T dv[M];
            load_col<T, M>(Dc, j, dv);
            const T g = g0[j];
#pragma unroll
            for (int k = 0; k < M; ++k) acc[k] = fma(g, dv[k], acc[k]);
          }
#pragma unroll
          for (int k = 0; k < M; ++k) acc[k] = warp_sum(acc[k]);
          if (lane == 0) {
#pragma unroll
            for (int k = 0; k < M; ++k) {
              if (k >= m) continue;
              const T incr = fma(dk[k], Dc[dpos<T, M>(i0 + ib, k)], -acc[k]);
              if (incr != T(0)) uhi[k * maxR + ib] += incr;
            }
          }
        }
      }
      __syncwarp();
    }
    for (int e = lane; e < m * (whi - wlo); e += 32) {
      const int k = e / (whi - wlo), i = wlo + e % (whi - wlo);
      const size_t o = (size_t)k * p + i0 + i;
      tk.st_u[2 * o] = (double)uhi[k * maxR + i];
      tk.st_u[2 * o + 1] = (double)ulo[k * maxR + i];
      tk.st_beta[o] = (double)bet[k * maxR + i];
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

size_t oem_iter_rows_smem_fixed(int p, int npen, int max_rows, int precision) {
  const int M = oem_iter_mpad(npen);
  const int tsz = precision == OEM_ITER_F64 ? 8 : 4;
  return iter_smem_layout(p, M, max_rows, tsz, 0).total;
}

size_t oem_iter_rows_smem_ucache(int p, int npen, int max_rows, int precision, int slots) {
  const int M = oem_iter_mpad(npen);
  const int tsz = precision == OEM_ITER_F64 ? 8 : 4;
  return iter_smem_layout(p, M, max_rows, tsz, 0, slots).total;
}

int oem_iter_rows_ucache_slots(int p, int npen, int max_rows, int precision, size_t cap) {
  if (precision == OEM_ITER_F64) return 0;
  const size_t base = oem_iter_rows_smem_ucache(p, npen, max_rows, precision, 0);
  if (base >= cap) return 0;
  const size_t per = (size_t)max_rows * 64;  // one slot: a 16-column block of every row
  const size_t q = (cap - base) / per;
  return (int)std::min<size_t>(std::min<size_t>(q, (size_t)iter_blocks(p)), (size_t)kMaxBlockSlots);
}

int oem_iter_rows_blocks(int p) { return iter_blocks(p); }

size_t oem_iter_rows_xbuf_bytes(int p, int M, int precision, int C) {
  const size_t W = precision == OEM_ITER_F64 ? 2 : 1, Mp = (size_t)oem_iter_mpad(M);
  return ((2 * (size_t)p * Mp * W + 2 * (size_t)C * 2 * Mp) * 8 + 16 + 255) & ~(size_t)255;
}

size_t oem_iter_rows_smem_per_row(int p, int precision) {
  const int tsz = precision == OEM_ITER_F64 ? 8 : 4;
  return (size_t)((p + 3) & ~3) * tsz;
}

template <typename T, int M, bool kGrid, int RG>
static cudaError_t launch_t(const IterLaunch& P, cudaStream_t s, bool query, int* out) {
  constexpr int NT = iter_threads<T, M>();
  auto kfn = oem_iter_rows_kernel<T, M, NT, kGrid, RG>;
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
// instances then fill fewer sums per lane and no load is wasted).
template <typename T, int M, int RG>
static cudaError_t dispatch_r(const IterLaunch& P, cudaStream_t s, bool q, int* out) {
  return P.grid ? launch_t<T, M, true, RG>(P, s, q, out) : launch_t<T, M, false, RG>(P, s, q, out);
}
template <typename T, int M>
static cudaError_t dispatch_g(const IterLaunch& P, cudaStream_t s, bool q, int* out) {
  constexpr int RGF = 16 / M;
  if constexpr (RGF > 4) {
    constexpr int NW = iter_threads<T, M>() / 32;
    if ((P.max_rows + NW - 1) / NW <= 4) return dispatch_r<T, M, 4>(P, s, q, out);
  }
  return dispatch_r<T, M, RGF>(P, s, q, out);
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

int oem_iter_rows_max_cluster(const IterLaunch& P0) {
  IterLaunch P = P0;
  int n = 0;
  cudaError_t e = (P.precision == OEM_ITER_F64) ? dispatch_m<double>(P, 0, true, &n)
                                                : dispatch_m<float>(P, 0, true, &n);
  if (e != cudaSuccess) { cudaGetLastError(); return 0; }
  return n;
}

cudaError_t launch_oem_iter_rows(const IterLaunch& P, cudaStream_t s) {
  if (P.precision == OEM_ITER_F64) return dispatch_m<double>(P, s, false, nullptr);
  return dispatch_m<float>(P, s, false, nullptr);
}

}  // namespace oem
