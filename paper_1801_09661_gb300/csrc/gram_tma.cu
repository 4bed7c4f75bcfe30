// Gram pass fed by TMA (split-BF16 and bfloat16 modes): per-fold partial
// upper triangles of Z^T Z, Z = [X | y-columns] (Section 3: the O(np^2) step
// that forms X_k^T X_k, X_k^T y_k for every fold in one pass).
//
// Two kernels:
//   1. zpack_kernel: one streaming pass over X in fold order writes Z as
//      bfloat16 — hi = bf16(z) and, in split mode, lo = bf16(z - hi) — with
//      q_pad = round_up(p + ycols, 128) columns and every fold's rows padded
//      with zero rows to a multiple of 64, so that the Gram kernel reads
//      whole boxes that never cross a fold;
//   2. gram_tma_kernel: one CTA per SM (persistent); a work item is a
//      128 x 128 tile (ti <= tj) over a chunk of packed rows. Two producer
//      warps issue the TMA loads of alternate 32 KB stages (32 rows of hi and
//      lo in split mode, 64 rows of hi in bfloat16 mode; 64-column boxes,
//      128-byte swizzle, the layout the tensor core reads as MN-major
//      bfloat16); one thread issues tcgen05.mma: hi.hi into a double-buffered
//      float32 accumulator in tensor memory, and in split mode the cross terms
//      hi.lo + lo.hi (+ lo.lo on diagonal tiles), 2^-8 smaller, into a
//      second accumulator that is emptied every 1,024 rows. Eight epilogue
//      warps add each finished window into a running TwoSum pair per
//      element — hi in a register, lo in tensor memory — and write hi + lo as
//      float64 at the end of the item.
// Every mbarrier wait is bounded; on expiry the kernel records a timeout in
// the status word, drains its MMAs, frees tensor memory and returns.
#include "tcgen05.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace oem {

namespace tc {

constexpr int kTNS = 6;                 // operand stages (even: two producers, three slots each)
constexpr int kTStageBytes = 32768;     // split: I_hi, I_lo, J_hi, J_lo of 32 rows; bfloat16: I_hi, J_hi of 64
constexpr int kTEpiWarps = 8;           // warps 0..7
constexpr int kTMmaWarp = 8;
constexpr int kTProdWarp = 9;           // warps 9, 10: producers of even / odd stages
constexpr int kTThreads = 11 * 32;
constexpr int kTEpiCols = 64;           // columns per epilogue thread
constexpr int kTCrossStages = 32;       // cross-term window (1,024 rows)

// Tensor-memory columns: the hi.hi accumulator (two buffers), in split mode
// the cross-term accumulator hi.lo + lo.hi (+ lo.lo) (one buffer), and the lo
// half of each element's running TwoSum pair (its hi half is a register).
constexpr uint32_t kTD1 = 0, kTD2 = 256, kTLo = 384;

struct TBars {
  unsigned long long full[kTNS];
  unsigned long long empty[kTNS];
  unsigned long long d1_full[2], d1_empty[2];
  unsigned long long d2_full, d2_empty;
  unsigned long long drain;
  unsigned tmem_base;
  int abort;
};

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// 2-D tiled TMA load of one box at (x = column, y = row) into shared memory,
// completing its bytes on bar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// Bounded wait that ignores the abort flag (used to drain copies in flight).
__device__ __forceinline__ bool mbar_wait_drain(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

struct TmaGramArgs {
  int32_t split;   // 1: four products from (hi, lo); 0: hi only
  int32_t nbx;     // bfloat16 mode: 64-column boxes below 64 nbx come from the
                   // first map (X itself in direct mode), the others from the
                   // second (the packed tail) at column c - 64 nbx
  int32_t ntile1, ntiles;
  ChunkTable pc;   // chunks of packed rows (row0, row1 multiples of kGramPackRows)
  double* partial; // [chunks][ntiles][128][128]
  unsigned* dstatus;
};

// The hi.hi window of an item ends at st1; the cross-term window ends there
// too when st1 is a multiple of kTCrossStages or the item's last stage.
__device__ __forceinline__ bool cross_ends(int st1, int nst) {
  return st1 == nst || st1 % kTCrossStages == 0;
}

// SPLIT: four products from (hi, lo), 32-row stages; otherwise hi.hi only,
// 64-row stages.
template <bool SPLIT>
__global__ void __launch_bounds__(kTThreads, 1)
    gram_tma_kernel(const __grid_constant__ CUtensorMap zhi, const __grid_constant__ CUtensorMap zlo,
                    TmaGramArgs a, int flush_stages) {
  constexpr int kRS = SPLIT ? 32 : 64;        // rows per stage
  constexpr uint32_t kAtom = kRS * 128;       // bytes of one 64-column box
  constexpr uint32_t kPanel = 2 * kAtom;      // 128 columns
  constexpr int kKS = kRS / 16;               // MMA k-steps per stage
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  TBars* bars = reinterpret_cast<TBars*>(smem + kTNS * kTStageBytes);
  volatile int* abort_flag = &bars->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool split = SPLIT;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTNS; ++s) {
      mbar_init(su32(&bars->full[s]), 1);
      mbar_init(su32(&bars->empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&bars->d1_full[b]), 1);
      mbar_init(su32(&bars->d1_empty[b]), kTEpiWarps);
    }
    mbar_init(su32(&bars->d2_full), 1);
    mbar_init(su32(&bars->d2_empty), kTEpiWarps);
    mbar_init(su32(&bars->drain), 1);
    bars->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kTMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     su32(&bars->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  const int nitems = *a.pc.count * a.ntiles;
  const uint32_t stage0 = su32(smem);

  if (warp == kTProdWarp || warp == kTProdWarp + 1) {
    // ------------------------------------------------ TMA producers (2 warps)
    // producer q issues the stages u with u % 2 == q (slots q, q + 2, q + 4)
    if (lane == 0) {
      const uint32_t q = (uint32_t)(warp - kTProdWarp);
      bool ok = true;
      uint32_t u0 = 0;
      int64_t last0 = -1, last1 = -1, last2 = -1;  // last stage issued into each of this producer's slots
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const int chunk = item / a.ntiles, tile = item % a.ntiles;
        int ti, tj;
        tile_coords(tile, a.ntile1, &ti, &tj);
        const bool diag = ti == tj;
        const int row0 = (int)a.pc.row0[chunk];
        const int nst = (int)((a.pc.row1[chunk] - a.pc.row0[chunk]) / kRS);
        const uint32_t bytes = (diag ? 1u : 2u) * 16384u;
        const int ci = ti * kTile, cj = tj * kTile;
        for (int st = (int)((u0 ^ q) & 1u); st < nst; st += 2) {
          const uint32_t u = u0 + (uint32_t)st;
          const uint32_t s = u % kTNS;
          if (!mbar_wait(su32(&bars->empty[s]), ((u / kTNS) & 1) ^ 1, abort_flag)) { ok = false; break; }
          const uint32_t bar = su32(&bars->full[s]);
          mbar_expect_tx(bar, bytes);
          if ((s >> 1) == 0) last0 = u; else if ((s >> 1) == 1) last1 = u; else last2 = u;
          const uint32_t pb = stage0 + s * kTStageBytes;
          const int row = row0 + st * kRS;
          // one 64-column box of hi (bfloat16 mode: from X or from the tail)
          auto hi_box = [&](uint32_t dst, int c) {
            if (split || c < 64 * a.nbx) tma_load_2d(dst, &zhi, c, row, bar);
            else tma_load_2d(dst, &zlo, c - 64 * a.nbx, row, bar);
          };
          hi_box(pb, ci);
          hi_box(pb + kAtom, ci + 64);
          if (split) {
            tma_load_2d(pb + kPanel, &zlo, ci, row, bar);
            tma_load_2d(pb + kPanel + kAtom, &zlo, ci + 64, row, bar);
          }
          if (!diag) {
            hi_box(pb + 16384, cj);
            hi_box(pb + 16384 + kAtom, cj + 64);
            if (split) {
              tma_load_2d(pb + 16384 + kPanel, &zlo, cj, row, bar);
              tma_load_2d(pb + 16384 + kPanel + kAtom, &zlo, cj + 64, row, bar);
            }
          }
        }
        u0 += (uint32_t)nst;
      }
      if (!ok) {
        bars->abort = 1;
        atomicOr(a.dstatus, kStatTimeout);
        // let this producer's copies in flight land before the CTA exits
        if (last0 >= 0) mbar_wait_drain(su32(&bars->full[(uint32_t)last0 % kTNS]), ((uint32_t)last0 / kTNS) & 1);
        if (last1 >= 0) mbar_wait_drain(su32(&bars->full[(uint32_t)last1 % kTNS]), ((uint32_t)last1 / kTNS) & 1);
        if (last2 >= 0) mbar_wait_drain(su32(&bars->full[(uint32_t)last2 % kTNS]), ((uint32_t)last2 / kTNS) & 1);
      }
    }
    __syncwarp();
  } else if (warp == kTMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc(1u, 1u);  // bfloat16, MN-major
      // descriptor of stage 0's first panel; other panels add their offset / 16
      const uint64_t desc0 = make_desc(stage0, kAtom, 1024);
      uint32_t u = 0, v1 = 0, v2 = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const int chunk = item / a.ntiles, tile = item % a.ntiles;
        int ti, tj;
        tile_coords(tile, a.ntile1, &ti, &tj);
        const uint32_t joff = ti == tj ? 0u : 16384u;
        // lo.lo only on diagonal tiles: there lo_i^2 > 0 would bias G_ii by
        // ~2^-18 / 3; off the diagonal lo_i lo_j has zero mean and is 2^-16
        // of the cross terms, so those tiles take the three products
        // hi.hi, hi.lo, lo.hi
        const bool lolo = ti == tj;
        const int nst = (int)((a.pc.row1[chunk] - a.pc.row0[chunk]) / kRS);
        bool d2_fresh = true;
        for (int st0 = 0; st0 < nst && ok; st0 += flush_stages, ++v1) {
          const uint32_t b1 = v1 & 1;
          if (!mbar_wait(su32(&bars->d1_empty[b1]), ((v1 >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
          if (split && d2_fresh) {
            if (!mbar_wait(su32(&bars->d2_empty), (v2 & 1) ^ 1, abort_flag)) { ok = false; break; }
          }
          tc_fence_after();
          const uint32_t d1 = tmem + kTD1 + b1 * kTile;
          const uint32_t d2 = tmem + kTD2;
          const int st1 = min(nst, st0 + flush_stages);
          for (int st = st0; st < st1; ++st, ++u) {
            const uint32_t s = u % kTNS;
            if (!mbar_wait(su32(&bars->full[s]), (u / kTNS) & 1, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint64_t ihi = desc0 + ((s * kTStageBytes) >> 4);
            const uint64_t ilo = ihi + (kPanel >> 4);
            const uint64_t jhi = ihi + (joff >> 4), jlo = jhi + (kPanel >> 4);
#pragma unroll
            for (int ks = 0; ks < kKS; ++ks) {
              const uint64_t kof = (uint64_t)((ks * 2048) >> 4);
              mma_f16(d1, ihi + kof, jhi + kof, idesc, (st > st0 || ks > 0) ? 1u : 0u);
              if (split) {
                mma_f16(d2, ihi + kof, jlo + kof, idesc, d2_fresh ? 0u : 1u);
                mma_f16(d2, ilo + kof, jhi + kof, idesc, 1u);
                if (lolo) mma_f16(d2, ilo + kof, jlo + kof, idesc, 1u);
                d2_fresh = false;
              }
            }
            tc_commit(su32(&bars->empty[s]));
          }
          if (!ok) break;
          tc_commit(su32(&bars->d1_full[b1]));
          if (split && cross_ends(st1, nst)) {
            tc_commit(su32(&bars->d2_full));
            ++v2;
            d2_fresh = true;
          }
        }
      }
      tc_commit(su32(&bars->drain));
      if (!mbar_wait(su32(&bars->drain), 0, abort_flag) && !*abort_flag) ok = false;
      if (!ok) {
        bars->abort = 1;
        atomicOr(a.dstatus, kStatTimeout);
        mbar_wait_drain(su32(&bars->drain), 0);  // MMAs in flight finish before tensor memory is freed
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    // warp w owns lanes 32 (w % 4) .. +31 and columns [64 (w / 4), +64); the
    // hi half of each of its 64 running TwoSum pairs stays in a register for
    // the whole item, the lo half in tensor memory
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t c0 = (uint32_t)(warp >> 2) * kTEpiCols;
    uint32_t v1 = 0, v2 = 0;
    bool ok = true;
    uint32_t h[kTEpiCols];
    const uint32_t tlo = tmem + lane_base + kTLo + c0;
    // adds the 64 float32 values of one finished window at taddr
    auto add_window = [&](uint32_t taddr) {
#pragma unroll
      for (int q = 0; q < kTEpiCols / 8; ++q) {
        uint32_t r[8], lo[8];
        tmem_ld8(taddr + q * 8, r);
        tmem_ld8(tlo + q * 8, lo);
        tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 8; i += 2) two_sum_x2(h[q * 8 + i], h[q * 8 + i + 1], lo[i], lo[i + 1], r[i], r[i + 1]);
        tmem_st8(tlo + q * 8, lo);
      }
      tmem_st_wait();
    };
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int chunk = item / a.ntiles, tile = item % a.ntiles;
      const int nst = (int)((a.pc.row1[chunk] - a.pc.row0[chunk]) / kRS);
#pragma unroll
      for (int i = 0; i < kTEpiCols; ++i) h[i] = 0u;
      {
        const uint32_t z[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
        for (int q = 0; q < kTEpiCols / 8; ++q) tmem_st8(tlo + q * 8, z);
        tmem_st_wait();
      }
      for (int st0 = 0; st0 < nst; st0 += flush_stages, ++v1) {
        const uint32_t b1 = v1 & 1;
        if (!mbar_wait(su32(&bars->d1_full[b1]), (v1 >> 1) & 1, abort_flag)) { ok = false; break; }
        tc_fence_after();
        add_window(tmem + lane_base + kTD1 + b1 * kTile + c0);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(su32(&bars->d1_empty[b1]));
        const int st1 = min(nst, st0 + flush_stages);
        if (split && cross_ends(st1, nst)) {
          if (!mbar_wait(su32(&bars->d2_full), v2 & 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
          add_window(tmem + lane_base + kTD2 + c0);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(su32(&bars->d2_empty));
          ++v2;
        }
      }
      if (!ok) break;
      double* out = a.partial + ((int64_t)chunk * a.ntiles + tile) * (kTile * kTile) +
                    (int64_t)((warp & 3) * 32 + lane) * kTile + c0;
#pragma unroll
      for (int q = 0; q < kTEpiCols / 8; ++q) {
        uint32_t lo[8];
        tmem_ld8(tlo + q * 8, lo);
        tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          double2 w;
          w.x = (double)__uint_as_float(h[q * 8 + i]) + (double)__uint_as_float(lo[i]);
          w.y = (double)__uint_as_float(h[q * 8 + i + 1]) + (double)__uint_as_float(lo[i + 1]);
          *reinterpret_cast<double2*>(out + q * 8 + i) = w;
        }
      }
    }
    if (!ok) { bars->abort = 1; atomicOr(a.dstatus, kStatTimeout); }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kTMmaWarp) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

}  // namespace tc

// ---------------------------------------------------------------- packing

// Chunks of the packed row space: fold k holds packed rows
// [poff[k], poff[k] + round_up(n_k, 32)), cut into chunks of chunk_rows (a
// multiple of kGramPackRows). One thread; K <= 64.
__global__ void packed_chunks_kernel(const int64_t* __restrict__ fold_off, int K, int64_t chunk_rows,
                                     ChunkTable pc, int max_chunks, unsigned* dstatus) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t off = 0;
  int c = 0;
  for (int k = 0; k < K; ++k) {
    const int64_t np = (fold_off[k + 1] - fold_off[k] + kGramPackRows - 1) / kGramPackRows * kGramPackRows;
    pc.fold_off[k] = off;
    pc.fold_c0[k] = c;
    for (int64_t r = 0; r < np; r += chunk_rows) {
      if (c >= max_chunks) { atomicOr(dstatus, kStatTimeout); break; }
      pc.row0[c] = off + r;
      pc.row1[c] = off + (r + chunk_rows < np ? r + chunk_rows : np);
      pc.fold[c] = k;
      ++c;
    }
    off += np;
  }
  pc.fold_off[K] = off;
  pc.fold_c0[K] = c;
  *pc.count = c;
}

struct ZPackArgs {
  const void* X;
  int32_t xtype;        // OEM_F32 or OEM_BF16
  int64_t ldx, p;
  const float* y;
  int32_t ycols;        // 1 (split) or 3 (bfloat16 pieces of y)
  int32_t ocols;        // 1: a column of ones after y (split mode)
  const float* shift;   // [p + 1] or NULL (split mode): subtracted exactly
  int32_t qp;           // packed columns (multiple of 64)
  const int32_t* perm;  // sorted -> original row, or NULL
  const int32_t* ipos;  // original -> packed row (-1: no fold), or NULL
  int64_t n;
  const int64_t* fold_off;  // [K+1] sorted offsets
  const int64_t* poff;      // [K+1] packed offsets
  int32_t K;
  int64_t rows_cap;     // packed rows allocated
  __nv_bfloat16* zhi;   // [rows_cap][qp]
  __nv_bfloat16* zlo;   // [rows_cap][qp] or NULL
};

// One warp per packed row; lane l converts columns [8 l, 8 l + 8) + 256 j.
// With ipos the warps take X's rows in their own order (reads stream through
// X; each row is written to its place in fold order), then the zero rows
// that pad every fold; without it, the packed rows in order.
__global__ void __launch_bounds__(256) zpack_kernel(ZPackArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t total = a.ipos ? a.n + (a.poff[a.K] - a.fold_off[a.K]) : a.poff[a.K];
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < total;
       task += nwarps) {
    int64_t row = -1, pr = task;
    if (a.ipos) {
      if (task < a.n) {
        pr = a.ipos[task];
        if (pr < 0) continue;  // outside every fold
        row = task;
      } else {
        int64_t j = task - a.n;
        int k = 0;
        for (;; ++k) {
          const int64_t pad = (a.poff[k + 1] - a.poff[k]) - (a.fold_off[k + 1] - a.fold_off[k]);
          if (j < pad || k + 1 >= a.K) break;
          j -= pad;
        }
        pr = a.poff[k] + (a.fold_off[k + 1] - a.fold_off[k]) + j;
      }
    } else {
      int k = 0;
      while (k + 1 < a.K && a.poff[k + 1] <= pr) ++k;
      const int64_t local = pr - a.poff[k];
      if (local < a.fold_off[k + 1] - a.fold_off[k]) {
        const int64_t sr = a.fold_off[k] + local;
        row = a.perm ? (int64_t)a.perm[sr] : sr;
      }
    }
    float yp[3] = {0.f, 0.f, 0.f};
    const float yshift = a.shift ? a.shift[a.p] : 0.f;
    if (row >= 0) {
      const float yv = a.y[row];
      yp[0] = yv;
      if (a.ycols == 3) {
        yp[0] = tc::bf16_round(yv);
        yp[1] = tc::bf16_round(yv - yp[0]);
        yp[2] = (yv - yp[0]) - yp[1];
      }
    }
    for (int c0 = lane * 8; c0 < a.qp; c0 += 256) {
      float v[8];
      if (row >= 0 && c0 + 8 <= a.p) {
        if (a.xtype == OEM_F32) {
          const float* src = (const float*)a.X + row * a.ldx + c0;
          const float4 q0 = __ldcs(reinterpret_cast<const float4*>(src));
          const float4 q1 = __ldcs(reinterpret_cast<const float4*>(src) + 1);
          v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
          v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
        } else {
          const uint4 q = __ldcs(reinterpret_cast<const uint4*>((const __nv_bfloat16*)a.X + row * a.ldx + c0));
          const uint32_t wq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            v[2 * i] = __uint_as_float(wq[i] << 16);
            v[2 * i + 1] = __uint_as_float(wq[i] & 0xFFFF0000u);
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + u;
          float x = 0.f;
          if (row >= 0) {
            if (c < a.p) {
              x = (a.xtype == OEM_F32) ? ((const float*)a.X)[row * a.ldx + c]
                                       : __bfloat162float(((const __nv_bfloat16*)a.X)[row * a.ldx + c]);
            } else if (c - a.p < a.ycols) {
              x = yp[c - a.p];
            } else if (c - a.p == a.ycols && a.ocols) {
              x = 1.f;
            }
          }
          v[u] = x;
        }
      }
      uint4 hi, lo;
      if (a.shift) {
        float m[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + u;
          m[u] = (row < 0) ? 0.f : (c < a.p ? a.shift[c] : (c == a.p ? yshift : 0.f));
        }
        tc::split8_shift(v, m, hi, lo);
      } else {
        tc::split8(v, hi, lo);
      }
      *reinterpret_cast<uint4*>(a.zhi + pr * a.qp + c0) = hi;
      if (a.zlo) *reinterpret_cast<uint4*>(a.zlo + pr * a.qp + c0) = lo;
    }
  }
}

size_t gram_tma_smem_bytes() { return (size_t)tc::kTNS * tc::kTStageBytes + sizeof(tc::TBars) + 1024; }

// 2-D bfloat16 tensor map: cols x rows, row stride ld elements, boxes of 64
// columns x box_rows rows, 128-byte swizzle; reads outside the extents give
// zeros.
static cudaError_t encode_bf16_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols,
                                   int64_t ld, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
static cudaError_t encode_z_map(CUtensorMap* m, void* base, int64_t rows, int qp, int box_rows) {
  return encode_bf16_map(m, base, rows, qp, qp, box_rows);
}

// Direct mode: the tail of Z for bfloat16 X -- X's columns [64 nbx, p), the
// three bfloat16 pieces of y (exact: y = y0 + y1 + y2), zeros up to
// tail_cols -- one 8-column unit per thread.
__global__ void tail_pack_kernel(const __nv_bfloat16* __restrict__ X, int64_t ldx, int64_t n, int64_t p,
                                 const float* __restrict__ y, int nbx, int tail_cols,
                                 __nv_bfloat16* __restrict__ tail) {
  const int units = tail_cols / 8;
  const int64_t total = n * units;
  const int64_t x0 = 64 * (int64_t)nbx;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / units;
    const int u = (int)(e % units);
    const float yv = y[r];
    const float y0 = tc::bf16_round(yv);
    const float y1 = tc::bf16_round(yv - y0);
    const float yp[3] = {y0, y1, (yv - y0) - y1};
    uint16_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t c = x0 + 8 * u + q;
      uint16_t b = 0;
      if (c < p) b = __bfloat16_as_ushort(X[r * ldx + c]);
      else if (c - p < 3) b = __bfloat16_as_ushort(__float2bfloat16_rn(yp[c - p]));
      w[q] = b;
    }
    uint4 v;
    v.x = (uint32_t)w[0] | ((uint32_t)w[1] << 16);
    v.y = (uint32_t)w[2] | ((uint32_t)w[3] << 16);
    v.z = (uint32_t)w[4] | ((uint32_t)w[5] << 16);
    v.w = (uint32_t)w[6] | ((uint32_t)w[7] << 16);
    *reinterpret_cast<uint4*>(tail + r * tail_cols + 8 * u) = v;
  }
}

cudaError_t launch_tail_pack(const GramArgs& a, const TmaBufs& t, cudaStream_t s) {
  packed_chunks_kernel<<<1, 1, 0, s>>>(a.ct.fold_off, 1, t.chunk_rows, t.pc, t.max_chunks, a.dstatus);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = kNumSMsHint;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  tail_pack_kernel<<<sms * 4, 256, 0, s>>>((const __nv_bfloat16*)a.X, a.ldx, a.n, a.p, (const float*)a.y, t.nbx,
                                           t.tail_cols, (__nv_bfloat16*)t.zhi);
  return cudaGetLastError();
}

cudaError_t launch_zpack(const GramArgs& a, int K, const TmaBufs& t, cudaStream_t s) {
  packed_chunks_kernel<<<1, 1, 0, s>>>(a.ct.fold_off, K, t.chunk_rows, t.pc, t.max_chunks, a.dstatus);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ZPackArgs z{};
  z.X = a.X; z.xtype = a.xtype; z.ldx = a.ldx; z.p = a.p; z.y = (const float*)a.y;
  z.ycols = a.ycols; z.ocols = a.ocols; z.shift = a.shift; z.qp = t.qp; z.perm = a.perm; z.fold_off = a.ct.fold_off; z.poff = t.pc.fold_off;
  z.ipos = a.ipos; z.n = a.n;
  z.K = K; z.rows_cap = t.rows_cap;
  z.zhi = (__nv_bfloat16*)t.zhi;
  z.zlo = (__nv_bfloat16*)t.zlo;
  int dev = 0, sms = kNumSMsHint;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  zpack_kernel<<<sms * 8, 256, 0, s>>>(z);
  return cudaGetLastError();
}

cudaError_t launch_gram_tma(const GramArgs& a, const TmaBufs& t, int flush_rows, cudaStream_t s) {
  if (flush_rows <= 0) flush_rows = 256;
  const bool split = t.zlo != nullptr;
  const int rs = split ? 32 : 64;  // rows per stage
  // hi.hi windows of a power-of-two number of stages that divides the
  // cross-term window, so both windows end together
  int flush_stages = 1;
  while (flush_stages * 2 * rs <= flush_rows && flush_stages * 2 <= tc::kTCrossStages) flush_stages *= 2;
  CUtensorMap mhi, mlo;
  cudaError_t e;
  if (t.direct) {
    // X itself (boxes below 64 nbx: inside its p columns) and the tail; rows
    // past n read as zeros
    e = encode_bf16_map(&mhi, a.X, a.n, a.p, a.ldx, rs);
    if (e != cudaSuccess) return e;
    e = encode_bf16_map(&mlo, t.zhi, a.n, t.tail_cols, t.tail_cols, rs);
  } else {
    e = encode_z_map(&mhi, t.zhi, t.rows_cap, t.qp, rs);
    if (e != cudaSuccess) return e;
    e = encode_z_map(&mlo, split ? t.zlo : t.zhi, t.rows_cap, t.qp, rs);
  }
  if (e != cudaSuccess) return e;
  const size_t smem = gram_tma_smem_bytes();
  auto kern = split ? tc::gram_tma_kernel<true> : tc::gram_tma_kernel<false>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = kNumSMsHint;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  tc::TmaGramArgs g{};
  g.split = split ? 1 : 0;
  g.nbx = t.direct ? t.nbx : (1 << 24);
  g.ntile1 = a.ntile1;
  g.ntiles = a.ntiles;
  g.pc = t.pc;
  g.partial = a.partial;
  g.dstatus = a.dstatus;
  const int64_t items = (int64_t)t.max_chunks * a.ntiles;
  const int grid = (int)(items < sms ? items : sms);
  kern<<<grid, tc::kTThreads, smem, s>>>(mhi, mlo, g, flush_stages);
  return cudaGetLastError();
}

}  // namespace oem
