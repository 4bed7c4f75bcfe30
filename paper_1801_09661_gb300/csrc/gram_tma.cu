// Gram pass fed by TMA (split-BF16 and bfloat16 modes): per-fold partial
// upper triangles of Z^T Z, Z = [X | y-columns] (Section 3: the O(np^2) step
// that forms X_k^T X_k, X_k^T y_k for every fold in one pass).
//
// Two kernels:
//   1. zpack_kernel: one streaming pass over X in fold order writes Z as
//      bfloat16 — hi = bf16(z) and, in split mode, lo = bf16(z - hi) — with
//      q_pad = round_up(p + ycols, 128) columns and every fold's rows padded
//      with zero rows to a multiple of 32, so that the Gram kernel reads
//      whole 32-row boxes that never cross a fold;
//   2. gram_tma_kernel: one CTA per SM (persistent); a work item is a
//      128 x 128 tile (ti <= tj) over a chunk of packed rows. One thread
//      issues the TMA loads of each 32-row stage (64-column boxes, 128-byte
//      swizzle, the layout the tensor core reads as MN-major bfloat16), one
//      thread issues tcgen05.mma (hi.hi + hi.lo + lo.hi + lo.lo in split
//      mode, hi.hi for bfloat16 data) into a double-buffered float32
//      accumulator in tensor memory, and 16 epilogue warps add each finished
//      flush window into a (hi, lo) float32 TwoSum pair in tensor memory and
//      write hi + lo as float64 at the end of the item.
// Every mbarrier wait is bounded; on expiry the kernel records a timeout in
// the status word, drains its MMAs, frees tensor memory and returns.
#include "tcgen05.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace oem {

namespace tc {

constexpr int kTK = 32;                 // rows per stage
constexpr int kTNS = 4;                 // operand stages
constexpr int kTStageBytes = 32768;     // I_hi, I_lo, J_hi, J_lo panels of 8 KB
constexpr int kTEpiWarps = 16;          // warps 0..15
constexpr int kTMmaWarp = 16;
constexpr int kTProdWarp = 17;
constexpr int kTThreads = 18 * 32;

struct TBars {
  unsigned long long full[kTNS];
  unsigned long long empty[kTNS];
  unsigned long long acc_full[2];
  unsigned long long acc_empty[2];
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

struct TmaGramArgs {
  int32_t split;   // 1: four products from (hi, lo); 0: hi only
  int32_t ntile1, ntiles;
  ChunkTable pc;   // chunks of packed rows (row0, row1 multiples of 32)
  double* partial; // [chunks][ntiles][128][128]
  unsigned* dstatus;
};

__global__ void __launch_bounds__(kTThreads, 1)
    gram_tma_kernel(const __grid_constant__ CUtensorMap zhi, const __grid_constant__ CUtensorMap zlo,
                    TmaGramArgs a, int flush_stages) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  TBars* bars = reinterpret_cast<TBars*>(smem + kTNS * kTStageBytes);
  volatile int* abort_flag = &bars->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool split = a.split != 0;
  const int nprod = split ? 4 : 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTNS; ++s) {
      mbar_init(su32(&bars->full[s]), 1);
      mbar_init(su32(&bars->empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&bars->acc_full[b]), 1);
      mbar_init(su32(&bars->acc_empty[b]), kTEpiWarps);
    }
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

  if (warp == kTProdWarp) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      bool ok = true;
      uint32_t u = 0;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const int chunk = item / a.ntiles, tile = item % a.ntiles;
        int ti, tj;
        tile_coords(tile, a.ntile1, &ti, &tj);
        const bool diag = ti == tj;
        const int64_t r0 = a.pc.row0[chunk];
        const int nst = (int)((a.pc.row1[chunk] - r0) / kTK);
        const uint32_t bytes = (uint32_t)((diag ? 1 : 2) * (split ? 16384 : 8192));
        for (int st = 0; st < nst; ++st, ++u) {
          const int s = u % kTNS;
          if (!mbar_wait(su32(&bars->empty[s]), ((u / kTNS) & 1) ^ 1, abort_flag)) { ok = false; break; }
          const uint32_t bar = su32(&bars->full[s]);
          mbar_expect_tx(bar, bytes);
          const uint32_t base = stage0 + s * kTStageBytes;
          const int row = (int)(r0 + (int64_t)st * kTK);
          for (int pan = 0; pan < (diag ? 1 : 2); ++pan) {
            const int col = (pan == 0 ? ti : tj) * kTile;
            const uint32_t pb = base + pan * 16384;
            tma_load_2d(pb, &zhi, col, row, bar);
            tma_load_2d(pb + 4096, &zhi, col + 64, row, bar);
            if (split) {
              tma_load_2d(pb + 8192, &zlo, col, row, bar);
              tma_load_2d(pb + 8192 + 4096, &zlo, col + 64, row, bar);
            }
          }
        }
      }
      if (!ok) { bars->abort = 1; atomicOr(a.dstatus, kStatTimeout); }
    }
    __syncwarp();
  } else if (warp == kTMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc(1u, 1u);  // bfloat16, MN-major
      uint32_t u = 0, v = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const int chunk = item / a.ntiles, tile = item % a.ntiles;
        int ti, tj;
        tile_coords(tile, a.ntile1, &ti, &tj);
        const bool diag = ti == tj;
        const int nst = (int)((a.pc.row1[chunk] - a.pc.row0[chunk]) / kTK);
        for (int st0 = 0; st0 < nst && ok; st0 += flush_stages, ++v) {
          const int buf = v & 1;
          if (!mbar_wait(su32(&bars->acc_empty[buf]), ((v >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * kTile);
          const int st1 = min(nst, st0 + flush_stages);
          for (int st = st0; st < st1; ++st, ++u) {
            const int s = u % kTNS;
            if (!mbar_wait(su32(&bars->full[s]), (u / kTNS) & 1, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t base = stage0 + s * kTStageBytes;
            const uint32_t ihi = base, ilo = base + 8192;
            const uint32_t jhi = diag ? ihi : base + 16384, jlo = diag ? ilo : base + 24576;
#pragma unroll
            for (int ks = 0; ks < kTK / 16; ++ks) {
              for (int pr = 0; pr < nprod; ++pr) {
                const uint32_t pa = (pr >= 2) ? ilo : ihi;
                const uint32_t pb = (pr & 1) ? jlo : jhi;
                const uint64_t ad = make_desc(pa + ks * 2048, 4096, 1024);
                const uint64_t bd = make_desc(pb + ks * 2048, 4096, 1024);
                mma_f16(d, ad, bd, idesc, (st > st0 || ks > 0 || pr > 0) ? 1u : 0u);
              }
            }
            tc_commit(su32(&bars->empty[s]));
          }
          if (!ok) break;
          tc_commit(su32(&bars->acc_full[buf]));
        }
      }
      tc_commit(su32(&bars->drain));
      if (!mbar_wait(su32(&bars->drain), 0, abort_flag) && !*abort_flag) ok = false;
      if (!ok) { bars->abort = 1; atomicOr(a.dstatus, kStatTimeout); }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    // warp w reads lanes 32 (w % 4) .. +31 and columns [32 (w / 4), +32)
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int c0 = (warp >> 2) * 32;
    uint32_t v = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int chunk = item / a.ntiles, tile = item % a.ntiles;
      const int nst = (int)((a.pc.row1[chunk] - a.pc.row0[chunk]) / kTK);
      bool first = true;
      for (int st0 = 0; st0 < nst; st0 += flush_stages, ++v) {
        const int buf = v & 1;
        if (!mbar_wait(su32(&bars->acc_full[buf]), (v >> 1) & 1, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t acc = tmem + lane_base + (uint32_t)(buf * kTile);
        const uint32_t thi = tmem + lane_base + 256u, tlo = tmem + lane_base + 384u;
#pragma unroll
        for (int cb = c0; cb < c0 + 32; cb += 16) {
          uint32_t ra[16], rh[16], rl[16];
          tmem_ld16(acc + cb, ra);
          if (!first) { tmem_ld16(thi + cb, rh); tmem_ld16(tlo + cb, rl); }
          tmem_ld_wait();
          if (first) {
#pragma unroll
            for (int i = 0; i < 16; ++i) { rh[i] = ra[i]; rl[i] = 0u; }
          } else {
#pragma unroll
            for (int i = 0; i < 16; i += 2) two_sum_x2(rh[i], rh[i + 1], rl[i], rl[i + 1], ra[i], ra[i + 1]);
          }
          tmem_st16(thi + cb, rh);
          tmem_st16(tlo + cb, rl);
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(su32(&bars->acc_empty[buf]));
        first = false;
      }
      if (!ok) break;
      double* out = a.partial + ((int64_t)chunk * a.ntiles + tile) * (kTile * kTile) +
                    (int64_t)((warp & 3) * 32 + lane) * kTile;
      const uint32_t thi = tmem + lane_base + 256u, tlo = tmem + lane_base + 384u;
#pragma unroll
      for (int cb = c0; cb < c0 + 32; cb += 16) {
        uint32_t rh[16], rl[16];
        if (nst > 0) {
          tmem_ld16(thi + cb, rh);
          tmem_ld16(tlo + cb, rl);
          tmem_ld_wait();
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) { rh[i] = 0u; rl[i] = 0u; }
        }
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          double2 w;
          w.x = (double)__uint_as_float(rh[i]) + (double)__uint_as_float(rl[i]);
          w.y = (double)__uint_as_float(rh[i + 1]) + (double)__uint_as_float(rl[i + 1]);
          *reinterpret_cast<double2*>(out + cb + i) = w;
        }
      }
      tc_fence_before();
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
// multiple of 32). One thread; K <= 64.
__global__ void packed_chunks_kernel(const int64_t* __restrict__ fold_off, int K, int64_t chunk_rows,
                                     ChunkTable pc, int max_chunks, unsigned* dstatus) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t off = 0;
  int c = 0;
  for (int k = 0; k < K; ++k) {
    const int64_t np = (fold_off[k + 1] - fold_off[k] + 31) / 32 * 32;
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
  int32_t qp;           // packed columns (multiple of 64)
  const int32_t* perm;  // sorted -> original row, or NULL
  const int64_t* fold_off;  // [K+1] sorted offsets
  const int64_t* poff;      // [K+1] packed offsets
  int32_t K;
  int64_t rows_cap;     // packed rows allocated
  __nv_bfloat16* zhi;   // [rows_cap][qp]
  __nv_bfloat16* zlo;   // [rows_cap][qp] or NULL
};

// One warp per packed row; lane l converts columns [8 l, 8 l + 8) + 256 j.
__global__ void __launch_bounds__(256) zpack_kernel(ZPackArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t total = a.poff[a.K];
  for (int64_t pr = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pr < total;
       pr += nwarps) {
    int k = 0;
    while (k + 1 < a.K && a.poff[k + 1] <= pr) ++k;
    const int64_t local = pr - a.poff[k];
    int64_t row = -1;
    if (local < a.fold_off[k + 1] - a.fold_off[k]) {
      const int64_t sr = a.fold_off[k] + local;
      row = a.perm ? (int64_t)a.perm[sr] : sr;
    }
    float yp[3] = {0.f, 0.f, 0.f};
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
            }
          }
          v[u] = x;
        }
      }
      uint4 hi, lo;
      tc::split8(v, hi, lo);
      *reinterpret_cast<uint4*>(a.zhi + pr * a.qp + c0) = hi;
      if (a.zlo) *reinterpret_cast<uint4*>(a.zlo + pr * a.qp + c0) = lo;
    }
  }
}

size_t gram_tma_smem_bytes() { return (size_t)tc::kTNS * tc::kTStageBytes + sizeof(tc::TBars) + 1024; }

static cudaError_t encode_z_map(CUtensorMap* m, void* base, int64_t rows, int qp) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)qp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)qp * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)tc::kTK};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_zpack(const GramArgs& a, int K, const TmaBufs& t, cudaStream_t s) {
  packed_chunks_kernel<<<1, 1, 0, s>>>(a.ct.fold_off, K, t.chunk_rows, t.pc, t.max_chunks, a.dstatus);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ZPackArgs z{};
  z.X = a.X; z.xtype = a.xtype; z.ldx = a.ldx; z.p = a.p; z.y = (const float*)a.y;
  z.ycols = a.ycols; z.qp = t.qp; z.perm = a.perm; z.fold_off = a.ct.fold_off; z.poff = t.pc.fold_off;
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
  const int flush_stages = (flush_rows + tc::kTK - 1) / tc::kTK;
  CUtensorMap mhi, mlo;
  cudaError_t e = encode_z_map(&mhi, t.zhi, t.rows_cap, t.qp);
  if (e != cudaSuccess) return e;
  e = encode_z_map(&mlo, t.zlo ? (void*)t.zlo : (void*)t.zhi, t.rows_cap, t.qp);
  if (e != cudaSuccess) return e;
  const size_t smem = gram_tma_smem_bytes();
  e = cudaFuncSetAttribute(tc::gram_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = kNumSMsHint;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  tc::TmaGramArgs g{};
  g.split = t.zlo ? 1 : 0;
  g.ntile1 = a.ntile1;
  g.ntiles = a.ntiles;
  g.pc = t.pc;
  g.partial = a.partial;
  g.dstatus = a.dstatus;
  const int64_t items = (int64_t)t.max_chunks * a.ntiles;
  const int grid = (int)(items < sms ? items : sms);
  tc::gram_tma_kernel<<<grid, tc::kTThreads, smem, s>>>(mhi, mlo, g, flush_stages);
  return cudaGetLastError();
}

}  // namespace oem
