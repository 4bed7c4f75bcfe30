// Gram pass on the 5th-generation tensor cores (tcgen05, sm_103a): per-fold
// partial upper triangles of Z^T Z, Z = [X | y-columns] (Section 3: the
// O(np^2) step that forms X_k^T X_k, X_k^T y_k for every fold in one pass).
//
// One CTA per SM (persistent). A work item is a 128 x 128 tile (ti <= tj) of
// the upper triangle over a chunk of fold-sorted rows. Roles per CTA:
//   * 8 converter warps stream 32-row stages of columns [128 ti, +128) and
//     [128 tj, +128) (rows gathered through the fold permutation) into a raw
//     shared-memory ring with cp.async, two stages ahead of the one they
//     convert; each thread then converts the bytes it loaded (float32 -> hi/lo
//     bfloat16 split, bfloat16 copy, or float32 -> tf32) into the operand
//     stage in the layout the tensor core reads (MN-major 128-byte swizzle for
//     bfloat16, K-major for tf32);
//   * 1 warp allocates tensor memory and one elected thread issues
//     tcgen05.mma (M = N = 128, float32 accumulation in tensor memory) for
//     each stage, double-buffering the accumulator per flush window;
//   * 8 epilogue warps (two per 32 tensor-memory lanes, 64 columns each) add
//     each finished window into a compensated (hi, lo) float32 pair kept in
//     tensor memory (TwoSum), and write hi + lo as float64 at the end of the
//     item.
// Every mbarrier wait is bounded by a clock budget; on expiry the kernel
// records a timeout in the status word, drains its MMAs, frees tensor memory
// and returns.
#include "tcgen05.cuh"

namespace oem {

namespace tc {

constexpr int kKS = 32;           // rows per stage
constexpr int kNS = 4;            // operand stages
constexpr int kStageBytes = 32768;
constexpr int kRawSlots = 3;      // raw ring: the stage being converted + 2 in flight
constexpr int kPrefetch = kRawSlots - 1;
constexpr int kRawBytes = 32768;
constexpr int kEpiWarps = 8;      // warps 0..7
constexpr int kMmaWarp = 8;
constexpr int kConvWarps = 8;     // warps 9..16
constexpr int kConvBase = (kEpiWarps + 1) * 32;
constexpr int kThreads = (kEpiWarps + 1 + kConvWarps) * 32;  // 544

struct Bars {
  unsigned long long full[kNS];
  unsigned long long empty[kNS];
  unsigned long long acc_full[2];
  unsigned long long acc_empty[2];
  unsigned long long drain;
  unsigned tmem_base;
  int abort;
};
// K-major float32 / tf32 panel (128 MN rows x 32 K): 8-row groups 1024 B
// apart, each row 128 B of K-contiguous data, 16-byte chunks (4 K values)
// XOR-swizzled by the row. Offset of the chunk holding K rows [4 kq, 4 kq+4)
// of MN index mn.
__device__ __forceinline__ uint32_t off_kmaj_f32(int mn, int kq) {
  return (uint32_t)((mn >> 3) * 1024 + (mn & 7) * 128 + ((kq ^ (mn & 7)) << 4));
}

// Column shift of Z (centring; 0 without a shift vector or past y).
__device__ __forceinline__ float zshift(const GramArgs& a, int col) {
  if (!a.shift) return 0.f;
  return col < a.p ? a.shift[col] : (col == a.p ? a.shift[a.p] : 0.f);
}

// One element of Z = [X | y | 1] (tf32 mode: one y column), shifted.
__device__ __forceinline__ float zval_f32(const GramArgs& a, int64_t row, int col) {
  if (col < a.p) return ((const float*)a.X)[row * a.ldx + col] - zshift(a, col);
  if (col == a.p) return ((const float*)a.y)[row] - zshift(a, col);
  if (col == a.p + a.ycols && a.ocols) return 1.f;
  return 0.f;
}

__device__ __forceinline__ uint32_t to_tf32(float a) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
  return r;
}

// Values of Z at 8 consecutive columns [c0, c0+8) of original row `row`
// (direct loads; used for the columns that hold y or run past p).
__device__ __forceinline__ void load8(const GramArgs& a, int64_t row, int c0, float (&v)[8]) {
  const int p = (int)a.p;
  // y columns: one (split mode) or three bfloat16 pieces hi + mid + lo that
  // hold a float32 y exactly (bfloat16 mode)
  const float yv = ((const float*)a.y)[row];
  float yp[3] = {yv, 0.f, 0.f};
  if (a.ycols == 3) {
    yp[0] = bf16_round(yv);
    yp[1] = bf16_round(yv - yp[0]);
    yp[2] = (yv - yp[0]) - yp[1];
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int c = c0 + u;
    float x = 0.f;
    if (c < p) {
      x = (a.xtype == OEM_F32) ? ((const float*)a.X)[row * a.ldx + c]
                               : __bfloat162float(((const __nv_bfloat16*)a.X)[row * a.ldx + c]);
    } else if (c - p < a.ycols) {
      x = yp[c - p];
    } else if (c - p == a.ycols && a.ocols) {
      x = 1.f;
    }
    v[u] = x;
  }
}

// The CTA's sequence of (item, stage) pairs, shared by the converter's load
// and convert cursors.
struct StageCursor {
  int item, st, nst, chunk, ti, tj;
  int64_t r0, r1;
  bool valid;
  __device__ void set_item(const GramArgs& a, int it, int nitems) {
    item = it;
    valid = it < nitems;
    if (!valid) return;
    chunk = it / a.ntiles;
    const int tile = it % a.ntiles;
    tile_coords(tile, a.ntile1, &ti, &tj);
    r0 = a.ct.row0[chunk];
    r1 = a.ct.row1[chunk];
    nst = (int)((r1 - r0 + kKS - 1) / kKS);
    st = 0;
    if (nst == 0) valid = false;
  }
  __device__ void next(const GramArgs& a, int nitems) {
    if (!valid) return;
    if (++st >= nst) set_item(a, item + gridDim.x, nitems);
  }
};

// Converter items of one stage (non-tf32): (panel, row, 8-column group),
// group fastest; 512 per panel. A thread owns items ct, ct + 256, ...
__device__ __forceinline__ bool item_async(const GramArgs& a, const StageCursor& c, int e,
                                           int64_t* row_out, int* col_out) {
  const int g = e & 15, r = (e >> 4) & (kKS - 1), pan = e >> 9;
  const int64_t sr = c.r0 + (int64_t)c.st * kKS + r;
  const int col = (pan == 0 ? c.ti : c.tj) * kTile + g * 8;
  *col_out = col;
  if (sr >= c.r1) { *row_out = -1; return false; }
  *row_out = a.perm ? (int64_t)a.perm[sr] : sr;
  return col + 8 <= a.p;
}

__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(GramArgs a, int flush_stages) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the operand stages (swizzle atoms)
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* raw = smem + kNS * kStageBytes;
  Bars* bars = reinterpret_cast<Bars*>(raw + kRawSlots * kRawBytes);
  volatile int* abort_flag = &bars->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mode = a.mode;
  const bool split = mode == OEM_GRAM_SPLIT_BF16;
  const bool tf32 = mode == OEM_GRAM_TF32;
  const int nprod = split ? 4 : 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kNS; ++s) {
      mbar_init(su32(&bars->full[s]), kConvWarps);
      mbar_init(su32(&bars->empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&bars->acc_full[b]), 1);
      mbar_init(su32(&bars->acc_empty[b]), kEpiWarps);
    }
    mbar_init(su32(&bars->drain), 1);
    bars->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     su32(&bars->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  const int nitems = *a.ct.count * a.ntiles;
  const uint32_t stage0 = su32(smem);

  if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // bfloat16 operands MN-major (rows of X land in shared memory as they
      // are); tf32 operands K-major (the converter transposes 4-row quads)
      const uint32_t idesc = tf32 ? make_idesc(2u, 0u) : make_idesc(1u, 1u);
      uint32_t u = 0, v = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const int chunk = item / a.ntiles, tile = item % a.ntiles;
        int ti, tj;
        tile_coords(tile, a.ntile1, &ti, &tj);
        const bool diag = ti == tj;
        const int64_t rows = a.ct.row1[chunk] - a.ct.row0[chunk];
        const int nst = (int)((rows + kKS - 1) / kKS);
        for (int st0 = 0; st0 < nst && ok; st0 += flush_stages, ++v) {
          const int buf = v & 1;
          if (!mbar_wait(su32(&bars->acc_empty[buf]), ((v >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * kTile);
          const int st1 = min(nst, st0 + flush_stages);
          for (int st = st0; st < st1; ++st, ++u) {
            const int s = u % kNS;
            if (!mbar_wait(su32(&bars->full[s]), (u / kNS) & 1, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t base = stage0 + s * kStageBytes;
            if (tf32) {
              const uint32_t pa = base, pb = diag ? base : base + 16384;
#pragma unroll
              for (int ks = 0; ks < kKS / 8; ++ks) {
                // K = 8 tf32 = 32 bytes: advance the start inside the 128-byte rows
                const uint64_t ad = make_desc(pa + ks * 32, 16, 1024);
                const uint64_t bd = make_desc(pb + ks * 32, 16, 1024);
                mma_tf32(d, ad, bd, idesc, (st > st0 || ks > 0) ? 1u : 0u);
              }
            } else {
              // panels: I_hi, I_lo, J_hi, J_lo (8 KB each); diagonal tiles reuse I
              const uint32_t ihi = base, ilo = base + 8192;
              const uint32_t jhi = diag ? ihi : base + 16384, jlo = diag ? ilo : base + 24576;
#pragma unroll
              for (int ks = 0; ks < kKS / 16; ++ks) {
                for (int pr = 0; pr < nprod; ++pr) {
                  const uint32_t pa = (pr >= 2) ? ilo : ihi;
                  const uint32_t pb = (pr & 1) ? jlo : jhi;
                  const uint64_t ad = make_desc(pa + ks * 2048, 4096, 1024);
                  const uint64_t bd = make_desc(pb + ks * 2048, 4096, 1024);
                  mma_f16(d, ad, bd, idesc, (st > st0 || ks > 0 || pr > 0) ? 1u : 0u);
                }
              }
            }
            tc_commit(su32(&bars->empty[s]));
          }
          if (!ok) break;
          tc_commit(su32(&bars->acc_full[buf]));
        }
      }
      // drain: wait until every issued MMA has completed
      tc_commit(su32(&bars->drain));
      if (!mbar_wait(su32(&bars->drain), 0, abort_flag) && !*abort_flag) ok = false;
      if (!ok) { bars->abort = 1; atomicOr(a.dstatus, kStatTimeout); }
    }
    __syncwarp();
  } else if (warp < kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    // warp w reads lanes 32 (w % 4) .. +31 and columns [64 (w / 4), +64)
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int c0 = (warp >> 2) * 64;
    uint32_t v = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int chunk = item / a.ntiles, tile = item % a.ntiles;
      const int64_t rows = a.ct.row1[chunk] - a.ct.row0[chunk];
      const int nst = (int)((rows + kKS - 1) / kKS);
      bool first = true;
      for (int st0 = 0; st0 < nst; st0 += flush_stages, ++v) {
        const int buf = v & 1;
        if (!mbar_wait(su32(&bars->acc_full[buf]), (v >> 1) & 1, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t acc = tmem + lane_base + (uint32_t)(buf * kTile);
        const uint32_t thi = tmem + lane_base + 256u, tlo = tmem + lane_base + 384u;
#pragma unroll 1
        for (int cb = c0; cb < c0 + 64; cb += 16) {
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
      // item done: hi + lo as float64 (row 32 (w % 4) + lane of the tile)
      double* out = a.partial + ((int64_t)chunk * a.ntiles + tile) * (kTile * kTile) +
                    (int64_t)((warp & 3) * 32 + lane) * kTile;
      const uint32_t thi = tmem + lane_base + 256u, tlo = tmem + lane_base + 384u;
#pragma unroll 1
      for (int cb = c0; cb < c0 + 64; cb += 16) {
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
  } else {
    // ------------------------------------------------------------ converters
    const int ct = threadIdx.x - kConvBase;  // 0..255
    const bool f32 = a.xtype == OEM_F32;
    StageCursor ld, cv;
    ld.set_item(a, blockIdx.x, nitems);
    cv.set_item(a, blockIdx.x, nitems);
    // issue the raw loads of one stage into raw slot `slot` (non-tf32 modes)
    auto issue = [&](const StageCursor& c, int slot) {
      if (!c.valid || tf32) return;
      const int npan = (c.ti == c.tj) ? 1 : 2;
      const uint32_t rbase = su32(raw + slot * kRawBytes);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e = ct + j * (kConvWarps * 32);
        if (e >= npan * kKS * 16) break;
        int64_t row;
        int col;
        if (item_async(a, c, e, &row, &col)) {
          if (f32) {
            const float* src = (const float*)a.X + row * a.ldx + col;
            cp_async16(rbase + e * 32, src);
            cp_async16(rbase + e * 32 + 16, src + 4);
          } else {
            cp_async16(rbase + e * 16, (const __nv_bfloat16*)a.X + row * a.ldx + col);
          }
        }
      }
    };
    for (int d = 0; d < kPrefetch; ++d) {
      issue(ld, d);
      cp_async_commit();
      ld.next(a, nitems);
    }
    uint32_t u = 0;
    bool ok = true;
    while (cv.valid) {
      issue(ld, (u + kPrefetch) % kRawSlots);
      cp_async_commit();
      ld.next(a, nitems);
      cp_async_wait<kPrefetch>();  // this thread's loads of stage u have landed
      const int s = u % kNS;
      if (!mbar_wait(su32(&bars->empty[s]), ((u / kNS) & 1) ^ 1, abort_flag)) { ok = false; break; }
      unsigned char* base = smem + s * kStageBytes;
      const int npan = (cv.ti == cv.tj) ? 1 : 2;
      if (tf32) {
        // items: (panel, 4-row quad, column); loads first, then one 16-byte
        // K-major chunk per item
        const int nit = npan * (kKS / 4) * kTile;
        float w[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int e = ct + j * (kConvWarps * 32);
          const int mn = e & (kTile - 1), kq = (e >> 7) & (kKS / 4 - 1), pan = e >> 10;
          const int col = (pan == 0 ? cv.ti : cv.tj) * kTile + mn;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int64_t sr = cv.r0 + (int64_t)cv.st * kKS + kq * 4 + i;
            w[j][i] = (e < nit && sr < cv.r1) ? zval_f32(a, a.perm ? (int64_t)a.perm[sr] : sr, col) : 0.f;
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int e = ct + j * (kConvWarps * 32);
          if (e < nit) {
            const int mn = e & (kTile - 1), kq = (e >> 7) & (kKS / 4 - 1), pan = e >> 10;
            *reinterpret_cast<uint4*>(base + pan * 16384 + off_kmaj_f32(mn, kq)) =
                make_uint4(to_tf32(w[j][0]), to_tf32(w[j][1]), to_tf32(w[j][2]), to_tf32(w[j][3]));
          }
        }
      } else {
        const unsigned char* rs = raw + (u % kRawSlots) * kRawBytes;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int e = ct + j * (kConvWarps * 32);
          if (e >= npan * kKS * 16) break;
          int64_t row;
          int col;
          float v[8];
          if (item_async(a, cv, e, &row, &col)) {
            if (f32) {
              const float4 q0 = *reinterpret_cast<const float4*>(rs + e * 32);
              const float4 q1 = *reinterpret_cast<const float4*>(rs + e * 32 + 16);
              v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
              v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
            } else {
              const uint4 q = *reinterpret_cast<const uint4*>(rs + e * 16);
              const uint32_t wq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                v[2 * i] = __uint_as_float(wq[i] << 16);
                v[2 * i + 1] = __uint_as_float(wq[i] & 0xFFFF0000u);
              }
            }
          } else if (row >= 0) {
            load8(a, row, col, v);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = 0.f;
          }
          const int g = e & 15, r = (e >> 4) & (kKS - 1), pan = e >> 9;
          unsigned char* ph = base + pan * 16384;
          const uint32_t o = off_bf16(g * 8, r);
          uint4 hi, lo;
          if (a.shift) {
            float m[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) m[i] = row >= 0 ? zshift(a, col + i) : 0.f;
            split8_shift(v, m, hi, lo);
          } else {
            split8(v, hi, lo);
          }
          *reinterpret_cast<uint4*>(ph + o) = hi;
          if (split) *reinterpret_cast<uint4*>(ph + 8192 + o) = lo;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(su32(&bars->full[s]));
      cv.next(a, nitems);
      ++u;
    }
    cp_async_wait<0>();
    if (!ok) { bars->abort = 1; atomicOr(a.dstatus, kStatTimeout); }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

}  // namespace tc

size_t gram_tc_smem_bytes() {
  return (size_t)tc::kNS * tc::kStageBytes + (size_t)tc::kRawSlots * tc::kRawBytes +
         sizeof(tc::Bars) + 1024;
}

cudaError_t launch_gram_tc(const GramArgs& a, int flush_rows, cudaStream_t s) {
  if (flush_rows <= 0) flush_rows = 256;
  const int flush_stages = (flush_rows + tc::kKS - 1) / tc::kKS;
  const size_t smem = gram_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(tc::gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = kNumSMsHint;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t items = (int64_t)a.max_chunks * a.ntiles;
  const int grid = (int)(items < sms ? items : sms);
  tc::gram_tc_kernel<<<grid, tc::kThreads, smem, s>>>(a, flush_stages);
  return cudaGetLastError();
}

}  // namespace oem
