// Gram pass on the 5th-generation tensor cores (tcgen05, sm_103a): per-fold
// partial upper triangles of Z^T Z, Z = [X | y-columns] (Section 3: the
// O(np^2) step that forms X_k^T X_k, X_k^T y_k for every fold in one pass).
//
// One CTA per SM (persistent). A work item is a 128 x 128 tile (ti <= tj) of
// the upper triangle over a chunk of fold-sorted rows. Roles per CTA:
//   * 8 converter warps load 32-row stages of columns [128 ti, +128) and
//     [128 tj, +128) (rows gathered through the fold permutation), convert
//     them (float32 -> hi/lo bfloat16 split, bfloat16 copy, or float32 ->
//     tf32) and store them in shared memory in the MN-major, 128-byte-swizzled
//     layout the tensor core reads;
//   * 1 warp allocates tensor memory and one elected thread issues
//     tcgen05.mma (M = N = 128, float32 accumulation in tensor memory) for
//     each stage, double-buffering the accumulator per flush window;
//   * 4 epilogue warps (one per 32 tensor-memory lanes) add each finished
//     window into a compensated (hi, lo) float32 pair kept in tensor memory
//     (TwoSum), and write hi + lo as float64 at the end of the item.
// Every mbarrier wait is bounded by a clock budget; on expiry the kernel
// records a timeout in the status word, drains its MMAs, frees tensor memory
// and returns.
#include "oem_internal.cuh"

#include <cuda_bf16.h>

namespace oem {

namespace tc {

constexpr int kTile = 128;
constexpr int kKS = 32;           // rows per stage
constexpr int kNS = 4;            // pipeline stages
constexpr int kStageBytes = 32768;
constexpr int kGuardBytes = 32768;  // unused slack after the stages: every descriptor
                                    // reading stays inside the allocation
constexpr int kConvWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kThreads = (kEpiWarps + 1 + kConvWarps) * 32;  // 416
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

struct Bars {
  unsigned long long full[kNS];
  unsigned long long empty[kNS];
  unsigned long long acc_full[2];
  unsigned long long acc_empty[2];
  unsigned long long drain;
  unsigned tmem_base;
  int abort;
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait. Returns false on timeout or when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

#define OEM_R16(x) "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), \
    "=r"(x[6]), "=r"(x[7]), "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]), \
    "=r"(x[13]), "=r"(x[14]), "=r"(x[15])
#define OEM_W16(x) "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), \
    "r"(x[7]), "r"(x[8]), "r"(x[9]), "r"(x[10]), "r"(x[11]), "r"(x[12]), "r"(x[13]), \
    "r"(x[14]), "r"(x[15])

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : OEM_R16(r)
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      OEM_W16(r)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: start, leading (MN-atom) and stride
// (8-row K group) byte offsets, fixed version bit, 128-byte swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: float32 D, A/B format fmt (1 = bf16, 2 = tf32),
// operands MN-major (mn = 1) or K-major (mn = 0), N = M = 128.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t mn) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (mn << 15) | (mn << 16) | ((uint32_t)(kTile >> 3) << 17) |
         ((uint32_t)(kTile >> 4) << 24);
}

// K-major float32 / tf32 panel (128 MN rows x 32 K): 8-row groups 1024 B
// apart, each row 128 B of K-contiguous data, 16-byte chunks (4 K values)
// XOR-swizzled by the row. Offset of the chunk holding K rows [4 kq, 4 kq+4)
// of MN index mn.
__device__ __forceinline__ uint32_t off_kmaj_f32(int mn, int kq) {
  return (uint32_t)((mn >> 3) * 1024 + (mn & 7) * 128 + ((kq ^ (mn & 7)) << 4));
}

// One element of Z = [X | y] (tf32 mode: one y column).
__device__ __forceinline__ float zval_f32(const GramArgs& a, int64_t row, int col) {
  if (col < a.p) return ((const float*)a.X)[row * a.ldx + col];
  if (col == a.p) return ((const float*)a.y)[row];
  return 0.f;
}

// Byte offset of the 16-byte chunk holding MN elements [mn, mn+8) (bf16) at
// K row k in a 128 x 32 panel: MN atoms of 64 elements 4096 B apart, K groups
// of 8 rows 1024 B apart, rows 128 B apart, chunks XOR-swizzled by the row.
__device__ __forceinline__ uint32_t off_bf16(int mn, int k) {
  return (uint32_t)((mn >> 6) * 4096 + (k >> 3) * 1024 + (k & 7) * 128 +
                    ((((mn & 63) >> 3) ^ (k & 7)) << 4));
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}
__device__ __forceinline__ float bf16_round(float a) {
  return __bfloat162float(__float2bfloat16_rn(a));
}
__device__ __forceinline__ uint32_t to_tf32(float a) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
  return r;
}

// Values of Z at 8 consecutive columns [c0, c0+8) of original row `row`.
__device__ __forceinline__ void load8(const GramArgs& a, int64_t row, int c0, float (&v)[8]) {
  const int p = (int)a.p;
  if (c0 + 8 <= p) {
    if (a.xtype == OEM_F32) {
      const float4* s = reinterpret_cast<const float4*>((const float*)a.X + row * a.ldx + c0);
      const float4 u0 = __ldg(s), u1 = __ldg(s + 1);
      v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
      v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
    } else {
      const uint4 u = __ldg(reinterpret_cast<const uint4*>((const __nv_bfloat16*)a.X + row * a.ldx + c0));
      const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        v[2 * i] = __uint_as_float(w[i] << 16);
        v[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
      }
    }
    return;
  }
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
    }
    v[u] = x;
  }
}

__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(GramArgs a, int flush_stages) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the operand stages (swizzle atoms)
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Bars* bars = reinterpret_cast<Bars*>(smem + kNS * kStageBytes + kGuardBytes);
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
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
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
        for (int cb = 0; cb < kTile; cb += 16) {
          uint32_t ra[16], rh[16], rl[16];
          tmem_ld16(acc + cb, ra);
          if (!first) { tmem_ld16(thi + cb, rh); tmem_ld16(tlo + cb, rl); }
          tmem_ld_wait();
          if (first) {
#pragma unroll
            for (int i = 0; i < 16; ++i) { rh[i] = ra[i]; rl[i] = 0u; }
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float h = __uint_as_float(rh[i]), x = __uint_as_float(ra[i]);
              const float s = h + x, bb = s - h;
              const float e = (h - (s - bb)) + (x - bb);
              const float lo = __uint_as_float(rl[i]) + e;
              const float t = s + lo;
              rl[i] = __float_as_uint(lo - (t - s));
              rh[i] = __float_as_uint(t);
            }
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
      // item done: hi + lo as float64 (row 32 * warp + lane of the tile)
      double* out = a.partial + ((int64_t)chunk * a.ntiles + tile) * (kTile * kTile) +
                    (int64_t)(warp * 32 + lane) * kTile;
      const uint32_t thi = tmem + lane_base + 256u, tlo = tmem + lane_base + 384u;
#pragma unroll 1
      for (int cb = 0; cb < kTile; cb += 16) {
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
    const int ct = threadIdx.x - (kEpiWarps + 1) * 32;  // 0..255
    uint32_t u = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int chunk = item / a.ntiles, tile = item % a.ntiles;
      int ti, tj;
      tile_coords(tile, a.ntile1, &ti, &tj);
      const bool diag = ti == tj;
      const int npan = diag ? 1 : 2;
      const int64_t r0 = a.ct.row0[chunk], r1 = a.ct.row1[chunk];
      const int nst = (int)((r1 - r0 + kKS - 1) / kKS);
      for (int st = 0; st < nst; ++st, ++u) {
        const int s = u % kNS;
        if (!mbar_wait(su32(&bars->empty[s]), ((u / kNS) & 1) ^ 1, abort_flag)) { ok = false; break; }
        unsigned char* base = smem + s * kStageBytes;
        const int64_t rb = r0 + (int64_t)st * kKS;
        if (tf32) {
          // items: (panel, 4-row quad, column); one 16-byte chunk each
          for (int e = ct; e < npan * (kKS / 4) * kTile; e += kConvWarps * 32) {
            const int mn = e & (kTile - 1), kq = (e >> 7) & (kKS / 4 - 1), pan = e >> 10;
            const int col = (pan == 0 ? ti : tj) * kTile + mn;
            uint32_t w4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int64_t sr = rb + kq * 4 + i;
              float x = 0.f;
              if (sr < r1) x = zval_f32(a, a.perm ? (int64_t)a.perm[sr] : sr, col);
              w4[i] = to_tf32(x);
            }
            *reinterpret_cast<uint4*>(base + pan * 16384 + off_kmaj_f32(mn, kq)) =
                make_uint4(w4[0], w4[1], w4[2], w4[3]);
          }
        }
        // items: (panel, row, 8-column group), group fastest
        for (int e = ct; !tf32 && e < npan * kKS * 16; e += kConvWarps * 32) {
          const int g = e & 15, r = (e >> 4) & (kKS - 1), pan = e >> 9;
          const int64_t sr = rb + r;
          float v[8];
          if (sr < r1) {
            const int64_t row = a.perm ? (int64_t)a.perm[sr] : sr;
            load8(a, row, (pan == 0 ? ti : tj) * kTile + g * 8, v);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = 0.f;
          }
          unsigned char* ph = base + pan * 16384;
          uint4 hi;
          hi.x = pack_bf16(v[0], v[1]); hi.y = pack_bf16(v[2], v[3]);
          hi.z = pack_bf16(v[4], v[5]); hi.w = pack_bf16(v[6], v[7]);
          const uint32_t o = off_bf16(g * 8, r);
          *reinterpret_cast<uint4*>(ph + o) = hi;
          if (split) {
            uint4 lo;
            lo.x = pack_bf16(v[0] - bf16_round(v[0]), v[1] - bf16_round(v[1]));
            lo.y = pack_bf16(v[2] - bf16_round(v[2]), v[3] - bf16_round(v[3]));
            lo.z = pack_bf16(v[4] - bf16_round(v[4]), v[5] - bf16_round(v[5]));
            lo.w = pack_bf16(v[6] - bf16_round(v[6]), v[7] - bf16_round(v[7]));
            *reinterpret_cast<uint4*>(ph + 8192 + o) = lo;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(su32(&bars->full[s]));
      }
    }
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

cudaError_t launch_gram_tc(const GramArgs& a, int flush_rows, cudaStream_t s) {
  if (flush_rows <= 0) flush_rows = 256;
  const int flush_stages = (flush_rows + tc::kKS - 1) / tc::kKS;
  const size_t smem = (size_t)tc::kNS * tc::kStageBytes + tc::kGuardBytes + sizeof(tc::Bars) + 1024;
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
