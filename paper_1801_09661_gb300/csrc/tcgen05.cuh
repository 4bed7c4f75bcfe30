// tcgen05 / mbarrier building blocks shared by the Gram kernels: bounded
// mbarrier waits, MMA issue and commit, tensor-memory loads and stores,
// shared-memory matrix and instruction descriptors, the 128-byte-swizzled
// bfloat16 panel layout, and the float32 -> (hi, lo) bfloat16 split.
#pragma once

#include "oem_internal.cuh"

#include <cuda_bf16.h>

namespace oem {
namespace tc {

constexpr int kTile = 128;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz


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
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      OEM_W16(r)
      : "memory");
}
// (hi, lo) += x for two elements at once (packed float32x2): TwoSum gives
// s + e = hi + x exactly; s becomes hi and e is added to lo.
__device__ __forceinline__ void two_sum_x2(uint32_t& h0, uint32_t& h1, uint32_t& l0, uint32_t& l1,
                                           uint32_t x0, uint32_t x1) {
  asm("{\n\t.reg .b64 h, x, s, bb, t, e1, e2, l;\n\t"
      "mov.b64 h, {%0, %1};\n\t"
      "mov.b64 l, {%2, %3};\n\t"
      "mov.b64 x, {%4, %5};\n\t"
      "add.rn.f32x2 s, h, x;\n\t"
      "sub.rn.f32x2 bb, s, h;\n\t"
      "sub.rn.f32x2 t, s, bb;\n\t"
      "sub.rn.f32x2 e1, h, t;\n\t"
      "sub.rn.f32x2 e2, x, bb;\n\t"
      "add.rn.f32x2 e1, e1, e2;\n\t"
      "add.rn.f32x2 l, l, e1;\n\t"
      "mov.b64 {%0, %1}, s;\n\t"
      "mov.b64 {%2, %3}, l;\n\t}"
      : "+r"(h0), "+r"(h1), "+r"(l0), "+r"(l1)
      : "r"(x0), "r"(x1));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared-memory matrix descriptor: start, leading and stride byte offsets,
// fixed version bit, 128-byte swizzle.
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
// Two float32 values rounded to bfloat16 (nearest even) in one instruction;
// the first argument lands in the low half.
__device__ __forceinline__ uint32_t cvt_bf16x2(float lo_elem, float hi_elem) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_elem), "f"(lo_elem));
  return r;
}
// hi = bf16(v), lo = bf16(v - hi) for 8 values, packed in pairs.
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = cvt_bf16x2(v[2 * i], v[2 * i + 1]);
    const float h0 = __uint_as_float(h[i] << 16), h1 = __uint_as_float(h[i] & 0xFFFF0000u);
    l[i] = cvt_bf16x2(v[2 * i] - h0, v[2 * i + 1] - h1);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}
// The same split of v - m, with the difference taken exactly: TwoSum gives
// s + e = v - m, hi = bf16(s), lo = bf16((s - hi) + e).
__device__ __forceinline__ void split8_shift(const float (&v)[8], const float (&m)[8], uint4& hi,
                                             uint4& lo) {
  float sv[8], ev[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float a = v[i], b = -m[i];
    const float s = a + b;
    const float bb = s - a;
    sv[i] = s;
    ev[i] = (a - (s - bb)) + (b - bb);
  }
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = cvt_bf16x2(sv[2 * i], sv[2 * i + 1]);
    const float h0 = __uint_as_float(h[i] << 16), h1 = __uint_as_float(h[i] & 0xFFFF0000u);
    l[i] = cvt_bf16x2((sv[2 * i] - h0) + ev[2 * i], (sv[2 * i + 1] - h1) + ev[2 * i + 1]);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}
}  // namespace tc
}  // namespace oem
