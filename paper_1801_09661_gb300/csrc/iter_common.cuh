// Device helpers shared by the two OEM iteration kernels (oem_iter.cu:
// replicated update, oem_iter_rows.cu: row-owned update for very large p):
// warp reductions, the mat-vec's reduce-scatter, the float32 dbeta layout,
// and the asynchronous DSMEM stores of the cluster-mode exchange.
#pragma once

#include "oem_internal.cuh"

namespace oem {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
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

// Reduce-scatter of V (4, 8 or 16) per-lane values over the warp: returns,
// in lane l, the warp sum of value l / (32 / V) (the 32 / V lanes of a group
// all hold it). The levels at lane offsets 16, 8, ... halve the values a lane
// keeps until one is left; the remaining offsets add plainly. The pairing
// tree of every value is the same as a full butterfly sum's.
template <int V, typename T>
__device__ __forceinline__ T reduce_scatter(const T (&a)[V], int lane) {
  static_assert(V == 4 || V == 8 || V == 16, "V");
  T b[V];
#pragma unroll
  for (int q = 0; q < V; ++q) b[q] = a[q];
  int n = V, o = 16;
#pragma unroll
  for (int lv = 0; lv < 5; ++lv, o >>= 1) {
    if (n > 1) {
      const bool up = lane & o;
      const int h = n >> 1;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < h) b[q] = (up ? b[q + h] : b[q]) + __shfl_xor_sync(0xffffffffu, up ? b[q] : b[q + h], o);
      n = h;
    } else {
      b[0] += __shfl_xor_sync(0xffffffffu, b[0], o);
    }
  }
  return b[0];
}

// The same for V = 1 or 2 (one or two full butterfly sums; every lane holds
// them): lane l returns the sum of value l / (32 / V).
template <int V, typename T>
__device__ __forceinline__ T reduce_scatter_any(const T (&a)[V], int lane) {
  if constexpr (V >= 4) {
    return reduce_scatter<V>(a, lane);
  } else {
    T r = T(0);
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const T sq = warp_sum(a[q]);
      if (lane / (32 / V) == q) r = sq;
    }
    return r;
  }
}

// Load the M entries of row j of a [rows][M] buffer.
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
  } else if constexpr (sizeof(T) == 4 && M == 2) {
    *reinterpret_cast<float2*>(dst) = *reinterpret_cast<const float2*>(src);
  } else if constexpr (sizeof(T) == 8 && M % 2 == 0) {
#pragma unroll
    for (int k = 0; k < M; k += 2)
      *reinterpret_cast<double2*>(dst + k) = *reinterpret_cast<const double2*>(src + k);
  } else {
#pragma unroll
    for (int k = 0; k < M; ++k) dst[k] = src[k];
  }
}

// Position of element (row i, instance k) in a dbeta buffer [rows][M]. In
// the float32 path a lane reads 4 consecutive rows (M float4 units) at a
// time; the 16-byte units are XOR-swizzled within each run of 8 units by
// (unit / 8) mod M, so that the 8 lanes of a shared-memory wavefront hit 8
// different bank groups. The float64 path keeps the plain layout.
template <typename T, int M>
__device__ __forceinline__ int dpos(int i, int k) {
  const int f = i * M + k;
  if constexpr (sizeof(T) == 4 && M > 1) {
    const int u = f >> 2;
    return ((u ^ ((u >> 3) & (M - 1))) << 2) | (f & 3);
  } else {
    return f;
  }
}
// Store the M values of row i (src[0..M)) at their positions in D.
template <typename T, int M>
__device__ __forceinline__ void store_row(T* __restrict__ D, int i, const T* __restrict__ src) {
  if constexpr (sizeof(T) == 4 && M == 8) {
    store_col<T, 4>(D + dpos<T, M>(i, 0), src);
    store_col<T, 4>(D + dpos<T, M>(i, 4), src + 4);
  } else {
    store_col<T, M>(D + dpos<T, M>(i, 0), src);
  }
}

// Order-preserving 32-bit images of non-negative maxima for the block table
// and the DSMEM atomic max (32-bit atomics only across the cluster). A
// float64 value is rounded up to float32 first, so a max|dbeta| is never
// under-stated and no convergence is declared early; max|beta| moves by at
// most 2^-24 relative.
__device__ __forceinline__ float to_red(float v) { return v; }
__device__ __forceinline__ float to_red(double v) { return __double2float_ru(v); }
__device__ __forceinline__ float from_red(unsigned int b) { return __uint_as_float(b); }

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Cluster-mode exchange by asynchronous stores: st.async writes into a peer
// CTA's shared memory and counts its bytes on that CTA's mbarrier, so each
// CTA waits for exactly the bytes addressed to it (no cluster barrier).
__device__ __forceinline__ uint32_t xs_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t xs_map(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void xs_st4(uint32_t a, float4 v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
               ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar) : "memory");
}
__device__ __forceinline__ void xs_st1(uint32_t a, uint32_t v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];"
               ::"r"(a), "r"(v), "r"(bar) : "memory");
}
__device__ __forceinline__ void xs_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void xs_arm(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool xs_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// mbarrier with `count` arrivals per phase; a plain arrival (release, CTA
// scope: the arriving thread's earlier shared-memory writes are visible to
// every thread that has seen the phase complete).
__device__ __forceinline__ void xs_init_n(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void xs_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Grid-mode exchange words: a 32-bit payload in the low half and the number
// of the exchange it belongs to in the high half, written and read as one
// 64-bit access (single-copy atomic), so that a reader that sees the tag it
// expects also sees that exchange's payload, with no flag and no fence.
__device__ __forceinline__ unsigned long long tag_word(uint32_t bits, uint32_t tag) {
  return ((unsigned long long)tag << 32) | bits;
}
__device__ __forceinline__ void st_tag1(unsigned long long* a, unsigned long long w) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(a), "l"(w) : "memory");
}
__device__ __forceinline__ void st_tag2(unsigned long long* a, unsigned long long w0, unsigned long long w1) {
  asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(a), "l"(w0), "l"(w1) : "memory");
}
__device__ __forceinline__ unsigned long long ld_tag1(const unsigned long long* a) {
  unsigned long long w;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(a) : "memory");
  return w;
}
__device__ __forceinline__ void ld_tag2(const unsigned long long* a, unsigned long long& w0,
                                        unsigned long long& w1) {
  asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(w0), "=l"(w1) : "l"(a) : "memory");
}

}  // namespace oem
