// Gram pass on CUDA cores (float64 and float32 modes): per-fold partial upper
// triangles of Z^T Z, Z = [X | y] (Section 3: X_k^T X_k, X_k^T y_k, y_k^T y_k).
// One work item = (64 x 64 tile of the upper triangle, chunk of fold-sorted
// rows); it writes a float64 partial that the reduction adds per fold.
#include "oem_internal.cuh"

#include <cuda_bf16.h>

namespace oem {

constexpr int kT = 64;      // tile edge
constexpr int kRS = 16;     // rows staged per step
constexpr int kF32Block = 256;  // rows summed in float32 before adding to float64

// One element of Z = [X | y | 1]. With a column shift (centring) the
// difference is taken in float64 and rounded once to A.
template <typename A>
__device__ __forceinline__ A zval(const GramArgs& a, int64_t row, int col) {
  if (col < a.p) {
    int64_t o = row * a.ldx + col;
    if (a.shift) {
      const double x = a.xtype == OEM_F64   ? ((const double*)a.X)[o]
                       : a.xtype == OEM_F32 ? (double)((const float*)a.X)[o]
                                            : (double)__bfloat162float(((const __nv_bfloat16*)a.X)[o]);
      return (A)(x - (double)a.shift[col]);
    }
    if (a.xtype == OEM_F64) return (A)((const double*)a.X)[o];
    if (a.xtype == OEM_F32) return (A)((const float*)a.X)[o];
    return (A)__bfloat162float(((const __nv_bfloat16*)a.X)[o]);
  }
  if (col == a.p) {
    const double yv = a.xtype == OEM_F64 ? ((const double*)a.y)[row] : (double)((const float*)a.y)[row];
    if (a.shift) return (A)(yv - (double)a.shift[a.p]);
    return (A)yv;
  }
  if (col == a.p + 1 && a.ocols) return (A)1;
  return (A)0;
}

template <typename A>
__global__ void __launch_bounds__(256) gram_simt_kernel(GramArgs a) {
  __shared__ A As[kRS][kT + 4];
  __shared__ A Bs[kRS][kT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int nitems = *a.ct.count * a.ntiles;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int chunk = item / a.ntiles, tile = item % a.ntiles;
    int ti, tj;
    tile_coords(tile, a.ntile1, &ti, &tj);
    const int64_t r0 = a.ct.row0[chunk], r1 = a.ct.row1[chunk];
    double acc64[4][4];
    A acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { acc64[i][j] = 0.0; acc[i][j] = (A)0; }
    int in_block = 0;
    for (int64_t rb = r0; rb < r1; rb += kRS) {
      for (int e = tid; e < kRS * kT; e += blockDim.x) {
        const int rr = e / kT, cc = e % kT;
        const int64_t srow = rb + rr;
        A va = (A)0, vb = (A)0;
        if (srow < r1) {
          const int64_t row = a.perm ? (int64_t)a.perm[srow] : srow;
          va = zval<A>(a, row, ti * kT + cc);
          vb = (ti == tj) ? va : zval<A>(a, row, tj * kT + cc);
        }
        As[rr][cc] = va;
        Bs[rr][cc] = vb;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kRS; ++k) {
        A av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) { av[i] = As[k][ty * 4 + i]; bv[i] = Bs[k][tx * 4 + i]; }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
      in_block += kRS;
      if (in_block >= kF32Block) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) { acc64[i][j] += (double)acc[i][j]; acc[i][j] = (A)0; }
        in_block = 0;
      }
    }
    double* out = a.partial + ((int64_t)chunk * a.ntiles + tile) * (kT * kT);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        out[(ty * 4 + i) * kT + tx * 4 + j] = acc64[i][j] + (double)acc[i][j];
  }
}

cudaError_t launch_gram_simt(const GramArgs& a, cudaStream_t s) {
  const int64_t items = (int64_t)a.max_chunks * a.ntiles;
  const int grid = (int)(items < 8 * kNumSMsHint ? items : 8 * kNumSMsHint);
  if (a.mode == OEM_GRAM_FP64)
    gram_simt_kernel<double><<<grid, 256, 0, s>>>(a);
  else
    gram_simt_kernel<float><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace oem
