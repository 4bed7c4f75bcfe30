// Fold partition of the rows (Section 3: X is randomly partitioned into K
// submatrices X_1..X_K). A stable counting sort of row indices by fold label
// lets the Gram pass visit each fold's rows contiguously, so every fold's
// partial sums X_k^T X_k come out of one pass over X.
#include "oem_internal.cuh"

namespace oem {

constexpr int kSortRows = 1024;  // rows per block (one per thread)
constexpr int kMaxK = 64;

__global__ void fold_count_kernel(const uint8_t* __restrict__ fold, int64_t n, int K,
                                  int32_t* __restrict__ blk_counts) {
  __shared__ int32_t cnt[kMaxK];
  for (int k = threadIdx.x; k < K; k += blockDim.x) cnt[k] = 0;
  __syncthreads();
  int64_t r = (int64_t)blockIdx.x * kSortRows + threadIdx.x;
  if (r < n) {
    int f = fold[r];
    if (f < K) atomicAdd(&cnt[f], 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x)
    blk_counts[(int64_t)blockIdx.x * K + k] = cnt[k];
}

// One block: per-fold exclusive scan over blocks, fold offsets, chunk table.
__global__ void fold_scan_kernel(const int32_t* __restrict__ blk_counts, int64_t nblk, int K,
                                 int64_t chunk_rows, int32_t* __restrict__ blk_offsets,
                                 ChunkTable ct, int max_chunks, unsigned* dstatus,
                                 int require_nonempty) {
  __shared__ int64_t total[kMaxK + 1];
  int k = threadIdx.x;
  if (k < K) {
    int64_t s = 0;
    for (int64_t b = 0; b < nblk; ++b) s += blk_counts[b * K + k];
    total[k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t off = 0;
    int nc = 0;
    for (int f = 0; f < K; ++f) {
      ct.fold_off[f] = off;
      ct.fold_c0[f] = nc;
      int64_t nf = total[f];
      if (nf == 0 && require_nonempty) atomicOr(dstatus, kStatEmptyFold);
      for (int64_t r0 = off; r0 < off + nf; r0 += chunk_rows) {
        if (nc < max_chunks) {
          ct.row0[nc] = r0;
          ct.row1[nc] = (r0 + chunk_rows < off + nf) ? r0 + chunk_rows : off + nf;
          ct.fold[nc] = f;
        }
        ++nc;
      }
      off += nf;
      total[f] = ct.fold_off[f];  // reuse as running base for the block offsets
    }
    ct.fold_off[K] = off;
    ct.fold_c0[K] = nc < max_chunks ? nc : max_chunks;
    *ct.count = nc < max_chunks ? nc : max_chunks;
  }
  __syncthreads();
  if (k < K) {
    int64_t run = total[k];
    for (int64_t b = 0; b < nblk; ++b) {
      blk_offsets[b * K + k] = (int32_t)run;
      run += blk_counts[b * K + k];
    }
  }
}

__global__ void fold_scatter_kernel(const uint8_t* __restrict__ fold, int64_t n, int K,
                                    const int32_t* __restrict__ blk_offsets,
                                    int32_t* __restrict__ perm, int32_t* __restrict__ ipos,
                                    const int64_t* __restrict__ fold_off) {
  __shared__ int32_t wcnt[32][kMaxK];
  __shared__ int64_t padpre[kMaxK];  // zero rows of the packed copy before fold f
  if (ipos && threadIdx.x == 0) {
    int64_t run = 0;
    for (int k = 0; k < K; ++k) {
      padpre[k] = run;
      const int64_t nk = fold_off[k + 1] - fold_off[k];
      run += (nk + kGramPackRows - 1) / kGramPackRows * kGramPackRows - nk;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < 32 * kMaxK; i += blockDim.x) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  int64_t r = (int64_t)blockIdx.x * kSortRows + threadIdx.x;
  int f = (r < n) ? (int)fold[r] : -1;
  if (f >= K) f = -1;
  unsigned same = __match_any_sync(0xffffffffu, f);
  int rank = __popc(same & ((1u << lane) - 1u));
  if (f >= 0 && rank == 0) wcnt[warp][f] = __popc(same);
  __syncthreads();
  // exclusive prefix over warps, per fold (in place)
  if (threadIdx.x < K) {
    int run = 0;
    for (int w = 0; w < 32; ++w) {
      int v = wcnt[w][threadIdx.x];
      wcnt[w][threadIdx.x] = run;
      run += v;
    }
  }
  __syncthreads();
  if (f >= 0) {
    int64_t pos = (int64_t)blk_offsets[(int64_t)blockIdx.x * K + f] + wcnt[warp][f] + rank;
    perm[pos] = (int32_t)r;
    if (ipos) ipos[r] = (int32_t)(pos + padpre[f]);
  } else if (ipos && r < n) {
    ipos[r] = -1;
  }
}

__global__ void identity_chunks_kernel(int64_t n, int64_t chunk_rows, ChunkTable ct, int max_chunks) {
  int64_t nc = (n + chunk_rows - 1) / chunk_rows;
  if (nc > max_chunks) nc = max_chunks;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    ct.row0[c] = c * chunk_rows;
    ct.row1[c] = (c + 1) * chunk_rows < n ? (c + 1) * chunk_rows : n;
    ct.fold[c] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *ct.count = (int32_t)nc;
    ct.fold_c0[0] = 0;
    ct.fold_c0[1] = (int32_t)nc;
    ct.fold_off[0] = 0;
    ct.fold_off[1] = n;
  }
}

cudaError_t launch_fold_count(const uint8_t* fold, int64_t n, int K, int32_t* blk_counts,
                              int64_t nblk, cudaStream_t s) {
  fold_count_kernel<<<(unsigned)nblk, kSortRows, 0, s>>>(fold, n, K, blk_counts);
  return cudaGetLastError();
}

cudaError_t launch_fold_scan(const int32_t* blk_counts, int64_t nblk, int K, int64_t chunk_rows,
                             int32_t* blk_offsets, ChunkTable ct, int max_chunks,
                             unsigned* dstatus, int require_nonempty, cudaStream_t s) {
  fold_scan_kernel<<<1, kMaxK, 0, s>>>(blk_counts, nblk, K, chunk_rows, blk_offsets, ct,
                                       max_chunks, dstatus, require_nonempty);
  return cudaGetLastError();
}

cudaError_t launch_fold_scatter(const uint8_t* fold, int64_t n, int K, const int32_t* blk_offsets,
                                int32_t* perm, int32_t* ipos, const int64_t* fold_off, cudaStream_t s) {
  int64_t nblk = (n + kSortRows - 1) / kSortRows;
  fold_scatter_kernel<<<(unsigned)nblk, kSortRows, 0, s>>>(fold, n, K, blk_offsets, perm, ipos, fold_off);
  return cudaGetLastError();
}

cudaError_t launch_identity_chunks(int64_t n, int64_t chunk_rows, ChunkTable ct, int max_chunks,
                                   cudaStream_t s) {
  identity_chunks_kernel<<<8, 256, 0, s>>>(n, chunk_rows, ct, max_chunks);
  return cudaGetLastError();
}

}  // namespace oem
