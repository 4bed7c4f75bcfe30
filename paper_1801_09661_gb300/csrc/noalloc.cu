// oem_gram_noalloc: the full-data Gram pass (same kernels as oem_gram) with
// all of its scratch in one file-scope device array, for callers that cannot
// allocate device memory at call time. See include/oem.h for the contract.
#include "oem_internal.cuh"

#include <algorithm>
#include <mutex>

namespace oem {

// The scratch every call shares: status word, chunk table, the reduced Z Gram
// and the tile partials. 48 MiB, held by every GPU that loads the library
// until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)48 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up once
// per device; the host-side symbol is not a device address).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Whether ptr is device (or managed) memory that the current device `dev`
// can use as this entry point's operand: host memory, pinned or not, and
// memory of another device are refused.
bool on_device(const void* ptr, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

// A device wait of the Gram pass that expired leaves its bit in the status
// word of the scratch array, which nobody reads back; this kernel turns it
// into NaN in every output so that the caller sees it.
__global__ void noalloc_flag_kernel(const unsigned* st, double* G, double* c, double* yty, int64_t p) {
  if ((*st & kStatTimeout) == 0) return;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  const int64_t n = p * p;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    G[i] = nan;
    if (i < p) c[i] = nan;
    if (i == 0) yty[0] = nan;
  }
}
}  // namespace oem

using namespace oem;

extern "C" int oem_gram_noalloc(const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
                                const void* y, int32_t mode, double* G, double* c, double* yty,
                                void* stream) {
  // ---- arguments (host checks only; nothing is launched on error)
  if (xtype != OEM_F64 && xtype != OEM_F32 && xtype != OEM_BF16) return OEM_EINVAL;
  if (n < 1 || p < 1 || n > INT32_MAX || ldx < p) return OEM_EINVAL;
  const int64_t esz = xtype == OEM_F64 ? 8 : xtype == OEM_F32 ? 4 : 2;
  if ((ldx * esz) % 16 != 0) return OEM_EINVAL;
  if (!X || !y || !G || !c || !yty) return OEM_EINVAL;
  if (((uintptr_t)X & 15) || ((uintptr_t)y & 15)) return OEM_EINVAL;
  if (p > 1024) return OEM_EBUDGET;  // the stated maximum of this entry point
  if (mode == OEM_GRAM_AUTO)
    mode = xtype == OEM_F64 ? OEM_GRAM_FP64 : xtype == OEM_BF16 ? OEM_GRAM_BF16 : OEM_GRAM_SPLIT_BF16;
  const bool tc = mode == OEM_GRAM_TF32 || mode == OEM_GRAM_BF16 || mode == OEM_GRAM_SPLIT_BF16;
  if (mode == OEM_GRAM_FP32 && xtype == OEM_F64) return OEM_EINVAL;
  if ((mode == OEM_GRAM_TF32 || mode == OEM_GRAM_SPLIT_BF16) && xtype != OEM_F32) return OEM_EINVAL;
  if (mode == OEM_GRAM_BF16 && xtype != OEM_BF16) return OEM_EINVAL;
  if (mode < OEM_GRAM_FP64 || mode > OEM_GRAM_SPLIT_BF16) return OEM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return OEM_ECUDA; }
    if (!on_device(X, dev) || !on_device(y, dev) || !on_device(G, dev) || !on_device(c, dev) ||
        !on_device(yty, dev))
      return OEM_EINVAL;
  }

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) { cudaGetLastError(); return OEM_ECUDA; }

  // ---- plan: tiles, and as many row chunks as the scratch holds
  GramArgs a{};
  a.X = X; a.xtype = xtype; a.n = n; a.p = p; a.ldx = ldx; a.y = y; a.perm = nullptr;
  a.mode = mode;
  a.ycols = mode == OEM_GRAM_BF16 ? 3 : 1;
  a.q = (int32_t)p + a.ycols;
  a.T = tc ? 128 : 64;
  a.ntile1 = (a.q + a.T - 1) / a.T;
  a.ntiles = a.ntile1 * (a.ntile1 + 1) / 2;
  int sms = kNumSMsHint, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t per_chunk = (size_t)a.ntiles * a.T * a.T * sizeof(double);
  const size_t table_max = 64 * 1024;  // chunk table for up to 2,900 chunks
  const size_t fixed = 256 + table_max + up256((size_t)a.q * a.q * sizeof(double)) + 256;
  if (fixed + per_chunk > kNoAllocScratchBytes) return OEM_EBUDGET;
  const int64_t cap = (int64_t)((kNoAllocScratchBytes - fixed) / per_chunk);
  const int64_t target = std::max<int64_t>(1, (4LL * sms + a.ntiles - 1) / a.ntiles);
  const int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(cap - 1, target));
  const int64_t align = tc ? 128 : 16;
  int64_t cr = (n + chunks - 1) / chunks;
  cr = std::max<int64_t>(tc ? 1024 : 256, (cr + align - 1) / align * align);
  a.max_chunks = (int)((n + cr - 1) / cr + 1);
  if ((size_t)a.max_chunks * (8 + 8 + 4) + 64 > table_max || a.max_chunks > cap) return OEM_EBUDGET;

  // ---- carve the scratch
  char* q = (char*)base;
  a.dstatus = (unsigned*)q;                      q += 256;
  char* t = q;                                    q += table_max;
  a.ct.row0 = (int64_t*)t;                        t += up256(sizeof(int64_t) * a.max_chunks);
  a.ct.row1 = (int64_t*)t;                        t += up256(sizeof(int64_t) * a.max_chunks);
  a.ct.fold = (int32_t*)t;                        t += up256(sizeof(int32_t) * a.max_chunks);
  a.ct.count = (int32_t*)t;                       t += 16;
  a.ct.fold_c0 = (int32_t*)t;                     t += 16;
  a.ct.fold_off = (int64_t*)t;                    t += 32;
  int64_t* nk = (int64_t*)t;
  double* Zg = (double*)q;                        q += up256((size_t)a.q * a.q * sizeof(double));
  a.partial = (double*)q;

  // ---- the status word must start at zero; everything else is overwritten
  cudaError_t e = cudaMemsetAsync(a.dstatus, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = launch_identity_chunks(n, cr, a.ct, a.max_chunks, s);
  if (e == cudaSuccess) e = tc ? launch_gram_tc(a, mode == OEM_GRAM_SPLIT_BF16 ? 32 :
                                                 mode == OEM_GRAM_TF32 ? 128 : 256, s)
                               : launch_gram_simt(a, s);
  if (e == cudaSuccess) e = launch_gram_reduce(a, 1, Zg, s);
  if (e == cudaSuccess)
    e = launch_extract_folds(Zg, 1, a.q, (int)p, a.ycols, G, c, yty, nk, a.ct.fold_off, s);
  if (e == cudaSuccess) {
    noalloc_flag_kernel<<<std::max<int>(1, (int)std::min<int64_t>(sms, (p * p + 255) / 256)), 256, 0, s>>>(
        a.dstatus, G, c, yty, p);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { cudaGetLastError(); return OEM_ECUDA; }
  return OEM_OK;
}
