// Allocation-free variant of the tensor-core Gram (lobpcg_gram_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// Gram: code running inside a framework that owns the whole memory pool,
// callbacks executed while a caller holds an allocator lock, or real-time
// loops that forbid cudaMalloc/cudaFree because they synchronise the device.
// For them this entry point takes its scratch (the per-slab partial sums)
// from a fixed array in the library's own device memory instead of asking for
// it.  The array lives in every GPU that loads the library until the process
// exits.
#include <mutex>

#include "kernels.cuh"

namespace {

constexpr int64_t kScratchBytes = 16ll << 20;  // 16 MiB of slab partials

// The scratch.  In host code `g_gram_scratch` names a host-side shadow, not a
// device address: it must never be passed to a kernel.  The device address is
// obtained per device with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_gram_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Once per device, with that device current: the device address of the array.
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return LOBPCG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gram_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LOBPCG_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return LOBPCG_OK;
}

}  // namespace

LOBPCG_EXPORT int lobpcg_gram_noalloc(int64_t n, const double* U, int64_t ldu, int64_t p,
                                      const double* V, int64_t ldv, int64_t q, double* G,
                                      int64_t ldg, int slices, void* stream) {
  if (n < 0 || p < 0 || q < 0 || p > (1 << 20) || q > (1 << 20)) return LOBPCG_ERR_ARG;
  if (p == 0 || q == 0) return LOBPCG_OK;
  if (!G || ldg < p || (n > 0 && (!U || ldu < p || !V || ldv < q))) return LOBPCG_ERR_ARG;
  if (slices != 0 && (slices < 3 || slices > 7)) return LOBPCG_ERR_ARG;
  // One slab needs p * q partials of 16 bytes: larger Grams do not fit.
  if (p * q * 16 > kScratchBytes) return LOBPCG_ERR_ARG;
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  return lob::gram_ozaki_bounded((cudaStream_t)stream, n, lob::seg1(U, ldu, (int)p),
                                 lob::seg1(V, ldv, (int)q), G, ldg, slices, scratch,
                                 kScratchBytes);
}
