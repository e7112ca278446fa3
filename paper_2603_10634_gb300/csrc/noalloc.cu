// ozk2_dgemm_noalloc: the emulated DGEMM for callers that must not allocate device
// memory, running in a workspace that is a static device array of this library.
//
// Who needs it: a program whose device memory is owned by someone else (a host
// application that hands a plug-in a fixed budget, a framework whose caching
// allocator already reserved the GPU), and code that must not stall: growing the
// library-owned workspace of ozk2_dgemm calls cudaFree and cudaMalloc, and both can
// synchronise the whole device.  This entry point calls neither, nor any other
// allocating routine; it runs the same kernels as ozk2_dgemm_ws in the array below.
//
// Limits and sharing: the array holds OZK2_NOALLOC_MAX_BYTES bytes on every GPU that
// loads this part of the library, until the process exits.  Problems whose
// ozk2_workspace_size exceeds it are rejected.  All calls on a device share the one
// array and each call overwrites it (the per-call state that must start at zero is
// cleared by the call itself), so two calls whose work overlaps on the GPU, on
// different streams or from different threads, race and corrupt each other's results.
#include <mutex>

#include "internal.h"
#include "ozk2.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_workspace[OZK2_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device.  The first call on a device
// looks it up with cudaGetSymbolAddress (which may load this module on that device);
// later calls reuse the cached address.
ozk2_status noalloc_workspace(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OZK2_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_workspace) != cudaSuccess || !p) {
      cudaGetLastError();
      return OZK2_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return OZK2_OK;
}

}  // namespace

extern "C" ozk2_status ozk2_dgemm_noalloc(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                                          const double* B, int64_t ldb, double* C, int64_t ldc, int num_moduli,
                                          ozk2_stream_t stream) {
  const size_t need = ozk2_workspace_size(m, n, k, num_moduli);
  if (need == 0) return OZK2_ERR_INVALID_VALUE;
  if (need > static_cast<size_t>(OZK2_NOALLOC_MAX_BYTES)) return OZK2_ERR_UNSUPPORTED;
  void* ws = nullptr;
  const ozk2_status s = noalloc_workspace(&ws);
  if (s != OZK2_OK) return s;
  return ozk2_dgemm_ws(m, n, k, A, lda, B, ldb, C, ldc, num_moduli, ws, static_cast<size_t>(OZK2_NOALLOC_MAX_BYTES),
                       stream);
}
