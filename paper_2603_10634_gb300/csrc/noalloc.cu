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
// array and each call overwrites it (the per-call state that must start at zero, the
// flag word included, is cleared by the call itself), so two calls whose work overlaps
// on the GPU, on different streams or from different threads, race and corrupt each
// other's results.  The flag word of the last call is read by
// ozk2_noalloc_device_status.
//
// Loading: this translation unit is its own module.  With lazy module loading (the CUDA
// default) the array is reserved on a device at the first cudaGetSymbolAddress, which is
// where a device without room for it fails (OZK2_ERR_CUDA from the first call); with
// CUDA_MODULE_LOADING=EAGER every process that loads the library reserves it on every
// device it initialises, whether or not it ever calls this entry point.
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
  // argument errors and the products that need no workspace (m or n = 0: nothing to do;
  // k = 0: C = 0) behave exactly as in ozk2_dgemm, before the size limit applies
  const int v = ozk2::validate_dgemm(m, n, k, A, lda, B, ldb, C, ldc, num_moduli);
  if (v != OZK2_OK) return static_cast<ozk2_status>(v);
  if (m == 0 || n == 0 || k == 0)
    return ozk2_dgemm(m, n, k, A, lda, B, ldb, C, ldc, num_moduli, stream);
  const size_t need = ozk2_workspace_size(m, n, k, num_moduli);
  if (need == 0) return OZK2_ERR_INTERNAL;  // validated sizes always have a workspace size
  if (need > static_cast<size_t>(OZK2_NOALLOC_MAX_BYTES)) return OZK2_ERR_UNSUPPORTED;
  void* ws = nullptr;
  const ozk2_status s = noalloc_workspace(&ws);
  if (s != OZK2_OK) return s;
  return static_cast<ozk2_status>(ozk2::dgemm_library_ws(m, n, k, A, lda, B, ldb, C, ldc, num_moduli, ws,
                                                          static_cast<size_t>(OZK2_NOALLOC_MAX_BYTES),
                                                          reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" ozk2_status ozk2_noalloc_device_status(ozk2_stream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OZK2_ERR_CUDA;
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    ws = g_noalloc_ptr[dev];
  }
  if (!ws) {  // no ozk2_dgemm_noalloc call has run on this device: nothing was recorded
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return OZK2_ERR_CUDA;
    return OZK2_OK;
  }
  return ozk2_device_status(ws, stream);
}
