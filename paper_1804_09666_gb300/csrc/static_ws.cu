// static_ws.cu -- band_solve_static: the NTDM / NPDM solve without a caller workspace.
//
// Some callers cannot allocate device memory at the point where they solve: code that
// runs where cudaMalloc would synchronise the whole device (a latency-critical loop
// between kernel launches), hosts that hand every byte of device memory to their own
// pool and forbid other allocations, or plain C callers with no allocator at all.
// For them this entry point runs band_solve's own path (every schedule) with its
// workspace in a fixed array in device memory that the library owns:
// kStaticScratchBytes per GPU, held from the first use of the library on that GPU
// until the process exits.
//
// Every call shares the array and it keeps whatever the last call wrote: calls whose
// kernels overlap on a GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.  Nothing in the array needs to start at
// zero (every row is written by the forward sweep before the backward sweep reads it).
#include <mutex>

#include "api_util.h"
#include "kernels.h"

namespace {

constexpr size_t kStaticScratchBytes = BAND_STATIC_SCRATCH_BYTES;   // 32 MiB per GPU
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Is p still device memory of the current device's context?  A cudaDeviceReset ends the
// context the address was looked up in; the lookup is then repeated.  (A failed query's
// error is taken off the runtime's last-error slot, so later launch checks do not see it.)
bool still_mapped(void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Device address of g_scratch on the current device: looked up on the first call on
// that device (with it current), and again if the device was reset since.  In host code
// `g_scratch` is only a host-side stand-in for the symbol, never a device address.
cudaError_t scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_ptr[dev] && !still_mapped(g_ptr[dev], dev)) g_ptr[dev] = nullptr;
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

}  // namespace

using namespace band;

extern "C" band_status band_solve_static(const band_desc* desc, int32_t method,
                                         const void* const diag[5], const void* f, void* x,
                                         int32_t* sys_status, void* stream) {
  if (!desc_ok(desc) || desc->systems) return BAND_ERR_ARG;
  if (method != BAND_NTDM && method != BAND_NPDM && method != BAND_AUTO_NUMERIC)
    return BAND_ERR_ARG;
  const int kmode = kmode_for(desc, method);
  if (kmode < 0) return BAND_ERR_ARG;
  const size_t need = single_solve_bytes(desc, method);   // band_solve's workspace
  if (need > kStaticScratchBytes) return BAND_ERR_WORKSPACE;   // batch too large
  if (desc->nsys == 0) return BAND_OK;
  if (!diag || !f || !x || !diag[1] || !diag[2] || !diag[3]) return BAND_ERR_ARG;
  if (may_be_pd(desc) && kmode != 1 && (!diag[0] || !diag[4])) return BAND_ERR_ARG;
  void* base = nullptr;
  if (scratch_on_current_device(&base) != cudaSuccess) return BAND_ERR_CUDA;
  // from here on band_solve's own path, with the static array as its workspace
  return run_single(desc, method, diag, f, x, sys_status, base, kStaticScratchBytes,
                    static_cast<cudaStream_t>(stream));
}
