// static_ws.cu -- band_solve_static: the NTDM / NPDM solve without a caller workspace.
//
// Some callers cannot allocate device memory at the point where they solve: code that
// runs where cudaMalloc would synchronise the whole device (a latency-critical loop
// between kernel launches), hosts that hand every byte of device memory to their own
// pool and forbid other allocations, or plain C callers with no allocator at all.
// For them this entry point takes its scratch rows (alpha and beta of the sweep) from
// a fixed array in device memory that the library owns: kStaticScratchBytes per GPU,
// held from the first use of the library on that GPU until the process exits.
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

// Device address of g_scratch on the current device (set up once per device).  In host
// code `g_scratch` is only a host-side stand-in for the symbol, never a device address.
cudaError_t scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
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
  const size_t esz = dtype_size(desc->dtype);
  const size_t rows = (size_t)spill_rows(desc);
  const size_t arr = (rows * esz + 255) & ~size_t(255);
  if (2 * arr > kStaticScratchBytes) return BAND_ERR_WORKSPACE;   // batch too large
  if (desc->nsys == 0) return BAND_OK;
  if (!diag || !f || !x || !diag[1] || !diag[2] || !diag[3]) return BAND_ERR_ARG;
  if (may_be_pd(desc) && kmode != 1 && (!diag[0] || !diag[4])) return BAND_ERR_ARG;
  void* base = nullptr;
  if (scratch_on_current_device(&base) != cudaSuccess) return BAND_ERR_CUDA;
  char* al = static_cast<char*>(base);
  char* be = al + arr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Layout L = layout_of(desc);
  const Spill W = spill_of(desc);
  if (desc->dtype == BAND_F64) {
    DirectArgs<double> p{L, W,
                         (const double*)diag[0], (const double*)diag[1], (const double*)diag[2],
                         (const double*)diag[3], (const double*)diag[4], (const double*)f,
                         (double*)x, (double*)al, (double*)be, nullptr, sys_status, nullptr,
                         nullptr};
    return cuda_status(launch_direct<double>(p, kmode, st));
  }
  DirectArgs<float> p{L, W,
                      (const float*)diag[0], (const float*)diag[1], (const float*)diag[2],
                      (const float*)diag[3], (const float*)diag[4], (const float*)f, (float*)x,
                      (float*)al, (float*)be, nullptr, sys_status, nullptr, nullptr};
  return cuda_status(launch_direct<float>(p, kmode, st));
}
