// fwi_forward_noalloc: forward modelling without any device allocation.
//
// Some callers cannot call cudaMalloc: a service that reserves all of its
// device memory at start-up and must not allocate (or risk an out-of-memory
// failure) while serving, a plugin running inside a host application whose
// allocator owns the device, or code that must not trigger the implicit
// synchronisation a cudaMalloc/cudaFree can cause.  For them this entry point
// runs the same forward solver as fwi_forward, but its workspace (wavefields,
// model fields, interpolation tables, counters) lives in one file-scope
// __device__ array of FWI_NOALLOC_SCRATCH_BYTES.  The caller still passes the
// inputs and the output array.
//
// The array exists once per device that loads this library and stays
// allocated until the process exits.  Its host-side name is only a stand-in:
// host code must use the device address returned by cudaGetSymbolAddress,
// which is looked up once per device, with that device current, on the first
// call made on it (so make the first call before any stream capture).  Every
// call reuses the same array: calls that overlap on the GPU (different
// streams, threads or processes sharing a context) race on it.  Each call
// clears what must start at zero before use.
#include "fwi.h"

#include <cuda_runtime.h>

#include <mutex>
#include <string>

namespace fwi {
void set_last_error(const std::string& msg);
fwi_status forward_in_buffer(const fwi_grid* grid, int nt, double dt, const fwi_model* model,
                             const fwi_geometry* geom, const float* wavelet, float* traces,
                             void* stream, char* base, size_t bytes, int device);
}

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FWI_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" fwi_status fwi_forward_noalloc(const fwi_grid* grid, int nt, double dt,
                                          const fwi_model* model, const fwi_geometry* geom,
                                          const float* wavelet, float* traces, void* stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    fwi::set_last_error("fwi_forward_noalloc: no usable CUDA device");
    return FWI_ERR_CUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        fwi::set_last_error(std::string("fwi_forward_noalloc: cudaGetSymbolAddress failed: ") +
                            cudaGetErrorString(e));
        return FWI_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  return fwi::forward_in_buffer(grid, nt, dt, model, geom, wavelet, traces, stream,
                                static_cast<char*>(base), (size_t)FWI_NOALLOC_SCRATCH_BYTES, dev);
}
