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
// call made on it.  The address is kept for the life of the process: after a cudaDeviceReset the
// entry point must not be used on that device again.  Every call reuses the
// same array: calls that overlap on the GPU (different streams, threads or
// processes sharing a context) race on it.  Each call clears what must start
// at zero before use, and returns only once its work on the scratch is
// finished (on success and on error).  All device arrays of a call must live
// on the current device; others are rejected.
#include "fwi_plan.cuh"

#include <cuda_runtime.h>

#include <mutex>
#include <string>

namespace fwi {

// Runs fwi_forward on a plan that lives on the stack and whose every device
// buffer is carved out of [base, base + bytes): no device allocation happens.
// Used by the fixed-scratch entry point (fwi_noalloc.cu).
fwi_status forward_in_buffer(const fwi_grid* grid, int nt, double dt, const fwi_model* model,
                             const fwi_geometry* geom, const float* wavelet, float* traces,
                             void* stream, char* base, size_t bytes, int device) {
  FWI_TRY(validate_grid(grid));
  if (nt < 1 || nt > (1 << 24)) return fail(FWI_ERR_INVALID_ARG, "nt must be in [1, 2^24]");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(FWI_ERR_INVALID_ARG, "dt must be positive");
  if (!traces) return fail(FWI_ERR_INVALID_ARG, "traces is NULL");
  if (!model || !model->vp) return fail(FWI_ERR_INVALID_ARG, "model or vp is NULL");
  fwi_plan P;
  P.grid = *grid;
  P.nt = nt;
  P.dt = dt;
  P.st = reinterpret_cast<cudaStream_t>(stream);
  P.device = device;
  P.c_ref = grid->c_ref;
  P.fixed_memory = true;
  if (cudaDeviceGetAttribute(&P.nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    P.nsm = 152;
  }
  build_layout(&P);
  FWI_TRY(validate_geometry(&P, geom));
  constexpr int JCAP = 4096;
  Carve C(base);
  P.d_stats = C.take<unsigned int>(16);
  P.d_flags = C.take<int>(16);
  P.d_J = C.take<double>(JCAP);
  P.d_J_cap = JCAP;
  P.spx = C.take<float>(P.L.nx_r + 8);
  P.spy = C.take<float>(P.L.ny_r + 8);
  P.spz = C.take<float>(std::max(P.L.nz, 1) + 8);
  Plan all;   // table bound for every shot in one batch, at the tile variant the call will use
  all.B = geom->nshots;
  if (!resolve_tile(&P, P.opt.tile, &all.tile, &all.shape, &all.tma, &all.x2))
    return fail(FWI_ERR_INVALID_ARG, "tile variant out of range");
  FWI_TRY(resolve_scheme(&P, model, &all.sc));
  const size_t tab = align_up(tables_bound(&P, geom, all) * 2, 256);
  P.tab = C.take<char>(tab);
  P.tab_cap = tab;
  C.off = align_up(C.off, 256);
  if (C.off >= bytes)
    return fail(FWI_ERR_BUDGET, "tables need " + std::to_string(C.off) +
                                    " bytes, more than the static scratch of " +
                                    std::to_string(bytes) + " bytes");
  P.arena = base + C.off;
  P.arena_cap = bytes - C.off;
  P.budget = P.arena_cap;
  Plan pl;
  if (choose_plan(&P, geom, model->rho != nullptr, false, pl, false, all.sc) != FWI_OK)
    return fail(FWI_ERR_BUDGET, "one shot of this grid needs more than the static scratch of " +
                                    std::to_string(bytes) + " bytes (use fwi_forward)");
  if ((geom->nshots + pl.B - 1) / pl.B > JCAP)
    return fail(FWI_ERR_BUDGET, "too many shot batches for the static scratch");
  if (P.c_ref > 0.0) FWI_TRY(build_sponge(&P));
  const fwi_status st = fwi_forward(&P, model, geom, wavelet, nt, dt, traces);
  if (st != FWI_OK) {
    // an error after work was enqueued: wait for it, so that no kernel of this
    // call still uses the shared scratch when the caller issues the next call
    cudaStreamSynchronize(P.st);
    cudaGetLastError();
  }
  return st;
}

// The device arrays of a call must live on the device the call runs on: the
// scratch is that device's, and a pointer to another device's memory would be
// read through the wrong address space.
fwi_status check_on_device(const void* ptr, const char* name, int dev) {
  if (!ptr) return FWI_OK;
  cudaPointerAttributes a{};
  const cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(FWI_ERR_INVALID_ARG, std::string("fwi_forward_noalloc: ") + name +
                                         " is not a CUDA pointer: " + cudaGetErrorString(e));
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(FWI_ERR_INVALID_ARG, std::string("fwi_forward_noalloc: ") + name +
                                         " is not device memory");
  if (a.device != dev)
    return fail(FWI_ERR_INVALID_ARG, std::string("fwi_forward_noalloc: ") + name + " lives on device " +
                                         std::to_string(a.device) + ", the call runs on device " +
                                         std::to_string(dev));
  return FWI_OK;
}

}  // namespace fwi


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
  if (!model || !model->vp || !wavelet || !traces) {
    fwi::set_last_error("fwi_forward_noalloc: model, vp, wavelet or traces is NULL");
    return FWI_ERR_INVALID_ARG;
  }
  for (const auto& a : {std::make_pair((const void*)model->vp, "vp"),
                        std::make_pair((const void*)model->rho, "rho"),
                        std::make_pair((const void*)wavelet, "wavelet"),
                        std::make_pair((const void*)traces, "traces")}) {
    const fwi_status s = fwi::check_on_device(a.first, a.second, dev);
    if (s != FWI_OK) return s;
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
