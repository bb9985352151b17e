// rox_xsec_static: the one-(P,T) cross-section with its scratch in a fixed device array
// owned by the library, for callers that cannot allocate device memory themselves -- a
// host application whose memory manager owns all device memory, a plugin that may not call
// cudaMalloc, or an interface with no way to pass a workspace through. The caller still
// passes the line list and the output; nothing here allocates or frees.
#include <cstdio>
#include <mutex>
#include "rox_internal.cuh"

// Size of the static scratch: enough for ROX_STATIC_MAX_LINES lines on a grid of
// ROX_STATIC_MAX_GRID points at one (P,T) point (include/rox.h).
#define ROX_STATIC_BYTES (16u << 20)
#define ROX_STATIC_MAX_DEVICES 64

// Library-owned scratch. Every GPU that loads the library keeps this array until exit.
static __device__ __align__(256) unsigned char rox_static_scratch[ROX_STATIC_BYTES];

int rox_set_error(int code, const char* msg);   // rox_api.cu
// rox_xsec with the tail scratch (the split work items of the Voigt launch) limited to
// tail_max items, and its workspace size (rox_api.cu)
int rox_xsec_tail(const rox_lines* lines, const rox_grid* grid, double P_bar, double T, double Q_T, double Q_ref,
                  double mass_amu, double cutoff, float* sigma_out, void* ws, size_t ws_bytes, void* stream,
                  long long tail_max);
size_t rox_xsec_workspace_size_tail(int64_t n_lines, const rox_grid* grid, long long tail_max);

// Split work items the static scratch has room for (16 KB each); the launch splits fewer items
// than usual, which changes how its warps share the last items, not the result.
#define ROX_STATIC_TAIL_ITEMS 256

namespace {

std::mutex g_static_mu;
void* g_static_ptr[ROX_STATIC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device. In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device, with
// that device current, and cached. The cache outlives a cudaDeviceReset (which unloads the
// array): after a reset the process must be restarted before this entry point is used again.
int static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rox_set_error(ROX_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= ROX_STATIC_MAX_DEVICES) return rox_set_error(ROX_ERANGE, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, rox_static_scratch);
    if (e != cudaSuccess) return rox_set_error(ROX_ECUDA, cudaGetErrorString(e));
    if (!p) return rox_set_error(ROX_ECUDA, "cudaGetSymbolAddress returned NULL");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return ROX_OK;
}

}  // namespace

extern "C" int rox_xsec_static(const rox_lines* lines, const rox_grid* grid, double P_bar, double T, double Q_T,
                               double Q_ref, double mass_amu, double cutoff, float* sigma_out, int32_t* status_out,
                               void* stream) {
  if (!lines || !grid) return rox_set_error(ROX_EINVAL, "lines or grid is NULL");
  if (lines->n > ROX_STATIC_MAX_LINES || grid->n > ROX_STATIC_MAX_GRID) {
    char msg[200];
    snprintf(msg, sizeof msg, "rox_xsec_static: %lld lines, %lld grid points; the static scratch holds at most %d lines "
             "and %d grid points (use rox_xsec with a workspace)", (long long)lines->n, (long long)grid->n,
             ROX_STATIC_MAX_LINES, ROX_STATIC_MAX_GRID);
    return rox_set_error(ROX_ERANGE, msg);
  }
  if (rox_xsec_workspace_size_tail(lines->n, grid, ROX_STATIC_TAIL_ITEMS) > ROX_STATIC_BYTES)
    return rox_set_error(ROX_ERANGE, "rox_xsec_static: the problem does not fit the static scratch");
  void* ws = nullptr;
  int rc = static_scratch(&ws);
  if (rc) return rc;
  rc = rox_xsec_tail(lines, grid, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, sigma_out, ws, ROX_STATIC_BYTES, stream,
                     ROX_STATIC_TAIL_ITEMS);
  if (rc) return rc;
  if (status_out) {
    // device-side status of this call (ROX_OK, or ROX_EUNSORTED with sigma untouched)
    cudaError_t e = cudaMemcpyAsync(status_out, ws, sizeof(int32_t), cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return rox_set_error(ROX_ECUDA, cudaGetErrorString(e));
  }
  return ROX_OK;
}
