// render_forward_noalloc: render_forward on a workspace that lives in a static
// device array of this library, for callers that may not allocate device
// memory themselves (see the declaration in gps.h).
//
// In host code `g_scratch` names a host-side shadow symbol, not a device
// address: its device address is obtained once per device, with that device
// current, through cudaGetSymbolAddress and cached here.  The array's first
// 256 bytes hold the workspace status word, which gps_noalloc_query_status
// reads back (the caller never sees the array's address).
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "gps_common.cuh"

namespace gps {
void set_error(const char* msg);  // capi.cu: sets gps_last_error() of this thread
}

namespace {

static __device__ __align__(256) unsigned char g_scratch[GPS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Device address of g_scratch on the current device (set-up on first use).
int32_t scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    char buf[160];
    snprintf(buf, sizeof(buf), "render_forward_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    gps::set_error(buf);
    return GPS_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    gps::set_error("render_forward_noalloc: device ordinal beyond the 64 supported");
    return GPS_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      char buf[160];
      snprintf(buf, sizeof(buf), "render_forward_noalloc: cudaGetSymbolAddress: %s",
               cudaGetErrorString(e));
      gps::set_error(buf);
      return GPS_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GPS_OK;
}

}  // namespace

extern "C" int32_t render_forward_noalloc(const GpsGaussians* gaussians, const GpsView* views,
                                          int32_t n_views, const GpsRenderSettings* settings,
                                          float* loss, void* stream) {
  if (!gaussians || !views || !settings || n_views <= 0) {
    gps::set_error("render_forward_noalloc: NULL argument or no views");
    return GPS_ERR_INVALID_ARG;
  }
  // every stage runs: nothing is read from a previous call's contents
  GpsRenderSettings s = *settings;
  s.stages = 0;
  size_t need = 0;
  if (int32_t rc = gps_workspace_size(gaussians->M, views, n_views, &s, &need)) return rc;
  if (need > (size_t)GPS_NOALLOC_SCRATCH_BYTES) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "render_forward_noalloc: this problem needs a %zu-byte workspace; the static "
             "scratch holds %zu bytes (use render_forward with a caller-allocated workspace)",
             need, (size_t)GPS_NOALLOC_SCRATCH_BYTES);
    gps::set_error(buf);
    return GPS_ERR_WORKSPACE_TOO_SMALL;
  }
  void* ws = nullptr;
  if (int32_t rc = scratch_on_current_device(&ws)) return rc;
  return render_forward(gaussians, views, n_views, &s, ws, (size_t)GPS_NOALLOC_SCRATCH_BYTES,
                        loss, stream);
}

extern "C" int32_t gps_noalloc_query_status(int32_t* status, void* stream) {
  if (!status) {
    gps::set_error("gps_noalloc_query_status: NULL status");
    return GPS_ERR_INVALID_ARG;
  }
  void* ws = nullptr;
  if (int32_t rc = scratch_on_current_device(&ws)) return rc;
  return gps_query_status(ws, (size_t)GPS_NOALLOC_SCRATCH_BYTES, status, stream);
}
