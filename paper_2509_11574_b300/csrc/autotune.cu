// gps_autotune_tiles: picks the tile shape (and with it the CTA shape of the
// binning split and both composite kernels: one thread per tile pixel) by
// timing render_forward + render_backward on the caller's own data.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "gps_common.cuh"

namespace gps {
void set_error(const char* msg);  // capi.cu: sets gps_last_error() of this thread
}

namespace {

struct Shape {
  int tw, th;
};
constexpr Shape kShapes[GPS_AUTOTUNE_SHAPES] = {{16, 16}, {16, 8}, {8, 8}, {32, 8}};
constexpr int kMaxRepeats = 64;  // timed rounds kept per shape

int32_t cuda_error(cudaError_t e, const char* where) {
  char buf[200];
  snprintf(buf, sizeof(buf), "gps_autotune_tiles: %s: %s", where, cudaGetErrorString(e));
  gps::set_error(buf);
  return GPS_ERR_CUDA;
}

}  // namespace

extern "C" int32_t gps_autotune_tiles(const GpsGaussians* g, const GpsView* views, int32_t n_views,
                                      const GpsRenderSettings* settings, void* ws, size_t ws_bytes,
                                      GpsGaussians* scratch_grads, int32_t repeats,
                                      int32_t* best_tile_w, int32_t* best_tile_h, float* times_ms,
                                      void* stream) {
  if (!g || !views || n_views <= 0 || !settings || !ws || !scratch_grads || !best_tile_w ||
      !best_tile_h || repeats <= 0) {
    gps::set_error("gps_autotune_tiles: NULL argument, no views or repeats <= 0");
    return GPS_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_error(ce, "cudaEventCreate");
  }
  int32_t rc = GPS_OK;
  // every candidate runs once untimed (and must leave status GPS_OK); then
  // the shapes are timed in interleaved rounds, so that drifting clocks or a
  // neighbour's load hit all of them alike, and each keeps its median
  const int reps = repeats < kMaxRepeats ? repeats : kMaxRepeats;
  bool cand[GPS_AUTOTUNE_SHAPES];
  float samples[GPS_AUTOTUNE_SHAPES][kMaxRepeats];
  GpsRenderSettings sk[GPS_AUTOTUNE_SHAPES];
  for (int k = 0; k < GPS_AUTOTUNE_SHAPES && rc == GPS_OK; ++k) {
    cand[k] = false;
    if (times_ms) times_ms[k] = -1.0f;
    sk[k] = *settings;
    sk[k].tile_w = kShapes[k].tw;
    sk[k].tile_h = kShapes[k].th;
    sk[k].stages = 0;
    sk[k].instrument = 0;
    size_t need = 0;
    if ((rc = gps_workspace_size(g->M, views, n_views, &sk[k], &need)) != GPS_OK) break;
    if (need > ws_bytes) continue;  // this shape's workspace does not fit: not a candidate
    rc = render_forward(g, views, n_views, &sk[k], ws, ws_bytes, nullptr, stream);
    if (rc == GPS_OK)
      rc = render_backward(g, views, n_views, &sk[k], ws, ws_bytes, nullptr, scratch_grads, stream);
    int32_t status = GPS_OK;
    if (rc == GPS_OK) rc = gps_query_status(ws, ws_bytes, &status, stream);
    cand[k] = rc == GPS_OK && status == GPS_OK;  // e.g. pair capacity exceeded with this shape
  }
  for (int r = 0; r < reps && rc == GPS_OK; ++r) {
    for (int k = 0; k < GPS_AUTOTUNE_SHAPES && rc == GPS_OK; ++k) {
      if (!cand[k]) continue;
      if ((ce = cudaEventRecord(e0, st)) != cudaSuccess) rc = cuda_error(ce, "record");
      if (rc == GPS_OK) rc = render_forward(g, views, n_views, &sk[k], ws, ws_bytes, nullptr, stream);
      if (rc == GPS_OK)
        rc = render_backward(g, views, n_views, &sk[k], ws, ws_bytes, nullptr, scratch_grads, stream);
      if (rc != GPS_OK) break;
      if ((ce = cudaEventRecord(e1, st)) != cudaSuccess) rc = cuda_error(ce, "record");
      else if ((ce = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_error(ce, "synchronize");
      float ms = 0.0f;
      if (rc == GPS_OK && (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
        rc = cuda_error(ce, "elapsed time");
      samples[k][r] = ms;
    }
  }
  float best = INFINITY;
  int best_k = -1;
  for (int k = 0; k < GPS_AUTOTUNE_SHAPES && rc == GPS_OK; ++k) {
    if (!cand[k]) continue;
    std::sort(samples[k], samples[k] + reps);
    const float med = reps % 2 ? samples[k][reps / 2]
                               : 0.5f * (samples[k][reps / 2 - 1] + samples[k][reps / 2]);
    if (times_ms) times_ms[k] = med;
    if (med < best) {
      best = med;
      best_k = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GPS_OK) return rc;
  if (best_k < 0) {
    gps::set_error("gps_autotune_tiles: no tile shape fits the workspace and the pair capacity");
    return GPS_ERR_WORKSPACE_TOO_SMALL;
  }
  *best_tile_w = kShapes[best_k].tw;
  *best_tile_h = kShapes[best_k].th;
  return GPS_OK;
}
