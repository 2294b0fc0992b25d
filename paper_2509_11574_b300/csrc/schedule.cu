// Keyframes and optimisation views of the online loop (Sec. 3.2 "Gaussian
// optimization", Fig. 5, App. C).  Host code only: the decisions are a few
// dozen flops per frame, so they stay on the CPU beside the caller's loop.
#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>

#include "../../include/gps.h"

namespace gps {
void set_error(const char* msg);  // capi.cu: sets gps_last_error() of this thread
}

namespace {

int32_t fail(const char* msg) {
  gps::set_error(msg);
  return GPS_ERR_INVALID_ARG;
}

// n-th output (n >= 1) of SplitMix64 seeded with `seed` (Steele, Lea and
// Flood 2014): state seed + n gamma, then the variant-13 finaliser.
uint64_t splitmix64_host(uint64_t seed, uint64_t n) {
  uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int32_t gps_is_keyframe(const GpsPose* last, const GpsPose* cur, const GpsViewSchedule* s,
                        int32_t* is_keyframe) {
  if (!cur || !s || !is_keyframe) return fail("gps_is_keyframe: NULL argument");
  if (!std::isfinite(s->delta_angle_deg) || !std::isfinite(s->delta_move))
    return fail("gps_is_keyframe: non-finite threshold");
  if (!last) {
    *is_keyframe = 1;
    return GPS_OK;
  }
  // trace(R_last^T R_cur) = sum of the element-wise products
  double tr = 0.0, d2 = 0.0;
  for (int i = 0; i < 9; ++i) tr += (double)last->R[i] * (double)cur->R[i];
  for (int i = 0; i < 3; ++i) {
    const double d = (double)cur->t[i] - (double)last->t[i];
    d2 += d * d;
  }
  // angle > delta  <=>  cos(angle) < cos(delta) on [0, pi]
  const double kPi = 3.14159265358979323846;
  const double cos_angle = (tr - 1.0) * 0.5;
  const double cos_delta = std::cos((double)s->delta_angle_deg * kPi / 180.0);
  const double move = (double)s->delta_move;
  *is_keyframe = (cos_angle < cos_delta || d2 > move * move) ? 1 : 0;
  return GPS_OK;
}

int32_t gps_select_views(const int32_t* keyframes, int32_t n_keyframes, int32_t frame,
                         int32_t event, const GpsViewSchedule* s, int32_t* views,
                         int32_t capacity, int32_t* n_views) {
  if (!s || !views || !n_views || (n_keyframes > 0 && !keyframes) || n_keyframes < 0)
    return fail("gps_select_views: NULL argument or negative keyframe count");
  if (frame < 0 || event < 0 || s->interval < 1 || s->n_local < 0 || s->n_global < 0 ||
      s->n_global > 1024)
    return fail("gps_select_views: frame, event, interval, n_local or n_global out of range");
  for (int32_t i = 0; i < n_keyframes; ++i)
    if (keyframes[i] < 0 || (i > 0 && keyframes[i] <= keyframes[i - 1]))
      return fail("gps_select_views: keyframe ids must be non-negative and strictly ascending");
  // history: the keyframes before the interval (ascending, so a prefix)
  const long long last_hist = (long long)frame - s->interval;
  int32_t H = 0;
  while (H < n_keyframes && keyframes[H] <= last_hist) ++H;
  const int32_t L = s->interval < frame + 1 ? s->interval : frame + 1;
  const int32_t nl = s->n_local < L ? s->n_local : L;
  const int32_t ng = s->n_global < H ? s->n_global : H;
  if (capacity < nl + ng) return fail("gps_select_views: capacity below the number of views");
  for (int32_t j = 0; j < nl; ++j)
    views[j] = frame - (int32_t)(((long long)j * L) / nl);
  // partial Fisher-Yates shuffle of a copy of the history
  std::vector<int32_t> hist(keyframes, keyframes + H);
  for (int32_t i = 0; i < ng; ++i) {
    const uint64_t r = splitmix64_host(s->seed, 1024ull * (uint64_t)event + (uint64_t)i + 1ull);
    const int32_t j = i + (int32_t)(((r >> 32) * (uint64_t)(H - i)) >> 32);
    std::swap(hist[i], hist[j]);
    views[nl + i] = hist[i];
  }
  *n_views = nl + ng;
  return GPS_OK;
}

}  // extern "C"
