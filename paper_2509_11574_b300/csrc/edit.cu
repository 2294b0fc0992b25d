// Gaussian insertion and removal (Sec. 3.2 "Gaussian reconstruction", App. A).
//
// Insertion: one pass over the pixels decides the mask (hit, colour error,
// Gaussian weight) and the 25 % draw (SplitMix64, one output per pixel); a
// scan over blocks gives every sampled pixel its slot, so new Gaussians are
// appended in pixel order; a second pass over the pixels builds each new
// Gaussian (the window search for the disc radius reads the mask of the
// first pass).  Removal: a flag pass over the Gaussians, the same scan, then
// a stable gather into scratch and a copy back, one parameter group at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "gps_common.cuh"
#include "sh.cuh"

namespace gps {

constexpr int kEditThreads = 256;

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long n) {
  unsigned long long z = seed + n * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct InsertArgs {
  GpsGaussians g, m, v, gr;  // m, v, gr arrays may be null
  int M, capacity, W, H, radius;
  float fx, cam[3];          // camera centre (world)
  const float* vertex;       // [H][W][3]
  const float* depth;        // D_t
  const void* rendered;      // C* (element type per prec)
  const float* weight;       // W_G
  const void* target;        // C_k
  int prec;
  float err3;                // float(3 delta_c)
  float delta_w;
  unsigned long long seed, keep_below;  // draw kept when (z >> 40) < keep_below
  uint8_t* mask;
  uint8_t* flag;
  uint32_t* block_counts;
  uint32_t* block_offsets;
  int32_t* count;
};

__global__ void __launch_bounds__(kEditThreads) insert_flag_kernel(InsertArgs a) {
  const long long npx = (long long)a.W * a.H;
  const long long p = (long long)blockIdx.x * kEditThreads + threadIdx.x;
  bool mk = false, fl = false;
  if (p < npx) {
    if (a.depth[p] > 0.0f) {
      const float e0 = fabsf(ld_col(a.rendered, p, a.prec) - ld_col(a.target, p, a.prec));
      const float e1 = fabsf(ld_col(a.rendered, npx + p, a.prec) - ld_col(a.target, npx + p, a.prec));
      const float e2 = fabsf(ld_col(a.rendered, 2 * npx + p, a.prec) - ld_col(a.target, 2 * npx + p, a.prec));
      const float e = __fadd_rn(__fadd_rn(e0, e1), e2);
      mk = e > a.err3 && a.weight[p] < a.delta_w;
    }
    fl = mk && (splitmix64_at(a.seed, (unsigned long long)p + 1ull) >> 40) < a.keep_below;
    a.mask[p] = mk;
    a.flag[p] = fl;
  }
  const int c = __syncthreads_count(fl);
  if (threadIdx.x == 0) a.block_counts[blockIdx.x] = (uint32_t)c;
}

// Exclusive scan of n block counts (one block of 1024 threads); writes
// base + total (clipped to limit) to *count.
__global__ void __launch_bounds__(1024) edit_scan_kernel(const uint32_t* counts, uint32_t* offsets,
                                                         int n, int base, int limit,
                                                         int32_t* count) {
  __shared__ uint32_t warp_sums[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + 1023) / 1024;
  const int b = tid * per, e = min(n, b + per);
  uint32_t local = 0;
  for (int k = b; k < e; ++k) local += counts[k];
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    warp_sums[lane] = w;
  }
  __syncthreads();
  uint32_t run = incl - local + (warp > 0 ? warp_sums[warp - 1] : 0u);
  for (int k = b; k < e; ++k) {
    offsets[k] = run;
    run += counts[k];
  }
  if (tid == 1023) *count = (int32_t)min((long long)base + run, (long long)limit);
}

// Rank of this thread's flag among the block's set flags (thread order).
__device__ __forceinline__ uint32_t block_rank(bool f, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if (lane == 0) s_warp[warp] = __popc(bal);
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += s_warp[w];
  return before + __popc(bal & ((1u << lane) - 1u));
}

__device__ __forceinline__ bool hit_at(const InsertArgs& a, int y, int x) {
  return y >= 0 && y < a.H && x >= 0 && x < a.W && a.depth[(long long)y * a.W + x] > 0.0f;
}

__device__ __forceinline__ float3 vtx(const InsertArgs& a, int y, int x) {
  const float* p = a.vertex + 3 * ((long long)y * a.W + x);
  return make_float3(p[0], p[1], p[2]);
}

// Difference of the vertex map along one axis at (y, x): central where both
// neighbours are hits, else one-sided; false if neither is.
__device__ __forceinline__ bool axis_diff(const InsertArgs& a, int y, int x, int dy, int dx,
                                          float3& d) {
  const bool ok0 = hit_at(a, y - dy, x - dx), ok1 = hit_at(a, y + dy, x + dx);
  if (!ok0 && !ok1) return false;
  const float3 p0 = ok0 ? vtx(a, y - dy, x - dx) : vtx(a, y, x);
  const float3 p1 = ok1 ? vtx(a, y + dy, x + dx) : vtx(a, y, x);
  d = make_float3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z);
  return true;
}

__global__ void __launch_bounds__(kEditThreads) insert_emit_kernel(InsertArgs a) {
  __shared__ uint32_t s_warp[kEditThreads / 32];
  const long long npx = (long long)a.W * a.H;
  const long long p = (long long)blockIdx.x * kEditThreads + threadIdx.x;
  const bool f = p < npx && a.flag[p];
  const uint32_t rank = block_rank(f, s_warp);
  if (!f) return;
  const long long slot = (long long)a.M + a.block_offsets[blockIdx.x] + rank;
  if (slot >= a.capacity) return;
  const int y = (int)(p / a.W), x = (int)(p % a.W);
  const float3 c = vtx(a, y, x);
  // the three mask pixels of the window whose vertices are nearest (ties: scan order)
  float best[3] = {INFINITY, INFINITY, INFINITY};
  int found = 0;
  for (int yy = max(0, y - a.radius); yy <= min(a.H - 1, y + a.radius); ++yy)
    for (int xx = max(0, x - a.radius); xx <= min(a.W - 1, x + a.radius); ++xx) {
      if ((yy == y && xx == x) || !a.mask[(long long)yy * a.W + xx]) continue;
      const float3 q = vtx(a, yy, xx);
      const float dx = q.x - c.x, dy = q.y - c.y, dz = q.z - c.z;
      const float d2 = dx * dx + dy * dy + dz * dz;
      ++found;
      if (d2 < best[2]) {
        if (d2 < best[1]) {
          best[2] = best[1];
          if (d2 < best[0]) {
            best[1] = best[0];
            best[0] = d2;
          } else {
            best[1] = d2;
          }
        } else {
          best[2] = d2;
        }
      }
    }
  float s1;
  if (found == 0) {
    s1 = fminf(0.1f, a.depth[p] / a.fx);
  } else {
    const int k = min(found, 3);
    float sum = 0.f;
    for (int i = 0; i < k; ++i) sum += best[i];
    s1 = fminf(0.1f, sqrtf(sum / (float)k));
  }
  // surface normal from the vertex map, facing the camera
  const float3 ray = make_float3(c.x - a.cam[0], c.y - a.cam[1], c.z - a.cam[2]);
  float3 gx, gy, n;
  if (axis_diff(a, y, x, 0, 1, gx) && axis_diff(a, y, x, 1, 0, gy)) {
    n = make_float3(gx.y * gy.z - gx.z * gy.y, gx.z * gy.x - gx.x * gy.z, gx.x * gy.y - gx.y * gy.x);
  } else {
    n = make_float3(-ray.x, -ray.y, -ray.z);
  }
  float nn = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
  if (!(nn > 0.0f)) {
    n = make_float3(-ray.x, -ray.y, -ray.z);
    nn = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
  }
  n = make_float3(n.x / nn, n.y / nn, n.z / nn);
  if (n.x * ray.x + n.y * ray.y + n.z * ray.z > 0.0f) n = make_float3(-n.x, -n.y, -n.z);
  // quaternion (w, x, y, z) taking the disc's short axis (local z) onto the
  // line of n; the disc is the same for -n, so n_z >= 0 keeps w = 1 + n_z >= 1
  if (n.z < 0.0f) n = make_float3(-n.x, -n.y, -n.z);
  const float w = 1.0f + n.z;
  const float qn = sqrtf(w * w + n.y * n.y + n.x * n.x);
  const float4 qt = make_float4(w / qn, -n.y / qn, n.x / qn, 0.f);
  const float ls = logf(s1);
  float* mean = a.g.means + 3 * slot;
  mean[0] = c.x;
  mean[1] = c.y;
  mean[2] = c.z;
  float* lsc = a.g.log_scales + 3 * slot;
  lsc[0] = ls;
  lsc[1] = ls;
  lsc[2] = logf(0.1f * s1);
  reinterpret_cast<float4*>(a.g.quats)[slot] = qt;
  a.g.opacity_logits[slot] = 0.0f;  // sigma = 0.5
  float* col = a.g.rgb + 3 * slot;
  col[0] = ld_col(a.target, p, a.prec);
  col[1] = ld_col(a.target, npx + p, a.prec);
  col[2] = ld_col(a.target, 2 * npx + p, a.prec);
  // no view dependence yet: SH coefficients of degree >= 1 start at zero
  const int nsh = a.g.sh_degree > 0 ? 3 * sh_coeffs(a.g.sh_degree) : 0;
  for (int c = 0; c < nsh; ++c) a.g.sh_rest[nsh * slot + c] = 0.f;
  const GpsGaussians* zs[3] = {&a.m, &a.v, &a.gr};
  for (int k = 0; k < 3; ++k) {
    const GpsGaussians& z = *zs[k];
    if (!z.means) continue;
    for (int c3 = 0; c3 < 3; ++c3) {
      z.means[3 * slot + c3] = 0.f;
      z.log_scales[3 * slot + c3] = 0.f;
      z.rgb[3 * slot + c3] = 0.f;
    }
    reinterpret_cast<float4*>(z.quats)[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    z.opacity_logits[slot] = 0.f;
    for (int c = 0; c < nsh; ++c) z.sh_rest[nsh * slot + c] = 0.f;
  }
}

cudaError_t launch_insert(const InsertArgs& a, cudaStream_t st) {
  const long long npx = (long long)a.W * a.H;
  const int nblk = (int)((npx + kEditThreads - 1) / kEditThreads);
  insert_flag_kernel<<<nblk, kEditThreads, 0, st>>>(a);
  edit_scan_kernel<<<1, 1024, 0, st>>>(a.block_counts, a.block_offsets, nblk, a.M, a.capacity,
                                       a.count);
  insert_emit_kernel<<<nblk, kEditThreads, 0, st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ removal
struct RemoveArgs {
  GpsGaussians g, m, v, gr;  // m, v, gr may be null
  int M;
  float t_logit, t_smax, t_smin;  // float constants ln(ds / (1 - ds)), ln(smax), ln(smin)
  uint8_t* keep;
  uint32_t* block_counts;
  uint32_t* block_offsets;
  float* scratch;  // [M][14]
  int32_t* count;
};

__global__ void __launch_bounds__(kEditThreads) remove_flag_kernel(RemoveArgs a) {
  const int i = blockIdx.x * kEditThreads + threadIdx.x;
  bool k = false;
  if (i < a.M) {
    const float* ls = a.g.log_scales + 3 * (size_t)i;
    const float mx = fmaxf(fmaxf(ls[0], ls[1]), ls[2]);
    k = !(a.g.opacity_logits[i] < a.t_logit || mx > a.t_smax || mx < a.t_smin);
    a.keep[i] = k;
  }
  const int c = __syncthreads_count(k);
  if (threadIdx.x == 0) a.block_counts[blockIdx.x] = (uint32_t)c;
}

// Row i of a parameter group as 14 floats: mean 3, log-scale 3, quat 4, logit, rgb 3.
__device__ __forceinline__ void load_row(const GpsGaussians& z, size_t i, float* r) {
  for (int c = 0; c < 3; ++c) r[c] = z.means[3 * i + c];
  for (int c = 0; c < 3; ++c) r[3 + c] = z.log_scales[3 * i + c];
  const float4 q = reinterpret_cast<const float4*>(z.quats)[i];
  r[6] = q.x; r[7] = q.y; r[8] = q.z; r[9] = q.w;
  r[10] = z.opacity_logits[i];
  for (int c = 0; c < 3; ++c) r[11 + c] = z.rgb[3 * i + c];
}
__device__ __forceinline__ void store_row(const GpsGaussians& z, size_t i, const float* r) {
  for (int c = 0; c < 3; ++c) z.means[3 * i + c] = r[c];
  for (int c = 0; c < 3; ++c) z.log_scales[3 * i + c] = r[3 + c];
  reinterpret_cast<float4*>(z.quats)[i] = make_float4(r[6], r[7], r[8], r[9]);
  z.opacity_logits[i] = r[10];
  for (int c = 0; c < 3; ++c) z.rgb[3 * i + c] = r[11 + c];
}

__global__ void __launch_bounds__(kEditThreads) remove_gather_kernel(RemoveArgs a, GpsGaussians z) {
  __shared__ uint32_t s_warp[kEditThreads / 32];
  const int i = blockIdx.x * kEditThreads + threadIdx.x;
  const bool k = i < a.M && a.keep[i];
  const uint32_t rank = block_rank(k, s_warp);
  if (!k) return;
  float r[14];
  load_row(z, (size_t)i, r);
  float* d = a.scratch + 14 * (size_t)(a.block_offsets[blockIdx.x] + rank);
  for (int c = 0; c < 14; ++c) d[c] = r[c];
}

// Rows [0, kept) from scratch; rows [kept, M) zeroed when `clear`.
__global__ void __launch_bounds__(kEditThreads) remove_scatter_kernel(RemoveArgs a, GpsGaussians z,
                                                                     int clear) {
  const int i = blockIdx.x * kEditThreads + threadIdx.x;
  if (i >= a.M) return;
  const int kept = *a.count;
  float r[14];
  if (i < kept) {
    const float* s = a.scratch + 14 * (size_t)i;
    for (int c = 0; c < 14; ++c) r[c] = s[c];
  } else if (clear) {
    for (int c = 0; c < 14; ++c) r[c] = 0.f;
  } else {
    return;
  }
  store_row(z, (size_t)i, r);
}

// The SH coefficient rows (3K floats) move through the same [M][14] scratch,
// 14 columns [c0, c0 + w) at a time.
__global__ void __launch_bounds__(kEditThreads) remove_gather_cols_kernel(RemoveArgs a,
                                                                         const float* src,
                                                                         int stride, int c0,
                                                                         int w) {
  __shared__ uint32_t s_warp[kEditThreads / 32];
  const int i = blockIdx.x * kEditThreads + threadIdx.x;
  const bool k = i < a.M && a.keep[i];
  const uint32_t rank = block_rank(k, s_warp);
  if (!k) return;
  float* d = a.scratch + 14 * (size_t)(a.block_offsets[blockIdx.x] + rank);
  for (int c = 0; c < w; ++c) d[c] = src[(size_t)i * stride + c0 + c];
}

__global__ void __launch_bounds__(kEditThreads) remove_scatter_cols_kernel(RemoveArgs a,
                                                                          float* dst, int stride,
                                                                          int c0, int w,
                                                                          int clear) {
  const int i = blockIdx.x * kEditThreads + threadIdx.x;
  if (i >= a.M) return;
  const int kept = *a.count;
  if (i < kept) {
    const float* s = a.scratch + 14 * (size_t)i;
    for (int c = 0; c < w; ++c) dst[(size_t)i * stride + c0 + c] = s[c];
  } else if (clear) {
    for (int c = 0; c < w; ++c) dst[(size_t)i * stride + c0 + c] = 0.f;
  }
}

cudaError_t launch_remove(const RemoveArgs& a, cudaStream_t st) {
  if (a.M <= 0) return cudaMemsetAsync(a.count, 0, sizeof(int32_t), st);
  const int nblk = (a.M + kEditThreads - 1) / kEditThreads;
  remove_flag_kernel<<<nblk, kEditThreads, 0, st>>>(a);
  edit_scan_kernel<<<1, 1024, 0, st>>>(a.block_counts, a.block_offsets, nblk, 0, a.M, a.count);
  const GpsGaussians* groups[4] = {&a.g, &a.m, &a.v, &a.gr};
  const int nsh = a.g.sh_degree > 0 ? 3 * sh_coeffs(a.g.sh_degree) : 0;
  for (int k = 0; k < 4; ++k) {
    if (!groups[k]->means) continue;
    remove_gather_kernel<<<nblk, kEditThreads, 0, st>>>(a, *groups[k]);
    remove_scatter_kernel<<<nblk, kEditThreads, 0, st>>>(a, *groups[k], k > 0 ? 1 : 0);
    for (int c0 = 0; c0 < nsh; c0 += 14) {
      const int w = nsh - c0 < 14 ? nsh - c0 : 14;
      remove_gather_cols_kernel<<<nblk, kEditThreads, 0, st>>>(a, groups[k]->sh_rest, nsh, c0, w);
      remove_scatter_cols_kernel<<<nblk, kEditThreads, 0, st>>>(a, groups[k]->sh_rest, nsh, c0,
                                                                w, k > 0 ? 1 : 0);
    }
  }
  return cudaGetLastError();
}

}  // namespace gps

// ------------------------------------------------------------------ C ABI
namespace gps {
void set_error(const char* msg);  // capi.cu: sets gps_last_error() of this thread
}

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct EditScratch {
  size_t mask, flag, keep, counts, offsets, rows, total;
};

EditScratch edit_scratch(long long capacity, long long npx) {
  EditScratch s{};
  const long long nb = (std::max(npx, capacity) + gps::kEditThreads - 1) / gps::kEditThreads;
  size_t off = 0;
  s.mask = off; off = a256(off + (size_t)npx);
  s.flag = off; off = a256(off + (size_t)npx);
  s.keep = off; off = a256(off + (size_t)capacity);
  s.counts = off; off = a256(off + (size_t)nb * 4);
  s.offsets = off; off = a256(off + (size_t)nb * 4);
  s.rows = off; off = a256(off + (size_t)capacity * 14 * 4);
  s.total = off;
  return s;
}

int32_t edit_fail(int32_t code, const char* msg) {
  gps::set_error(msg);
  return code;
}

bool complete(const GpsGaussians* z) {
  return z && z->means && z->log_scales && z->quats && z->opacity_logits && z->rgb &&
         (reinterpret_cast<uintptr_t>(z->quats) & 15) == 0 && z->sh_degree >= 0 &&
         z->sh_degree <= 3 && (z->sh_degree == 0 || z->sh_rest);
}

GpsGaussians or_null(const GpsGaussians* z) {
  GpsGaussians n{};
  return z ? *z : n;
}

}  // namespace

extern "C" {

int32_t gps_edit_scratch_size(int32_t capacity, int32_t width, int32_t height, size_t* bytes) {
  if (capacity < 0 || width < 0 || height < 0 || !bytes)
    return edit_fail(GPS_ERR_INVALID_ARG, "gps_edit_scratch_size: bad arguments");
  *bytes = edit_scratch(capacity, (long long)width * height).total;
  return GPS_OK;
}

int32_t insert_gaussians(GpsGaussians* gaussians, int32_t capacity, GpsGaussians* m,
                         GpsGaussians* v, GpsGaussians* grads, const GpsIntrinsics* K,
                         const GpsPose* T_wc, const float* vertex, const float* sdf_depth,
                         const void* rendered_rgb, const float* weight, const void* target_rgb,
                         const GpsEditSettings* s, void* scratch, size_t scratch_bytes,
                         int32_t* count, void* stream) {
  if (!complete(gaussians) || !K || !T_wc || !vertex || !sdf_depth || !rendered_rgb || !weight ||
      !target_rgb || !s || !scratch || !count)
    return edit_fail(GPS_ERR_INVALID_ARG, "insert_gaussians: NULL argument or Gaussian array");
  for (const GpsGaussians* z : {m, v, grads})
    if (z && (!complete(z) || z->sh_degree != gaussians->sh_degree))
      return edit_fail(GPS_ERR_INVALID_ARG,
                       "insert_gaussians: incomplete moment / gradient set or another SH degree");
  if (gaussians->M < 0 || capacity < gaussians->M || K->width <= 0 || K->height <= 0 ||
      !(K->fx > 0) || s->radius < 0 || s->radius > 16 || !(s->sample_fraction >= 0) ||
      !(s->sample_fraction <= 1) || !(s->delta_c >= 0) || !(s->delta_w > 0) ||
      (s->precision != GPS_PREC_FP32 && s->precision != GPS_PREC_FP16 &&
       s->precision != GPS_PREC_BF16))
    return edit_fail(GPS_ERR_INVALID_ARG, "insert_gaussians: bad sizes or settings");
  const long long npx = (long long)K->width * K->height;
  const EditScratch L = edit_scratch(capacity, npx);
  if (scratch_bytes < L.total || (reinterpret_cast<uintptr_t>(scratch) & 255))
    return edit_fail(GPS_ERR_WORKSPACE_TOO_SMALL,
                     "insert_gaussians: scratch smaller than gps_edit_scratch_size or unaligned");
  char* b = static_cast<char*>(scratch);
  gps::InsertArgs a{};
  a.g = *gaussians;
  a.m = or_null(m);
  a.v = or_null(v);
  a.gr = or_null(grads);
  a.M = gaussians->M;
  a.capacity = capacity;
  a.W = K->width;
  a.H = K->height;
  a.radius = s->radius;
  a.fx = K->fx;
  for (int k = 0; k < 3; ++k) a.cam[k] = T_wc->t[k];
  a.vertex = vertex;
  a.depth = sdf_depth;
  a.rendered = rendered_rgb;
  a.weight = weight;
  a.target = target_rgb;
  a.prec = s->precision;
  a.err3 = (float)(3.0 * (double)s->delta_c);
  a.delta_w = s->delta_w;
  a.seed = s->seed;
  a.keep_below = (unsigned long long)((double)s->sample_fraction * 16777216.0);
  a.mask = reinterpret_cast<uint8_t*>(b + L.mask);
  a.flag = reinterpret_cast<uint8_t*>(b + L.flag);
  a.block_counts = reinterpret_cast<uint32_t*>(b + L.counts);
  a.block_offsets = reinterpret_cast<uint32_t*>(b + L.offsets);
  a.count = count;
  const cudaError_t e = gps::launch_insert(a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return edit_fail(GPS_ERR_CUDA, cudaGetErrorString(e));
  return GPS_OK;
}

int32_t remove_gaussians(GpsGaussians* gaussians, GpsGaussians* m, GpsGaussians* v,
                         GpsGaussians* grads, const GpsEditSettings* s, void* scratch,
                         size_t scratch_bytes, int32_t* count, void* stream) {
  if (!complete(gaussians) || !s || !scratch || !count || gaussians->M < 0)
    return edit_fail(GPS_ERR_INVALID_ARG, "remove_gaussians: NULL argument or Gaussian array");
  for (const GpsGaussians* z : {m, v, grads})
    if (z && (!complete(z) || z->M != gaussians->M || z->sh_degree != gaussians->sh_degree))
      return edit_fail(GPS_ERR_INVALID_ARG, "remove_gaussians: moment / gradient set mismatch");
  if (!(s->delta_sigma > 0 && s->delta_sigma < 1) || !(s->delta_smax > 0) || !(s->delta_smin > 0))
    return edit_fail(GPS_ERR_INVALID_ARG, "remove_gaussians: bad thresholds");
  const EditScratch L = edit_scratch(gaussians->M, 0);
  if (scratch_bytes < L.total || (reinterpret_cast<uintptr_t>(scratch) & 255))
    return edit_fail(GPS_ERR_WORKSPACE_TOO_SMALL,
                     "remove_gaussians: scratch smaller than gps_edit_scratch_size or unaligned");
  char* b = static_cast<char*>(scratch);
  gps::RemoveArgs a{};
  a.g = *gaussians;
  a.m = or_null(m);
  a.v = or_null(v);
  a.gr = or_null(grads);
  a.M = gaussians->M;
  const double ds = s->delta_sigma;
  a.t_logit = (float)std::log(ds / (1.0 - ds));
  a.t_smax = (float)std::log((double)s->delta_smax);
  a.t_smin = (float)std::log((double)s->delta_smin);
  a.keep = reinterpret_cast<uint8_t*>(b + L.keep);
  a.block_counts = reinterpret_cast<uint32_t*>(b + L.counts);
  a.block_offsets = reinterpret_cast<uint32_t*>(b + L.offsets);
  a.scratch = reinterpret_cast<float*>(b + L.rows);
  a.count = count;
  const cudaError_t e = gps::launch_remove(a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return edit_fail(GPS_ERR_CUDA, cudaGetErrorString(e));
  return GPS_OK;
}

}  // extern "C"
