// Camera tracking by point-to-plane ICP (Sec. 3.2 "Camera tracking", Eq. 5).
//
// Per frame: the depth pyramid (2x2 means), one vertex map and one normal map
// per level, the reference normals from the ray-cast vertex map, then one
// kernel per Gauss-Newton iteration.  That kernel associates every pixel of
// the level with the reference view, accumulates the 21 + 6 + 2 sums of the
// normal equations per thread, reduces them per block in a fixed order, and
// its last block (an atomic ticket; nothing waits) adds the block partials in
// a fixed order, solves the 6x6 system by Cholesky and updates the pose in
// device memory, all in single precision.  No host synchronisation: the whole track is one stream of
// launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <algorithm>
#include <cstdio>

#include "gps_common.cuh"

namespace gps {

constexpr int kIcpThreads = 256;
constexpr int kIcpSums = 29;   // A upper triangle (21), b (6), sum r^2, inliers
constexpr int kIcpMaxLevels = 4;

// level l + 1 = mean of the valid depths of each 2x2 block of level l
__global__ void icp_downsample_kernel(const float* __restrict__ src, int Ws, float* dst, int Wd,
                                      int Hd) {
  chain_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Wd * Hd) return;
  const int x = i % Wd, y = i / Wd;
  float s = 0.f;
  int n = 0;
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const float d = src[(size_t)(2 * y + dy) * Ws + 2 * x + dx];
      if (d > 0.f) {
        s += d;
        ++n;
      }
    }
  dst[i] = n > 0 ? s / (float)n : 0.f;
}

// camera-frame vertex map (x, y, z, valid)
__global__ void icp_vertex_kernel(const float* __restrict__ depth, int W, int H, float fx,
                                  float fy, float cx, float cy, float4* __restrict__ vert) {
  chain_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= W * H) return;
  const float z = depth[i];
  const int x = i % W, y = i / W;
  vert[i] = z > 0.f ? make_float4(((float)x - cx) / fx * z, ((float)y - cy) / fy * z, z, 1.f)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
}

// the reference's ray-cast vertex map ([H][W][3] world, hit where depth > 0)
__global__ void icp_pack_reference_kernel(const float* __restrict__ v3,
                                          const float* __restrict__ depth, int n,
                                          float4* __restrict__ vert) {
  chain_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  vert[i] = depth[i] > 0.f ? make_float4(v3[3 * (size_t)i], v3[3 * (size_t)i + 1],
                                         v3[3 * (size_t)i + 2], 1.f)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
}

// normals: (V(x+1) - V(x-1)) x (V(y+1) - V(y-1)) with all four neighbours
// valid, turned to face `centre`
__global__ void icp_normal_kernel(const float4* __restrict__ vert, int W, int H, float ox,
                                  float oy, float oz, float4* __restrict__ norm) {
  chain_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= W * H) return;
  const int x = i % W, y = i / W;
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  if (x > 0 && y > 0 && x < W - 1 && y < H - 1) {
    const float4 c = vert[i], l = vert[i - 1], r = vert[i + 1], u = vert[i - W], d = vert[i + W];
    if (c.w > 0.f && l.w > 0.f && r.w > 0.f && u.w > 0.f && d.w > 0.f) {
      const float ax = r.x - l.x, ay = r.y - l.y, az = r.z - l.z;
      const float bx = d.x - u.x, by = d.y - u.y, bz = d.z - u.z;
      float nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
      const float nn = sqrtf(nx * nx + ny * ny + nz * nz);
      if (nn > 0.f) {
        nx /= nn;
        ny /= nn;
        nz /= nn;
        if ((c.x - ox) * nx + (c.y - oy) * ny + (c.z - oz) * nz > 0.f) {
          nx = -nx;
          ny = -ny;
          nz = -nz;
        }
        out = make_float4(nx, ny, nz, 1.f);
      }
    }
  }
  norm[i] = out;
}

struct IcpIter {
  const float4* vert;  // level maps
  const float4* norm;
  int n;               // level pixels
  const float4* rvert; // reference maps, full resolution
  const float4* rnorm;
  int Wr, Hr;
  float fx, fy, cx, cy;   // reference intrinsics
  float Rr[9], tr[3];     // reference pose (camera -> world)
  float eps_d2, cos_theta;
  float* pose;            // [12] R row-major, t
  float* partials;        // [grid][32]
  unsigned int* ticket;
  float* stats;           // nullable: [2] for this iteration
};

// Cholesky of the 6x6 normal equations and the SE(3) exponential in single
// precision, one thread (B300's FP64 rate is a small fraction of its FP32
// rate, and Gauss-Newton corrects the rounding of one step in the next).
// Leaves the pose unchanged when the system has fewer than six inliers or a
// pivot at most 1e-6 of the largest diagonal.
__device__ void icp_solve_and_update(const float* S, float* pose, float* stats) {
  float A[6][6], b[6];
  int k = 0;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int c = a; c < 6; ++c) {
      A[a][c] = S[k];
      A[c][a] = S[k];
      ++k;
    }
#pragma unroll
  for (int a = 0; a < 6; ++a) b[a] = S[21 + a];
  if (stats) {
    stats[0] = S[28];
    stats[1] = S[27];
  }
  if (!(S[28] >= 6.0f)) return;
  float dmax = 0.0f;
#pragma unroll
  for (int a = 0; a < 6; ++a) dmax = fmaxf(dmax, A[a][a]);
  float L[6][6] = {};
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float sj = A[j][j];
#pragma unroll
    for (int m = 0; m < j; ++m) sj -= L[j][m] * L[j][m];
    if (!(sj > 1e-6f * dmax)) return;
    L[j][j] = sqrtf(sj);
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      float t = A[i][j];
#pragma unroll
      for (int m = 0; m < j; ++m) t -= L[i][m] * L[j][m];
      L[i][j] = t / L[j][j];
    }
  }
  float y[6], xi[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float t = -b[i];
#pragma unroll
    for (int m = 0; m < i; ++m) t -= L[i][m] * y[m];
    y[i] = t / L[i][i];
  }
#pragma unroll
  for (int i = 5; i >= 0; --i) {
    float t = y[i];
#pragma unroll
    for (int m = i + 1; m < 6; ++m) t -= L[m][i] * xi[m];
    xi[i] = t / L[i][i];
  }
  // exp of the twist (v, w): R = I + a [w] + b [w]^2, V = I + b [w] + c [w]^2
  // with a = sin t / t, b = (1 - cos t) / t^2 = 2 sin^2(t/2) / t^2 and
  // c = (t - sin t) / t^3, the last by its Taylor series below t = 0.1
  // (truncation below 1e-12; the closed form cancels in single precision)
  const float wx = xi[3], wy = xi[4], wz = xi[5];
  const float th2 = wx * wx + wy * wy + wz * wz, th = sqrtf(th2);
  float ca, cb, cc;
  if (th < 0.1f) {
    ca = 1.0f - th2 * (1.0f / 6.0f) * (1.0f - th2 * (1.0f / 20.0f));
    cb = 0.5f - th2 * (1.0f / 24.0f) * (1.0f - th2 * (1.0f / 30.0f));
    cc = (1.0f / 6.0f) - th2 * (1.0f / 120.0f) * (1.0f - th2 * (1.0f / 42.0f));
  } else {
    const float sh = sinf(0.5f * th);
    ca = sinf(th) / th;
    cb = 2.0f * sh * sh / th2;
    cc = (th - sinf(th)) / (th2 * th);
  }
  const float W[9] = {0.f, -wz, wy, wz, 0.f, -wx, -wy, wx, 0.f};
  float W2[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      W2[r * 3 + c] = W[r * 3] * W[c] + W[r * 3 + 1] * W[3 + c] + W[r * 3 + 2] * W[6 + c];
  float Re[9], Ve[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const float I = (e % 4 == 0) ? 1.0f : 0.0f;
    Re[e] = I + ca * W[e] + cb * W2[e];
    Ve[e] = I + cb * W[e] + cc * W2[e];
  }
  float R[9], t[3];
#pragma unroll
  for (int e = 0; e < 9; ++e) R[e] = pose[e];
#pragma unroll
  for (int e = 0; e < 3; ++e) t[e] = pose[9 + e];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      pose[r * 3 + c] = Re[r * 3] * R[c] + Re[r * 3 + 1] * R[3 + c] + Re[r * 3 + 2] * R[6 + c];
    pose[9 + r] = Re[r * 3] * t[0] + Re[r * 3 + 1] * t[1] + Re[r * 3 + 2] * t[2] +
                  Ve[r * 3] * xi[0] + Ve[r * 3 + 1] * xi[1] + Ve[r * 3 + 2] * xi[2];
  }
}

__global__ void __launch_bounds__(kIcpThreads) icp_iteration_kernel(const __grid_constant__ IcpIter a) {
  chain_wait();
  __shared__ float s_part[kIcpThreads / 32][kIcpSums];
  __shared__ float s_sum[kIcpSums];
  __shared__ bool s_last;
  float R[9], t[3];
#pragma unroll
  for (int e = 0; e < 9; ++e) R[e] = a.pose[e];
#pragma unroll
  for (int e = 0; e < 3; ++e) t[e] = a.pose[9 + e];
  float acc[kIcpSums];
#pragma unroll
  for (int k = 0; k < kIcpSums; ++k) acc[k] = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const float4 v = a.vert[i], nl = a.norm[i];
    if (!(v.w > 0.f && nl.w > 0.f)) continue;
    const float px = R[0] * v.x + R[1] * v.y + R[2] * v.z + t[0];
    const float py = R[3] * v.x + R[4] * v.y + R[5] * v.z + t[1];
    const float pz = R[6] * v.x + R[7] * v.y + R[8] * v.z + t[2];
    const float ncx = R[0] * nl.x + R[1] * nl.y + R[2] * nl.z;
    const float ncy = R[3] * nl.x + R[4] * nl.y + R[5] * nl.z;
    const float ncz = R[6] * nl.x + R[7] * nl.y + R[8] * nl.z;
    // reference camera frame: X = R_ref^T (p - t_ref)
    const float dx = px - a.tr[0], dy = py - a.tr[1], dz = pz - a.tr[2];
    const float X = a.Rr[0] * dx + a.Rr[3] * dy + a.Rr[6] * dz;
    const float Y = a.Rr[1] * dx + a.Rr[4] * dy + a.Rr[7] * dz;
    const float Z = a.Rr[2] * dx + a.Rr[5] * dy + a.Rr[8] * dz;
    if (!(Z > 0.f)) continue;
    const float u = floorf(a.fx * X / Z + a.cx + 0.5f), w = floorf(a.fy * Y / Z + a.cy + 0.5f);
    if (!(u >= 0.f && u < (float)a.Wr && w >= 0.f && w < (float)a.Hr)) continue;
    const int j = (int)w * a.Wr + (int)u;
    const float4 q = a.rvert[j], n = a.rnorm[j];
    if (!(q.w > 0.f && n.w > 0.f)) continue;
    const float ex = px - q.x, ey = py - q.y, ez = pz - q.z;
    if (!(ex * ex + ey * ey + ez * ez < a.eps_d2)) continue;
    if (!(ncx * n.x + ncy * n.y + ncz * n.z > a.cos_theta)) continue;
    const float r = ex * n.x + ey * n.y + ez * n.z;
    const float J[6] = {n.x, n.y, n.z, py * n.z - pz * n.y, pz * n.x - px * n.z,
                        px * n.y - py * n.x};
    int k = 0;
#pragma unroll
    for (int p = 0; p < 6; ++p)
#pragma unroll
      for (int c = p; c < 6; ++c) acc[k++] += J[p] * J[c];
#pragma unroll
    for (int p = 0; p < 6; ++p) acc[21 + p] += J[p] * r;
    acc[27] += r * r;
    acc[28] += 1.f;
  }
  // block sums in a fixed order: butterfly within each warp, then warps in order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kIcpSums; ++k) {
    float x = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_part[warp][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < kIcpSums) {
    float x = 0.f;
#pragma unroll
    for (int w2 = 0; w2 < kIcpThreads / 32; ++w2) x += s_part[w2][threadIdx.x];
    a.partials[(size_t)blockIdx.x * 32 + threadIdx.x] = x;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  // last block: every partial is visible (fence before each ticket); the
  // block's threads add them in the same fixed order as above
#pragma unroll
  for (int k = 0; k < kIcpSums; ++k) acc[k] = 0.f;
  for (int bk = threadIdx.x; bk < (int)gridDim.x; bk += blockDim.x) {
#pragma unroll
    for (int k = 0; k < kIcpSums; ++k) acc[k] += __ldcg(a.partials + (size_t)bk * 32 + k);
  }
#pragma unroll
  for (int k = 0; k < kIcpSums; ++k) {
    float x = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_part[warp][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < kIcpSums) {
    float x = 0.f;
#pragma unroll
    for (int w2 = 0; w2 < kIcpThreads / 32; ++w2) x += s_part[w2][threadIdx.x];
    s_sum[threadIdx.x] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    icp_solve_and_update(s_sum, a.pose, a.stats);
    *a.ticket = 0u;  // ready for the next iteration's launch
  }
}

}  // namespace gps

// ------------------------------------------------------------------ C ABI
namespace gps {
void set_error(const char* msg);  // capi.cu: sets gps_last_error() of this thread
}

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct IcpLayout {
  int W[gps::kIcpMaxLevels], H[gps::kIcpMaxLevels];
  size_t depth[gps::kIcpMaxLevels];  // level >= 1 depth maps
  size_t vert[gps::kIcpMaxLevels], norm[gps::kIcpMaxLevels];
  size_t rvert, rnorm, partials, ticket, total;
  int grid;
};

int icp_grid() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 148;
  }
  return 4 * sms;
}

bool icp_settings_ok(const GpsIcpSettings* s) {
  if (!s || s->levels < 1 || s->levels > gps::kIcpMaxLevels) return false;
  for (int l = 0; l < gps::kIcpMaxLevels; ++l)
    if (s->iters[l] < 0) return false;
  return s->eps_d > 0.f && s->eps_theta_deg > 0.f && s->eps_theta_deg < 180.f;
}

bool icp_layout(int W, int H, const GpsIcpSettings* s, int grid, IcpLayout& L) {
  size_t off = 0;
  for (int l = 0; l < s->levels; ++l) {
    L.W[l] = l ? L.W[l - 1] / 2 : W;
    L.H[l] = l ? L.H[l - 1] / 2 : H;
    if (L.W[l] < 3 || L.H[l] < 3) return false;
    const size_t n = (size_t)L.W[l] * L.H[l];
    L.depth[l] = off;
    if (l) off = a256(off + n * 4);
    L.vert[l] = off; off = a256(off + n * 16);
    L.norm[l] = off; off = a256(off + n * 16);
  }
  const size_t n0 = (size_t)W * H;
  L.rvert = off; off = a256(off + n0 * 16);
  L.rnorm = off; off = a256(off + n0 * 16);
  L.partials = off; off = a256(off + (size_t)grid * 32 * 4);
  L.ticket = off; off = a256(off + 4);
  L.total = off;
  L.grid = grid;
  return true;
}

int32_t icp_fail(int32_t code, const char* msg) {
  gps::set_error(msg);
  return code;
}

}  // namespace

extern "C" {

int32_t gps_icp_workspace_size(int32_t width, int32_t height, const GpsIcpSettings* s,
                               size_t* bytes) {
  IcpLayout L{};
  if (!bytes || !icp_settings_ok(s) || width <= 0 || height <= 0 ||
      !icp_layout(width, height, s, icp_grid(), L))
    return icp_fail(GPS_ERR_INVALID_ARG, "gps_icp_workspace_size: bad sizes or settings");
  *bytes = L.total;
  return GPS_OK;
}

int32_t icp_track(const GpsIntrinsics* K, const float* depth, const float* ref_vertex,
                  const float* ref_depth, const GpsPose* T_ref, const GpsIcpSettings* s,
                  float* pose, void* ws, size_t ws_bytes, float* stats, void* stream) {
  if (!K || !depth || !ref_vertex || !ref_depth || !T_ref || !pose || !ws)
    return icp_fail(GPS_ERR_INVALID_ARG, "icp_track: NULL argument");
  if (!icp_settings_ok(s) || K->width <= 0 || K->height <= 0 || !(K->fx > 0) || !(K->fy > 0))
    return icp_fail(GPS_ERR_INVALID_ARG, "icp_track: bad intrinsics or settings");
  IcpLayout L{};
  if (!icp_layout(K->width, K->height, s, icp_grid(), L))
    return icp_fail(GPS_ERR_INVALID_ARG, "icp_track: a pyramid level is smaller than 3 x 3");
  if (ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255))
    return icp_fail(GPS_ERR_WORKSPACE_TOO_SMALL,
                    "icp_track: workspace smaller than gps_icp_workspace_size or unaligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* b = static_cast<char*>(ws);
  const int T = gps::kIcpThreads;
  auto blocks = [&](size_t n) { return (unsigned)((n + T - 1) / T); };
  // pyramid, vertex and normal maps (camera frame: the camera at the origin)
  const float* dl[gps::kIcpMaxLevels];
  float fx = K->fx, fy = K->fy, cx = K->cx, cy = K->cy;
  for (int l = 0; l < s->levels; ++l) {
    if (l) {
      float* d = reinterpret_cast<float*>(b + L.depth[l]);
      gps::launch_chained(gps::icp_downsample_kernel, dim3(blocks((size_t)L.W[l] * L.H[l])),
                          dim3(T), 0, st, dl[l - 1], L.W[l - 1], d, L.W[l], L.H[l]);
      dl[l] = d;
      fx *= 0.5f;
      fy *= 0.5f;
      cx *= 0.5f;
      cy *= 0.5f;
    } else {
      dl[0] = depth;
    }
    float4* v = reinterpret_cast<float4*>(b + L.vert[l]);
    const size_t n = (size_t)L.W[l] * L.H[l];
    gps::launch_chained(gps::icp_vertex_kernel, dim3(blocks(n)), dim3(T), 0, st, dl[l], L.W[l],
                        L.H[l], fx, fy, cx, cy, v);
    gps::launch_chained(gps::icp_normal_kernel, dim3(blocks(n)), dim3(T), 0, st, v, L.W[l], L.H[l],
                        0.f, 0.f, 0.f, reinterpret_cast<float4*>(b + L.norm[l]));
  }
  const size_t n0 = (size_t)K->width * K->height;
  float4* rv = reinterpret_cast<float4*>(b + L.rvert);
  float4* rn = reinterpret_cast<float4*>(b + L.rnorm);
  gps::launch_chained(gps::icp_pack_reference_kernel, dim3(blocks(n0)), dim3(T), 0, st,
                      ref_vertex, ref_depth, (int)n0, rv);
  gps::launch_chained(gps::icp_normal_kernel, dim3(blocks(n0)), dim3(T), 0, st, rv, K->width,
                      K->height, T_ref->t[0], T_ref->t[1], T_ref->t[2], rn);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(b + L.ticket);
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st);
  gps::IcpIter a{};
  a.rvert = rv;
  a.rnorm = rn;
  a.Wr = K->width;
  a.Hr = K->height;
  a.fx = K->fx;
  a.fy = K->fy;
  a.cx = K->cx;
  a.cy = K->cy;
  for (int k = 0; k < 9; ++k) a.Rr[k] = T_ref->R[k];
  for (int k = 0; k < 3; ++k) a.tr[k] = T_ref->t[k];
  a.eps_d2 = s->eps_d * s->eps_d;
  a.cos_theta = (float)std::cos((double)s->eps_theta_deg * 3.14159265358979323846 / 180.0);
  a.pose = pose;
  a.partials = reinterpret_cast<float*>(b + L.partials);
  a.ticket = ticket;
  int it_index = 0;
  for (int l = s->levels - 1; l >= 0 && e == cudaSuccess; --l) {
    a.vert = reinterpret_cast<const float4*>(b + L.vert[l]);
    a.norm = reinterpret_cast<const float4*>(b + L.norm[l]);
    a.n = L.W[l] * L.H[l];
    // about two pixels per thread, at most L.grid blocks
    const unsigned grid = (unsigned)std::min<size_t>(L.grid, (a.n + 2 * T - 1) / (2 * T));
    for (int it = 0; it < s->iters[l]; ++it, ++it_index) {
      a.stats = stats ? stats + 2 * it_index : nullptr;
      gps::launch_chained(gps::icp_iteration_kernel, dim3(grid), dim3(T), 0, st, a);
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return icp_fail(GPS_ERR_CUDA, cudaGetErrorString(e));
  return GPS_OK;
}

}  // extern "C"
