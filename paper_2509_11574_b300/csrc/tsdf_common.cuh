// TSDF helpers shared by the dense grid (tsdf.cu) and the voxel-hash volume
// (hash.cu): the per-voxel fusion update and the ray-cast march, written once
// over a volume accessor so that both volumes run the same arithmetic.
// Internal header.
#pragma once
#include <cuda_runtime.h>

#include "gps_common.cuh"

namespace gps {

// camera coordinates of a world point: X_c = R^T (X_w - t)
__device__ __forceinline__ void world_to_cam(const Cam& c, float wx, float wy, float wz,
                                             float& x, float& y, float& z) {
  const float d0 = wx - c.t[0], d1 = wy - c.t[1], d2 = wz - c.t[2];
  x = c.R[0] * d0 + c.R[3] * d1 + c.R[6] * d2;
  y = c.R[1] * d0 + c.R[4] * d1 + c.R[7] * d2;
  z = c.R[2] * d0 + c.R[5] * d1 + c.R[8] * d2;
}

// Fusion (Sec. 3.2.1) of the voxel with integer coordinates (x, y, z), part
// 1: the pixel its centre projects to (nearest, floor(u + 0.5)) and
// eta = D - z_c.  Returns -1 when the frame has nothing for it (behind the
// camera, outside the image, no depth).
__device__ __forceinline__ long long voxel_pixel(float voxel, float ox, float oy, float oz,
                                                 const Cam& cam, const float* __restrict__ depth,
                                                 int x, int y, int z, float& eta) {
  const float wx = ox + (x + 0.5f) * voxel, wy = oy + (y + 0.5f) * voxel,
              wz = oz + (z + 0.5f) * voxel;
  float xc, yc, zc;
  world_to_cam(cam, wx, wy, wz, xc, yc, zc);
  if (!(zc > 0.0f)) return -1;
  const float u = cam.fx * xc / zc + cam.cx, vv = cam.fy * yc / zc + cam.cy;
  const float pu = floorf(u + 0.5f), pv = floorf(vv + 0.5f);
  if (!(pu >= 0.0f) || !(pv >= 0.0f) || pu > (float)(cam.W - 1) || pv > (float)(cam.H - 1))
    return -1;
  const long long pix = (long long)pv * cam.W + (long long)pu;
  const float D = __ldg(depth + pix);
  if (!(D > 0.0f)) return -1;
  eta = D - zc;
  return pix;
}

// part 2: the running averages at storage index id, for eta >= -trunc.
// Returns the new sdf.
__device__ __forceinline__ float voxel_update(float trunc, float wmax, const Cam& cam,
                                              const float* __restrict__ rgb, long long pix,
                                              float eta, float* sdf, float* weight,
                                              float4* rgbw, long long id) {
  const float f = fminf(1.0f, eta / trunc);
  const float w0 = weight[id], s0 = sdf[id];
  const float s1 = (w0 * s0 + f) / (w0 + 1.0f);
  sdf[id] = s1;
  weight[id] = fminf(w0 + 1.0f, wmax);
  if (fabsf(eta) < trunc) {
    float4 c = rgbw[id];
    const long long npx = (long long)cam.W * cam.H;
    const float cw = c.w, inv = 1.0f / (cw + 1.0f);
    c.x = (cw * c.x + __ldg(rgb + pix)) * inv;
    c.y = (cw * c.y + __ldg(rgb + npx + pix)) * inv;
    c.z = (cw * c.z + __ldg(rgb + 2 * npx + pix)) * inv;
    c.w = fminf(cw + 1.0f, wmax);
    rgbw[id] = c;
  }
  return s1;
}

// Trilinear samples at continuous voxel coordinate g (centres at integers),
// the stencil clamped to the grid.  A volume accessor provides
//   bool load8(ix, iy, iz, float c[8])  - the sdf of the 8 stencil voxels
//                                          (c[k] at (ix + (k&1), iy + (k>>1&1),
//                                          iz + (k>>2))); false, with c
//                                          untouched, when all are known to
//                                          hold 1
//   float4 rgbw(ix, iy, iz)             - the colour of one voxel
template <class Vol>
__device__ __forceinline__ float sample_sdf(const Vol& v, float gx, float gy, float gz) {
  int ix = (int)floorf(gx), iy = (int)floorf(gy), iz = (int)floorf(gz);
  ix = min(max(ix, 0), v.nx - 2);
  iy = min(max(iy, 0), v.ny - 2);
  iz = min(max(iz, 0), v.nz - 2);
  const float fx = gx - ix, fy = gy - iy, fz = gz - iz;
  float c[8] = {1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f};
  v.load8(ix, iy, iz, c);
  const float c00 = c[0] * (1.0f - fx) + c[1] * fx, c10 = c[2] * (1.0f - fx) + c[3] * fx;
  const float c01 = c[4] * (1.0f - fx) + c[5] * fx, c11 = c[6] * (1.0f - fx) + c[7] * fx;
  const float c0 = c00 * (1.0f - fy) + c10 * fy, c1 = c01 * (1.0f - fy) + c11 * fy;
  return c0 * (1.0f - fz) + c1 * fz;
}

template <class Vol>
__device__ __forceinline__ float3 sample_rgb(const Vol& v, float gx, float gy, float gz) {
  int ix = (int)floorf(gx), iy = (int)floorf(gy), iz = (int)floorf(gz);
  ix = min(max(ix, 0), v.nx - 2);
  iy = min(max(iy, 0), v.ny - 2);
  iz = min(max(iz, 0), v.nz - 2);
  const float fx = gx - ix, fy = gy - iy, fz = gz - iz;
  float3 acc = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    const float w = (dx ? fx : 1.0f - fx) * (dy ? fy : 1.0f - fy) * (dz ? fz : 1.0f - fz);
    const float4 c = v.rgbw(ix + dx, iy + dy, iz + dz);
    acc.x += w * c.x;
    acc.y += w * c.y;
    acc.z += w * c.z;
  }
  return acc;
}

// Ray-cast (Sec. 3.1 first pass; the step rule and secant refinement of
// InfiniTAM): a warp covers an 8 x 4 pixel block, so neighbouring rays touch
// the same bricks.
template <class Vol>
__global__ void __launch_bounds__(256) raycast_kernel(const __grid_constant__ Vol v, Cam cam, float near_, float far_,
                                                      void* __restrict__ out_rgb, int rgb_prec,
                                                      float* __restrict__ out_depth,
                                                      float* __restrict__ out_vertex) {
  chain_wait();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int px = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
  const int py = blockIdx.y * 16 + (warp >> 1) * 4 + (lane >> 3);
  if (px >= cam.W || py >= cam.H) return;
  const long long npx = (long long)cam.W * cam.H, pix = (long long)py * cam.W + px;
  float dc0 = (px - cam.cx) / cam.fx, dc1 = (py - cam.cy) / cam.fy;
  float dw[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) dw[r] = cam.R[r * 3 + 0] * dc0 + cam.R[r * 3 + 1] * dc1 + cam.R[r * 3 + 2];
  const float inv_n = rsqrtf(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
  dw[0] *= inv_n;
  dw[1] *= inv_n;
  dw[2] *= inv_n;
  const float lo[3] = {v.ox + 0.5f * v.voxel, v.oy + 0.5f * v.voxel, v.oz + 0.5f * v.voxel};
  const float hi[3] = {v.ox + (v.nx - 0.5f) * v.voxel, v.oy + (v.ny - 0.5f) * v.voxel,
                       v.oz + (v.nz - 0.5f) * v.voxel};
  float s_in = -INFINITY, s_out = INFINITY;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (dw[k] != 0.0f) {
      const float a = (lo[k] - cam.t[k]) / dw[k], b = (hi[k] - cam.t[k]) / dw[k];
      s_in = fmaxf(s_in, fminf(a, b));
      s_out = fminf(s_out, fmaxf(a, b));
    } else if (cam.t[k] < lo[k] || cam.t[k] > hi[k]) {
      s_in = INFINITY;
    }
  }
  const float s0 = fmaxf(near_, s_in);
  const float s1 = far_ > 0.0f ? fminf(far_, s_out) : s_out;
  float3 col = make_float3(0.f, 0.f, 0.f);
  float depth = 0.0f, V[3] = {0.f, 0.f, 0.f};
  if (s0 < s1) {
    const float inv_vox = 1.0f / v.voxel;
    const float gox = (cam.t[0] - v.ox) * inv_vox - 0.5f, goy = (cam.t[1] - v.oy) * inv_vox - 0.5f,
                goz = (cam.t[2] - v.oz) * inv_vox - 0.5f;
    const float gdx = dw[0] * inv_vox, gdy = dw[1] * inv_vox, gdz = dw[2] * inv_vox;
    float sa = s0, fa = sample_sdf(v, gox + sa * gdx, goy + sa * gdy, goz + sa * gdz);
    float sb = 0.f, fb = 0.f;
    bool hit = false;
    const float min_step = 0.5f * v.voxel;
    // the march advances by at least min_step, so it ends after (s1 - s0) / min_step steps
    while (true) {
      const float step = fmaxf(fminf(fa, 1.0f) * v.trunc, min_step);
      sb = sa + step;
      if (sb > s1) break;
      fb = sample_sdf(v, gox + sb * gdx, goy + sb * gdy, goz + sb * gdz);
      if (fa > 0.0f && fb <= 0.0f) {
        hit = true;
        break;
      }
      sa = sb;
      fa = fb;
    }
    if (hit) {
      const float ss = sa + (sb - sa) * fa / (fa - fb);
      V[0] = cam.t[0] + ss * dw[0];
      V[1] = cam.t[1] + ss * dw[1];
      V[2] = cam.t[2] + ss * dw[2];
      float xc, yc, zc;
      world_to_cam(cam, V[0], V[1], V[2], xc, yc, zc);
      depth = zc;
      col = sample_rgb(v, (V[0] - v.ox) * inv_vox - 0.5f, (V[1] - v.oy) * inv_vox - 0.5f,
                       (V[2] - v.oz) * inv_vox - 0.5f);
    }
  }
  out_depth[pix] = depth;
  st_col(out_rgb, pix, rgb_prec, col.x);
  st_col(out_rgb, npx + pix, rgb_prec, col.y);
  st_col(out_rgb, 2 * npx + pix, rgb_prec, col.z);
  if (out_vertex) {
    out_vertex[pix * 3 + 0] = V[0];
    out_vertex[pix * 3 + 1] = V[1];
    out_vertex[pix * 3 + 2] = V[2];
  }
}

}  // namespace gps
