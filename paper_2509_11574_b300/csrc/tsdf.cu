// Colourised TSDF fusion and SDF ray-cast (Sec. 3.1 first pass, Sec. 3.2.1).
//
// Layout: 8^3 bricks, x fastest inside a brick (see GpsTsdf).  A warp of the
// fusion kernel covers an 8 x 4 x 1 slab of one brick, so its 32 voxels project
// to a compact image patch and its sdf / weight loads are one 128-byte line.
// The ray-cast maps a warp to an 8 x 4 pixel block so neighbouring rays touch
// the same bricks.
#include <cuda_runtime.h>

#include "gps_common.cuh"

namespace gps {

struct VolDev {
  int nx, ny, nz;
  float voxel, ox, oy, oz, trunc, wmax;
  float* sdf;
  float* weight;
  float4* rgbw;
  uint8_t* flags;  // nullable: per brick, nonzero if some voxel may be != 1
};

__device__ __forceinline__ long long brick_of(const VolDev& v, int x, int y, int z) {
  return ((long long)(z >> 3) * (v.ny >> 3) + (y >> 3)) * (v.nx >> 3) + (x >> 3);
}

__device__ __forceinline__ long long vox_index(const VolDev& v, int x, int y, int z) {
  const int nbx = v.nx >> 3, nby = v.ny >> 3;
  const long long brick = ((long long)(z >> 3) * nby + (y >> 3)) * nbx + (x >> 3);
  return brick * 512 + ((z & 7) << 6) + ((y & 7) << 3) + (x & 7);
}

// camera coordinates of a world point: X_c = R^T (X_w - t)
__device__ __forceinline__ void world_to_cam(const Cam& c, float wx, float wy, float wz,
                                             float& x, float& y, float& z) {
  const float d0 = wx - c.t[0], d1 = wy - c.t[1], d2 = wz - c.t[2];
  x = c.R[0] * d0 + c.R[3] * d1 + c.R[6] * d2;
  y = c.R[1] * d0 + c.R[4] * d1 + c.R[7] * d2;
  z = c.R[2] * d0 + c.R[5] * d1 + c.R[8] * d2;
}

__global__ void __launch_bounds__(256) fuse_kernel(VolDev v, const float* __restrict__ depth,
                                                   const float* __restrict__ rgb, Cam cam) {
  const long long n = (long long)v.nx * v.ny * v.nz;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n) return;
  const int local = (int)(id & 511);
  const long long brick = id >> 9;
  const int nbx = v.nx >> 3, nby = v.ny >> 3;
  const int bx = (int)(brick % nbx), by = (int)((brick / nbx) % nby),
            bz = (int)(brick / ((long long)nbx * nby));
  const int x = (bx << 3) + (local & 7), y = (by << 3) + ((local >> 3) & 7),
            z = (bz << 3) + (local >> 6);
  const float wx = v.ox + (x + 0.5f) * v.voxel, wy = v.oy + (y + 0.5f) * v.voxel,
              wz = v.oz + (z + 0.5f) * v.voxel;
  float xc, yc, zc;
  world_to_cam(cam, wx, wy, wz, xc, yc, zc);
  if (!(zc > 0.0f)) return;
  const float u = cam.fx * xc / zc + cam.cx, vv = cam.fy * yc / zc + cam.cy;
  const float pu = floorf(u + 0.5f), pv = floorf(vv + 0.5f);
  if (!(pu >= 0.0f) || !(pv >= 0.0f) || pu > (float)(cam.W - 1) || pv > (float)(cam.H - 1)) return;
  const long long pix = (long long)pv * cam.W + (long long)pu;
  const float D = __ldg(depth + pix);
  if (!(D > 0.0f)) return;
  const float eta = D - zc;
  if (eta < -v.trunc) return;
  const float f = fminf(1.0f, eta / v.trunc);
  const float w0 = v.weight[id], s0 = v.sdf[id];
  const float s1 = (w0 * s0 + f) / (w0 + 1.0f);
  v.sdf[id] = s1;
  if (v.flags && s1 != 1.0f) v.flags[brick] = 1;
  v.weight[id] = fminf(w0 + 1.0f, v.wmax);
  if (fabsf(eta) < v.trunc) {
    float4 c = v.rgbw[id];
    const long long npx = (long long)cam.W * cam.H;
    const float cw = c.w, inv = 1.0f / (cw + 1.0f);
    c.x = (cw * c.x + __ldg(rgb + pix)) * inv;
    c.y = (cw * c.y + __ldg(rgb + npx + pix)) * inv;
    c.z = (cw * c.z + __ldg(rgb + 2 * npx + pix)) * inv;
    c.w = fminf(cw + 1.0f, v.wmax);
    v.rgbw[id] = c;
  }
}

// trilinear sample of the sdf at continuous voxel coordinate g (centres at integers)
__device__ __forceinline__ float sample_sdf(const VolDev& v, float gx, float gy, float gz) {
  int ix = (int)floorf(gx), iy = (int)floorf(gy), iz = (int)floorf(gz);
  ix = min(max(ix, 0), v.nx - 2);
  iy = min(max(iy, 0), v.ny - 2);
  iz = min(max(iz, 0), v.nz - 2);
  const float fx = gx - ix, fy = gy - iy, fz = gz - iz;
  // all eight voxels in clear bricks: they hold 1, no loads (the arithmetic
  // below is the same, so is the sample)
  bool clear = v.flags != nullptr;
  if (clear) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      clear = clear && !v.flags[brick_of(v, ix + (k & 1), iy + ((k >> 1) & 1), iz + (k >> 2))];
  }
  float c000 = 1.0f, c100 = 1.0f, c010 = 1.0f, c110 = 1.0f, c001 = 1.0f, c101 = 1.0f,
        c011 = 1.0f, c111 = 1.0f;
  if (!clear) {
    const float* s = v.sdf;
    c000 = __ldg(s + vox_index(v, ix, iy, iz));
    c100 = __ldg(s + vox_index(v, ix + 1, iy, iz));
    c010 = __ldg(s + vox_index(v, ix, iy + 1, iz));
    c110 = __ldg(s + vox_index(v, ix + 1, iy + 1, iz));
    c001 = __ldg(s + vox_index(v, ix, iy, iz + 1));
    c101 = __ldg(s + vox_index(v, ix + 1, iy, iz + 1));
    c011 = __ldg(s + vox_index(v, ix, iy + 1, iz + 1));
    c111 = __ldg(s + vox_index(v, ix + 1, iy + 1, iz + 1));
  }
  const float c00 = c000 * (1.0f - fx) + c100 * fx, c10 = c010 * (1.0f - fx) + c110 * fx;
  const float c01 = c001 * (1.0f - fx) + c101 * fx, c11 = c011 * (1.0f - fx) + c111 * fx;
  const float c0 = c00 * (1.0f - fy) + c10 * fy, c1 = c01 * (1.0f - fy) + c11 * fy;
  return c0 * (1.0f - fz) + c1 * fz;
}

__device__ __forceinline__ float3 sample_rgb(const VolDev& v, float gx, float gy, float gz) {
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
    const float4 c = __ldg(v.rgbw + vox_index(v, ix + dx, iy + dy, iz + dz));
    acc.x += w * c.x;
    acc.y += w * c.y;
    acc.z += w * c.z;
  }
  return acc;
}

__global__ void __launch_bounds__(256) raycast_kernel(VolDev v, Cam cam, float near_, float far_,
                                                      void* __restrict__ out_rgb, int rgb_prec,
                                                      float* __restrict__ out_depth,
                                                      float* __restrict__ out_vertex) {
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

// One block per brick: flag = some voxel's sdf differs from 1.
__global__ void __launch_bounds__(256) mark_bricks_kernel(const float* __restrict__ sdf,
                                                          uint8_t* __restrict__ flags) {
  const float* b = sdf + (size_t)blockIdx.x * 512;
  const bool any = b[threadIdx.x] != 1.0f || b[threadIdx.x + 256] != 1.0f;
  const int n = __syncthreads_or(any);
  if (threadIdx.x == 0) flags[blockIdx.x] = n ? 1 : 0;
}

cudaError_t launch_mark_bricks(const GpsTsdf& t, cudaStream_t st) {
  const long long nb = ((long long)t.nx * t.ny * t.nz) >> 9;
  if (nb > 0) mark_bricks_kernel<<<(unsigned)nb, 256, 0, st>>>(t.sdf, t.brick_flags);
  return cudaGetLastError();
}

cudaError_t launch_fuse(const GpsTsdf& t, const float* depth, const float* rgb, const Cam& cam,
                        cudaStream_t st) {
  VolDev v{t.nx, t.ny, t.nz, t.voxel, t.origin[0], t.origin[1], t.origin[2], t.trunc,
           t.max_weight, t.sdf, t.weight, reinterpret_cast<float4*>(t.rgbw), t.brick_flags};
  const long long n = (long long)t.nx * t.ny * t.nz;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  fuse_kernel<<<blocks, 256, 0, st>>>(v, depth, rgb, cam);
  return cudaGetLastError();
}

cudaError_t launch_raycast(const GpsTsdf& t, const Cam& cam, float near_, float far_, void* rgb,
                           int rgb_prec, float* depth, float* vertex, cudaStream_t st) {
  VolDev v{t.nx, t.ny, t.nz, t.voxel, t.origin[0], t.origin[1], t.origin[2], t.trunc,
           t.max_weight, t.sdf, t.weight, reinterpret_cast<float4*>(t.rgbw), t.brick_flags};
  dim3 grid((cam.W + 15) / 16, (cam.H + 15) / 16);
  raycast_kernel<<<grid, 256, 0, st>>>(v, cam, near_, far_, rgb, rgb_prec, depth, vertex);
  return cudaGetLastError();
}

}  // namespace gps
