// Colourised TSDF fusion and SDF ray-cast (Sec. 3.1 first pass, Sec. 3.2.1).
//
// Layout: 8^3 bricks, x fastest inside a brick (see GpsTsdf).  A warp of the
// fusion kernel covers an 8 x 4 x 1 slab of one brick, so its 32 voxels project
// to a compact image patch and its sdf / weight loads are one 128-byte line.
// The ray-cast maps a warp to an 8 x 4 pixel block so neighbouring rays touch
// the same bricks.
#include <cuda_runtime.h>

#include "tsdf_common.cuh"

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


// Dense accessor of the shared sampling and ray-cast code.
struct DenseVol : VolDev {
  __device__ __forceinline__ bool load8(int ix, int iy, int iz, float* c) const {
    // all eight voxels in clear bricks: they hold 1, no loads.  The stencil
    // spans one or two bricks per axis; each distinct brick's flag is read
    // once (one flag for the 2 x 2 x 2 stencils inside one brick).
    if (flags) {
      const int nbx = nx >> 3, nby = ny >> 3;
      const bool dx = ((ix + 1) >> 3) != (ix >> 3), dy = ((iy + 1) >> 3) != (iy >> 3),
                 dz = ((iz + 1) >> 3) != (iz >> 3);
      const long long b0 = brick_of(*this, ix, iy, iz), sy = nbx, sz = (long long)nbx * nby;
      bool clear = !flags[b0] && !(dx && flags[b0 + 1]);
      if (dy) clear = clear && !flags[b0 + sy] && !(dx && flags[b0 + sy + 1]);
      if (dz) {
        clear = clear && !flags[b0 + sz] && !(dx && flags[b0 + sz + 1]);
        if (dy) clear = clear && !flags[b0 + sz + sy] && !(dx && flags[b0 + sz + sy + 1]);
      }
      if (clear) return false;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      c[k] = __ldg(sdf + vox_index(*this, ix + (k & 1), iy + ((k >> 1) & 1), iz + (k >> 2)));
    return true;
  }
  __device__ __forceinline__ float4 rgbw(int ix, int iy, int iz) const {
    return __ldg(VolDev::rgbw + vox_index(*this, ix, iy, iz));
  }
};

// One CTA of 512 threads per 8^3 brick, the grid laid out as the bricks
// (gridDim = bricks per axis), so a voxel's coordinates come from its block
// and thread indices without integer division.
__global__ void __launch_bounds__(512) fuse_kernel(VolDev v, const float* __restrict__ depth,
                                                   const float* __restrict__ rgb, Cam cam) {
  chain_wait();
  const int local = threadIdx.x;
  const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
  const long long brick = ((long long)bz * gridDim.y + by) * gridDim.x + bx;
  const long long id = brick * 512 + local;
  const int x = (bx << 3) + (local & 7), y = (by << 3) + ((local >> 3) & 7),
            z = (bz << 3) + (local >> 6);
  float eta;
  const long long pix = voxel_pixel(v.voxel, v.ox, v.oy, v.oz, cam, depth, x, y, z, eta);
  if (pix < 0 || eta < -v.trunc) return;
  const float s1 = voxel_update(v.trunc, v.wmax, cam, rgb, pix, eta, v.sdf, v.weight, v.rgbw, id);
  if (v.flags && s1 != 1.0f) v.flags[brick] = 1;
}

// One block per brick: flag = some voxel's sdf differs from 1.
__global__ void __launch_bounds__(256) mark_bricks_kernel(const float* __restrict__ sdf,
                                                          uint8_t* __restrict__ flags) {
  chain_wait();
  const float* b = sdf + (size_t)blockIdx.x * 512;
  const bool any = b[threadIdx.x] != 1.0f || b[threadIdx.x + 256] != 1.0f;
  const int n = __syncthreads_or(any);
  if (threadIdx.x == 0) flags[blockIdx.x] = n ? 1 : 0;
}

cudaError_t launch_mark_bricks(const GpsTsdf& t, cudaStream_t st) {
  const long long nb = ((long long)t.nx * t.ny * t.nz) >> 9;
  if (nb > 0) launch_chained(mark_bricks_kernel, dim3((unsigned)nb), dim3(256), 0, st, t.sdf,
                             t.brick_flags);
  return cudaGetLastError();
}

cudaError_t launch_fuse(const GpsTsdf& t, const float* depth, const float* rgb, const Cam& cam,
                        cudaStream_t st) {
  VolDev v{t.nx, t.ny, t.nz, t.voxel, t.origin[0], t.origin[1], t.origin[2], t.trunc,
           t.max_weight, t.sdf, t.weight, reinterpret_cast<float4*>(t.rgbw), t.brick_flags};
  const dim3 grid((unsigned)(t.nx >> 3), (unsigned)(t.ny >> 3), (unsigned)(t.nz >> 3));
  launch_chained(fuse_kernel, grid, dim3(512), 0, st, v, depth, rgb, cam);
  return cudaGetLastError();
}

cudaError_t launch_raycast(const GpsTsdf& t, const Cam& cam, float near_, float far_, void* rgb,
                           int rgb_prec, float* depth, float* vertex, cudaStream_t st) {
  DenseVol v{};
  static_cast<VolDev&>(v) = VolDev{t.nx, t.ny, t.nz, t.voxel, t.origin[0], t.origin[1],
                                   t.origin[2], t.trunc, t.max_weight, t.sdf, t.weight,
                                   reinterpret_cast<float4*>(t.rgbw), t.brick_flags};
  dim3 grid((cam.W + 15) / 16, (cam.H + 15) / 16);
  launch_chained(raycast_kernel<DenseVol>, grid, dim3(256), 0, st, v, cam, near_, far_, rgb,
                 rgb_prec, depth, vertex);
  return cudaGetLastError();
}

}  // namespace gps
