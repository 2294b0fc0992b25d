// Voxel-hashed TSDF (Sec. 3.2.1: the SDF lives in a hash table of voxel
// blocks, as in InfiniTAM).
//
// Per fused frame:
//   1. candidates: every pixel walks its band segment (camera depth D +- mu)
//      at half-brick steps and inserts the bricks within reach of the pixel's
//      frustum into a per-frame set (open addressing, cleared each frame);
//   2. allocation: one CTA per candidate brick tests its 512 voxels with the
//      fusion's own projection and band test; a brick with a band voxel is
//      inserted into the volume's table (CAS on the key, a slot from an
//      atomic counter, voxels initialised) - nothing waits on another thread;
//   3. fusion: the dense update on every allocated brick in view (a CTA per
//      brick, a conservative frustum cull first).
// The ray-cast reuses the dense march through an accessor that looks bricks
// up in the table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "tsdf_common.cuh"

namespace gps {

constexpr int kMaxProbe = 64;

__device__ __forceinline__ unsigned long long bucket_of(unsigned long long brick, int log2n) {
  return (brick * 0x9E3779B97F4A7C15ull) >> (64 - log2n);  // Fibonacci hashing
}

struct HashDev {
  int nx, ny, nz;
  float voxel, ox, oy, oz, trunc, wmax;
  int log2n;
  unsigned long long mask;
  int capacity;
  unsigned long long* keys;
  int* slots;
  long long* brick_of_slot;
  int* state;
  float* sdf;
  float* weight;
  float4* rgbw_p;
  uint8_t* flags;  // per slot, nullable: 1 once a voxel left sdf 1

  __device__ __forceinline__ long long brick(int x, int y, int z) const {
    return ((long long)(z >> 3) * (ny >> 3) + (y >> 3)) * (nx >> 3) + (x >> 3);
  }
  // pool slot of a brick, -1 when it is not stored (read-only use: the
  // table does not change during the kernels that call this)
  __device__ __forceinline__ int find(long long b) const {
    unsigned long long h = bucket_of((unsigned long long)b, log2n);
    const unsigned long long k1 = (unsigned long long)b + 1ull;
    for (int p = 0; p < kMaxProbe; ++p) {
      const unsigned long long k = __ldg(keys + h);
      if (k == k1) return __ldg(slots + h);
      if (k == 0ull) return -1;
      h = (h + 1ull) & mask;
    }
    return -1;
  }
  // accessor of the shared sampling code
  __device__ __forceinline__ bool load8(int ix, int iy, int iz, float* c) const {
    if ((ix & 7) != 7 && (iy & 7) != 7 && (iz & 7) != 7) {  // stencil inside one brick
      const int s = find(brick(ix, iy, iz));
      if (s < 0 || (flags && !flags[s])) return false;  // not stored, or only 1s
      const float* b = sdf + (size_t)s * 512 + ((iz & 7) << 6) + ((iy & 7) << 3) + (ix & 7);
#pragma unroll
      for (int k = 0; k < 8; ++k) c[k] = __ldg(b + (k & 1) + (((k >> 1) & 1) << 3) + ((k >> 2) << 6));
      return true;
    }
    bool any = false;
    long long last = -1;
    int s = -1;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int x = ix + (k & 1), y = iy + ((k >> 1) & 1), z = iz + (k >> 2);
      const long long b = brick(x, y, z);
      if (b != last) {
        last = b;
        s = find(b);
      }
      if (s >= 0 && (!flags || flags[s])) {  // else the voxel holds 1: c[k] stays
        c[k] = __ldg(sdf + (size_t)s * 512 + ((z & 7) << 6) + ((y & 7) << 3) + (x & 7));
        any = true;
      }
    }
    return any;
  }
  __device__ __forceinline__ float4 rgbw(int x, int y, int z) const {
    const int s = find(brick(x, y, z));
    if (s < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
    return __ldg(rgbw_p + (size_t)s * 512 + ((z & 7) << 6) + ((y & 7) << 3) + (x & 7));
  }
};

struct CandDev {
  unsigned long long* keys;  // [buckets], 0 = empty
  unsigned long long* list;  // [max]
  int* count;
  int log2n;
  unsigned long long mask;
  int max;
};

__device__ __forceinline__ void candidate_insert(const CandDev& c, unsigned long long b, int* state) {
  unsigned long long h = bucket_of(b, c.log2n);
  const unsigned long long k1 = b + 1ull;
  for (int p = 0; p < kMaxProbe; ++p) {
    // keys only ever change from 0 to their final value, so a stale read is
    // either that value or 0, which the CAS settles
    unsigned long long cur = c.keys[h];
    if (cur == k1) return;
    if (cur == 0ull) {
      cur = atomicCAS(c.keys + h, 0ull, k1);
      if (cur == 0ull) {
        const int i = atomicAdd(c.count, 1);
        if (i < c.max) c.list[i] = b;
        else set_status(state + 1, GPS_ERR_CAPACITY);
        return;
      }
      if (cur == k1) return;
    }
    h = (h + 1ull) & c.mask;
  }
  set_status(state + 1, GPS_ERR_CAPACITY);
}

// 1. candidate bricks of every pixel's band segment.  A voxel centre that
// projects to pixel (px, py) lies in the pixel's frustum, within
// sqrt((z / 2fx)^2 + (z / 2fy)^2) < 0.75 z / min(f) of the central ray at the
// same depth; the central ray is sampled every half brick, so every band
// voxel of the pixel is within 0.75 z_hi / min(f) + brick / 4 (+ one voxel of
// slack) of a sample, and the bricks meeting that box around each sample
// hold them all.
__global__ void __launch_bounds__(256) hash_candidates_kernel(HashDev h, Cam cam,
                                                              const float* __restrict__ depth,
                                                              CandDev c) {
  chain_wait();
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= cam.W * cam.H) return;
  const float D = __ldg(depth + pix);
  if (!(D > 0.0f)) return;
  const int px = pix % cam.W, py = pix / cam.W;
  const float dcx = ((float)px - cam.cx) / cam.fx, dcy = ((float)py - cam.cy) / cam.fy;
  float dw[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) dw[r] = cam.R[r * 3 + 0] * dcx + cam.R[r * 3 + 1] * dcy + cam.R[r * 3 + 2];
  const float len = sqrtf(dcx * dcx + dcy * dcy + 1.0f);  // 3D length per unit depth
  const float bsz = 8.0f * h.voxel;
  const float z_lo = fmaxf(D - h.trunc, 0.0f), z_hi = D + h.trunc;
  const float step = 0.5f * bsz / len;
  const int ns = (int)ceilf((z_hi - z_lo) / step) + 1;
  const float r = 0.75f * z_hi / fminf(cam.fx, cam.fy) + 0.25f * bsz + h.voxel;
  const int nb[3] = {h.nx >> 3, h.ny >> 3, h.nz >> 3};
  const float org[3] = {h.ox, h.oy, h.oz};
  for (int k = 0; k < ns; ++k) {
    const float z = fminf(z_lo + (float)k * step, z_hi);
    int lo[3], hi[3];
    bool out = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float p = cam.t[a] + z * dw[a] - org[a];
      lo[a] = max((int)floorf((p - r) / bsz), 0);
      hi[a] = min((int)floorf((p + r) / bsz), nb[a] - 1);
      out = out || lo[a] > hi[a];
    }
    if (out) continue;
    for (int bz = lo[2]; bz <= hi[2]; ++bz)
      for (int by = lo[1]; by <= hi[1]; ++by)
        for (int bx = lo[0]; bx <= hi[0]; ++bx)
          candidate_insert(c, ((unsigned long long)bz * nb[1] + by) * nb[0] + bx, h.state);
  }
}

// Coordinates (in bricks) of linear brick index b (x fastest).
__device__ __forceinline__ void brick_xyz(long long b, int nbx, int nby, int* out) {
  const long long q = b / nbx, r = q / nby;
  out[0] = (int)(b - q * nbx);
  out[1] = (int)(q - r * nby);
  out[2] = (int)r;
}

// 2. allocation: the exact band test on each candidate's voxels, then the
// table insert and the initialisation of new bricks.  One 512-thread CTA per
// candidate (grid-stride over the candidates).
__global__ void __launch_bounds__(512) hash_alloc_kernel(HashDev h, Cam cam,
                                                         const float* __restrict__ depth,
                                                         CandDev c) {
  chain_wait();
  __shared__ int s_slot, s_new, s_b[3];
  const int n = min(*c.count, c.max);
  const int local = threadIdx.x;
  for (int ci = blockIdx.x; ci < n; ci += gridDim.x) {
    const long long b = (long long)c.list[ci];
    // the brick's coordinates: 64-bit divisions, once per CTA
    __syncthreads();
    if (local == 0) brick_xyz(b, h.nx >> 3, h.ny >> 3, s_b);
    __syncthreads();
    const int bx = s_b[0], by = s_b[1], bz = s_b[2];
    const int x = (bx << 3) + (local & 7), y = (by << 3) + ((local >> 3) & 7),
              z = (bz << 3) + (local >> 6);
    float eta = 0.0f;
    const long long pix = voxel_pixel(h.voxel, h.ox, h.oy, h.oz, cam, depth, x, y, z, eta);
    const bool band = pix >= 0 && fabsf(eta) < h.trunc;
    if (!__syncthreads_or(band)) continue;
    if (local == 0) {
      int slot = -1, fresh = 0;
      bool done = false;
      unsigned long long hh = bucket_of((unsigned long long)b, h.log2n);
      const unsigned long long k1 = (unsigned long long)b + 1ull;
      for (int p = 0; p < kMaxProbe && !done; ++p) {
        unsigned long long cur = h.keys[hh];
        if (cur == 0ull) cur = atomicCAS(h.keys + hh, 0ull, k1);
        if (cur == 0ull) {  // inserted here
          slot = atomicAdd(h.state, 1);
          if (slot >= h.capacity) {
            set_status(h.state + 1, GPS_ERR_CAPACITY);
            slot = -1;
          } else {
            h.brick_of_slot[slot] = b;
            fresh = 1;
          }
          h.slots[hh] = slot;
          done = true;
        } else if (cur == k1) {  // stored by an earlier frame
          slot = h.slots[hh];
          done = true;
        } else {
          hh = (hh + 1ull) & h.mask;
        }
      }
      if (!done) set_status(h.state + 1, GPS_ERR_CAPACITY);
      s_slot = slot;
      s_new = fresh;
    }
    __syncthreads();
    if (s_new) {
      const size_t id = (size_t)s_slot * 512 + local;
      h.sdf[id] = 1.0f;
      h.weight[id] = 0.0f;
      h.rgbw_p[id] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (local == 0 && h.flags) h.flags[s_slot] = 0;
    }
    __syncthreads();  // s_slot / s_new are rewritten by the next candidate
  }
}

// 3. fusion of every allocated brick in view.  The cull is conservative: a
// brick is skipped only when its voxel centres' bounding box lies wholly
// behind the camera, or in front of it and projecting outside the image by
// more than a pixel; the per-voxel test then decides exactly as fuse_frame.
__global__ void __launch_bounds__(256) hash_fuse_kernel(HashDev h, const float* __restrict__ depth,
                                                        const float* __restrict__ rgb, Cam cam) {
  chain_wait();
  __shared__ int s_b[3];
  const int n = min(*h.state, h.capacity);
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    const long long b = h.brick_of_slot[s];
    // the brick's coordinates: 64-bit divisions, once per CTA
    __syncthreads();
    if (threadIdx.x == 0) brick_xyz(b, h.nx >> 3, h.ny >> 3, s_b);
    __syncthreads();
    const int bx = s_b[0], by = s_b[1], bz = s_b[2];
    int behind = 0, front = 0;
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float wx = h.ox + ((bx << 3) + ((k & 1) ? 7.5f : 0.5f)) * h.voxel;
      const float wy = h.oy + ((by << 3) + (((k >> 1) & 1) ? 7.5f : 0.5f)) * h.voxel;
      const float wz = h.oz + ((bz << 3) + ((k >> 2) ? 7.5f : 0.5f)) * h.voxel;
      float xc, yc, zc;
      world_to_cam(cam, wx, wy, wz, xc, yc, zc);
      if (zc > 0.0f) {
        ++front;
        const float u = cam.fx * xc / zc + cam.cx, v = cam.fy * yc / zc + cam.cy;
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
        vmin = fminf(vmin, v);
        vmax = fmaxf(vmax, v);
      } else {
        ++behind;
      }
    }
    if (behind == 8) continue;
    if (front == 8 && (umax < -1.5f || umin > (float)cam.W + 0.5f || vmax < -1.5f ||
                       vmin > (float)cam.H + 0.5f))
      continue;
    for (int local = threadIdx.x; local < 512; local += blockDim.x) {
      const int x = (bx << 3) + (local & 7), y = (by << 3) + ((local >> 3) & 7),
                z = (bz << 3) + (local >> 6);
      float eta;
      const long long pix = voxel_pixel(h.voxel, h.ox, h.oy, h.oz, cam, depth, x, y, z, eta);
      if (pix < 0 || eta < -h.trunc) continue;
      const float s1 = voxel_update(h.trunc, h.wmax, cam, rgb, pix, eta, h.sdf, h.weight,
                                    h.rgbw_p, (long long)s * 512 + local);
      if (h.flags && s1 != 1.0f) h.flags[s] = 1;
    }
  }
}

__global__ void __launch_bounds__(256) hash_to_dense_kernel(HashDev h, float* __restrict__ sdf,
                                                            float* __restrict__ weight,
                                                            float4* __restrict__ rgbw,
                                                            uint8_t* __restrict__ flags) {
  chain_wait();
  const int n = min(*h.state, h.capacity);
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    const long long b = h.brick_of_slot[s];
    bool nonunit = false;
    for (int local = threadIdx.x; local < 512; local += blockDim.x) {
      const size_t src = (size_t)s * 512 + local, dst = (size_t)b * 512 + local;
      const float v = h.sdf[src];
      sdf[dst] = v;
      weight[dst] = h.weight[src];
      rgbw[dst] = h.rgbw_p[src];
      nonunit = nonunit || v != 1.0f;
    }
    const int any = __syncthreads_or(nonunit);
    if (flags && threadIdx.x == 0 && any) flags[b] = 1;
  }
}

}  // namespace gps

// ------------------------------------------------------------------ C ABI
namespace gps {
void set_error(const char* msg);  // capi.cu: sets gps_last_error() of this thread
}

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int32_t hash_fail(int32_t code, const char* msg) {
  gps::set_error(msg);
  return code;
}

int log2_exact(long long n) {
  int l = 0;
  while ((1ll << l) < n) ++l;
  return (1ll << l) == n ? l : -1;
}

bool hash_ok(const GpsHashTsdf* v) {
  if (!v || !v->keys || !v->slots || !v->brick_of_slot || !v->state || !v->sdf || !v->weight ||
      !v->rgbw)
    return false;
  const int lim = 1 << 21;
  if (v->nx <= 0 || v->ny <= 0 || v->nz <= 0 || (v->nx & 7) || (v->ny & 7) || (v->nz & 7) ||
      v->nx >= lim || v->ny >= lim || v->nz >= lim)
    return false;
  if (!(v->voxel > 0) || !(v->trunc > 0) || !(v->max_weight >= 1) || v->capacity <= 0 ||
      v->n_buckets < 2 || log2_exact(v->n_buckets) < 0)
    return false;
  return (reinterpret_cast<uintptr_t>(v->rgbw) & 15) == 0;
}

gps::HashDev hash_dev(const GpsHashTsdf& v) {
  gps::HashDev h{};
  h.nx = v.nx;
  h.ny = v.ny;
  h.nz = v.nz;
  h.voxel = v.voxel;
  h.ox = v.origin[0];
  h.oy = v.origin[1];
  h.oz = v.origin[2];
  h.trunc = v.trunc;
  h.wmax = v.max_weight;
  h.log2n = log2_exact(v.n_buckets);
  h.mask = (unsigned long long)v.n_buckets - 1ull;
  h.capacity = v.capacity;
  h.keys = reinterpret_cast<unsigned long long*>(v.keys);
  h.slots = v.slots;
  h.brick_of_slot = reinterpret_cast<long long*>(v.brick_of_slot);
  h.state = v.state;
  h.sdf = v.sdf;
  h.weight = v.weight;
  h.rgbw_p = reinterpret_cast<float4*>(v.rgbw);
  h.flags = v.slot_flags;
  return h;
}

struct CandLayout {
  size_t keys, list, count, total;
  long long buckets;
};

CandLayout cand_layout(int max_candidates) {
  CandLayout L{};
  long long b = 2;
  while (b < 2ll * max_candidates) b <<= 1;
  L.buckets = b;
  size_t off = 0;
  L.keys = off; off = a256(off + (size_t)b * 8);
  L.list = off; off = a256(off + (size_t)max_candidates * 8);
  L.count = off; off = a256(off + 4);
  L.total = off;
  return L;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
  }
  return n;
}

bool cam_ok(const GpsIntrinsics* K, const GpsPose* P) {
  if (!K || !P || K->width <= 0 || K->height <= 0 || !(K->fx > 0) || !(K->fy > 0)) return false;
  bool ok = std::isfinite(K->cx) && std::isfinite(K->cy);
  for (int k = 0; k < 9; ++k) ok = ok && std::isfinite(P->R[k]);
  for (int k = 0; k < 3; ++k) ok = ok && std::isfinite(P->t[k]);
  return ok;
}

}  // namespace

extern "C" {

int32_t gps_hash_scratch_size(int32_t max_candidates, size_t* bytes) {
  if (!bytes || max_candidates <= 0)
    return hash_fail(GPS_ERR_INVALID_ARG, "gps_hash_scratch_size: bad arguments");
  *bytes = cand_layout(max_candidates).total;
  return GPS_OK;
}

int32_t fuse_frame_hashed(GpsHashTsdf* vol, const float* depth, const float* rgb,
                          const GpsIntrinsics* K, const GpsPose* T_wc, void* scratch,
                          size_t scratch_bytes, int32_t max_candidates, void* stream) {
  if (!hash_ok(vol) || !depth || !rgb || !scratch || !cam_ok(K, T_wc) || max_candidates <= 0)
    return hash_fail(GPS_ERR_INVALID_ARG, "fuse_frame_hashed: bad volume, camera or arguments");
  const CandLayout L = cand_layout(max_candidates);
  if (scratch_bytes < L.total || (reinterpret_cast<uintptr_t>(scratch) & 255))
    return hash_fail(GPS_ERR_WORKSPACE_TOO_SMALL,
                     "fuse_frame_hashed: scratch smaller than gps_hash_scratch_size or unaligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* b = static_cast<char*>(scratch);
  gps::CandDev c{};
  c.keys = reinterpret_cast<unsigned long long*>(b + L.keys);
  c.list = reinterpret_cast<unsigned long long*>(b + L.list);
  c.count = reinterpret_cast<int*>(b + L.count);
  c.log2n = log2_exact(L.buckets);
  c.mask = (unsigned long long)L.buckets - 1ull;
  c.max = max_candidates;
  cudaError_t e = cudaMemsetAsync(b, 0, L.keys + (size_t)L.buckets * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.count, 0, 4, st);
  const gps::HashDev h = hash_dev(*vol);
  const gps::Cam cam = gps::make_cam(*K, *T_wc);
  const long long npx = (long long)K->width * K->height;
  if (e == cudaSuccess) {
    gps::launch_chained(gps::hash_candidates_kernel, dim3((unsigned)((npx + 255) / 256)),
                        dim3(256), 0, st, h, cam, depth, c);
    gps::launch_chained(gps::hash_alloc_kernel, dim3(4 * sm_count()), dim3(512), 0, st, h, cam,
                        depth, c);
    gps::launch_chained(gps::hash_fuse_kernel, dim3(8 * sm_count()), dim3(256), 0, st, h, depth,
                        rgb, cam);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return hash_fail(GPS_ERR_CUDA, cudaGetErrorString(e));
  return GPS_OK;
}

int32_t raycast_sdf_hashed(const GpsHashTsdf* vol, const GpsIntrinsics* K, const GpsPose* T_wc,
                           float near_plane, float far_plane, void* out_rgb, int32_t rgb_precision,
                           float* out_depth, float* out_vertex, void* stream) {
  if (!hash_ok(vol) || !cam_ok(K, T_wc) || !out_rgb || !out_depth || !(near_plane >= 0) ||
      (rgb_precision != GPS_PREC_FP32 && rgb_precision != GPS_PREC_FP16 &&
       rgb_precision != GPS_PREC_BF16))
    return hash_fail(GPS_ERR_INVALID_ARG, "raycast_sdf_hashed: bad volume, camera or outputs");
  const gps::HashDev h = hash_dev(*vol);
  const gps::Cam cam = gps::make_cam(*K, *T_wc);
  dim3 grid((K->width + 15) / 16, (K->height + 15) / 16);
  gps::launch_chained(gps::raycast_kernel<gps::HashDev>, grid, dim3(256), 0,
                      static_cast<cudaStream_t>(stream), h, cam, near_plane, far_plane, out_rgb,
                      rgb_precision, out_depth, out_vertex);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hash_fail(GPS_ERR_CUDA, cudaGetErrorString(e));
  return GPS_OK;
}

int32_t tsdf_hash_to_dense(const GpsHashTsdf* vol, GpsTsdf* dense, void* stream) {
  if (!hash_ok(vol) || !dense || !dense->sdf || !dense->weight || !dense->rgbw ||
      dense->nx != vol->nx || dense->ny != vol->ny || dense->nz != vol->nz)
    return hash_fail(GPS_ERR_INVALID_ARG, "tsdf_hash_to_dense: bad volumes or sizes differ");
  const gps::HashDev h = hash_dev(*vol);
  gps::launch_chained(gps::hash_to_dense_kernel, dim3(8 * sm_count()), dim3(256), 0,
                      static_cast<cudaStream_t>(stream), h, dense->sdf, dense->weight,
                      reinterpret_cast<float4*>(dense->rgbw), dense->brick_flags);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hash_fail(GPS_ERR_CUDA, cudaGetErrorString(e));
  return GPS_OK;
}

}  // extern "C"
