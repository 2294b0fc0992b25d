// Shared device helpers of libgps (sm_103a).  Internal header.
#pragma once
#include <cstdint>
#include <utility>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/gps.h"

namespace gps {

constexpr int kRecFloats = 16;    // projected record, see GpsWorkspaceLayout
constexpr int kGrad2d = 12;       // per-Gaussian 2D gradient slots
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kExtRel = 1.0f + 0.0078125f;  // 1 + 2^-7: conservative extent
constexpr float kExtAbs = 0.0625f;             // 2^-4 px
constexpr float kAlphaMax = 0.99f;             // Table 7 variant (3DGS clamp)
constexpr float kTMin = 1e-4f;                 // Table 7 variant termination
// Binning super-tiles are 16 x 16 px (32 x 32 px for 32-px-wide tiles):
// log2 of their edge for a tile width.
__host__ __device__ constexpr int super_shift_for(int tw) { return tw > 16 ? 5 : 4; }

// grad2d slot names
enum { G_MX = 0, G_MY, G_CA, G_CB, G_CC, G_SIG, G_R, G_G, G_B, G_D };

struct Cam {
  float fx, fy, cx, cy;
  int W, H;
  float R[9];  // camera -> world
  float t[3];
};

// Device camera from the ABI's intrinsics and pose.
inline Cam make_cam(const GpsIntrinsics& K, const GpsPose& P) {
  Cam c;
  c.fx = K.fx; c.fy = K.fy; c.cx = K.cx; c.cy = K.cy;
  c.W = K.width; c.H = K.height;
  for (int k = 0; k < 9; ++k) c.R[k] = P.R[k];
  for (int k = 0; k < 3; ++k) c.t[k] = P.t[k];
  return c;
}

// Per-view device-side description (passed by value to kernels).
struct ViewDev {
  Cam cam;
  const void* Ct;     // [3][H][W], element type per `prec`
  const float* Dt;    // [H][W]
  const void* Ctgt;   // nullable, element type per `prec`
  const float* Dtgt;  // nullable
  void* out_rgb;      // nullable, element type per `prec`
  float* out_depth;
  float* out_weight;
  const float* g_rgb;    // nullable
  const float* g_depth;  // nullable
  // workspace regions
  float4* rec;           // [M][4] float4
  uint32_t* sup_count;   // [nsup]
  uint32_t* block_base;  // [bin_blocks(M)][nsup]
  uint2* sup_ranges;     // [nsup]
  unsigned long long* sup_keys;
  unsigned long long* sup_tmp;
  uint2* tile_ranges;    // [tiles]
  unsigned long long* keys;  // tile lists
  float4* pix_a;  // [npx] (C*.rgb, D*)
  float4* pix_b;  // [npx] (W_G | T_end, n_last, -, -)
  float4* tile_partials;  // [tiles] (sum|dC|, sum|dD|, n_valid, -)
  float* scalars;         // [8]
  float4* grad2d;         // [M][3] float4
  float4* pair_grads;     // [pair_slots][3] float4, Gaussian-major (deterministic mode)
  uint32_t* pair_base;    // [M] first slot of each Gaussian (deterministic mode)
  long long pair_slots;
  float4* pix_g;          // [npx][2] per-Gaussian backward: (h), (sv, thr, -, -)
  int* tile_order;        // [tiles] longest lists first (by their bin's entry count)
  long long* grad_fixed;  // [M][10] fixed-point 2D gradient sums (deterministic OIT), else null
  int tiles_x, tiles_y, tw, th;
  // bins of the binning pass (sup_x * sup_y of them, 2^bin_sx x 2^bin_sy
  // pixels each): square super-tiles, or the tiles themselves
  int sup_x, sup_y, bin_sx, bin_sy;
  // the bins' lists in ascending Gaussian index, placed without atomics
  // (deterministic mode, OIT blend, tile bins; see emit_super_kernel)
  int fixed_order;
  int tile_bin;  // the bins are the tiles (else super-tiles, sorted and split)
  int sorted;    // the tile lists are sorted by (depth, index)
  int fused;  // backward: upstream gradients from the fused L1 loss (1) or g_rgb/g_depth (0)
  int prec;   // GPS_PREC_* storage type of the colour images Ct, Ctgt, out_rgb
  long long cap;
};

// Views rendered by one launch per stage.  Work items of the per-tile and
// per-super-tile kernels are numbered view after view in `order` (largest
// views first, so that the small views' tiles fill the tail of the grid);
// view order[k] owns items [tile_start[k], tile_start[k + 1]).  Passed to the
// kernels by value as a __grid_constant__ parameter (about 2.6 KB).
constexpr int kMaxBatch = 8;
struct ViewBatch {
  int n;
  int order[kMaxBatch];
  int tile_start[kMaxBatch + 1];
  int sup_start[kMaxBatch + 1];
  ViewDev v[kMaxBatch];
};

// Position k in `order` of the view owning work item `item` (n <= kMaxBatch).
__device__ __forceinline__ int batch_slot(const int* start, int n, int item) {
  int k = 0;
#pragma unroll 1
  while (k + 1 < n && item >= start[k + 1]) ++k;
  return k;
}

// The tile of a view's per-tile work item: its tiles are taken in order of
// decreasing list length (the binning's tile_order), so that the longest
// lists start first and the grid's tail holds short ones.  An entry outside
// the tile grid (a workspace that no binning pass has written) falls back to
// the item's own tile.
__device__ __forceinline__ int tile_of(const ViewDev& v, int item) {
  if (!v.tile_order) return item;
  const int t = __ldg(v.tile_order + item);
  return (unsigned)t < (unsigned)(v.tiles_x * v.tiles_y) ? t : item;
}

// Colour images are stored as float, IEEE binary16 or bfloat16 (GPS_PREC_*);
// every value is converted to float on load and rounded to nearest-even on
// store.
__device__ __forceinline__ float ld_col(const void* p, long long i, int prec) {
  if (prec == GPS_PREC_FP16) return __half2float(static_cast<const __half*>(p)[i]);
  if (prec == GPS_PREC_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
  return __ldg(static_cast<const float*>(p) + i);
}
__device__ __forceinline__ void st_col(void* p, long long i, int prec, float x) {
  if (prec == GPS_PREC_FP16) static_cast<__half*>(p)[i] = __float2half_rn(x);
  else if (prec == GPS_PREC_BF16) static_cast<__nv_bfloat16*>(p)[i] = __float2bfloat16_rn(x);
  else static_cast<float*>(p)[i] = x;
}

// Pixel rectangle of a record, clipped to the image: [x0, x1] x [y0, y1].
// Float arithmetic spelled out so that the oracle can reproduce it bit for bit.
__device__ __forceinline__ bool record_rect(float mx, float my, float ex, float ey, int W, int H,
                                            int& x0, int& x1, int& y0, int& y1) {
  if (!(ex >= 0.0f) || !(ey >= 0.0f)) return false;
  const float lx = __fsub_rn(mx, ex), hx = __fadd_rn(mx, ex);
  const float ly = __fsub_rn(my, ey), hy = __fadd_rn(my, ey);
  if (!(hx >= 0.0f) || !(lx <= (float)(W - 1)) || !(hy >= 0.0f) || !(ly <= (float)(H - 1)))
    return false;
  x0 = max(0, (int)ceilf(fmaxf(lx, -1.0f)));
  x1 = min(W - 1, (int)floorf(fminf(hx, (float)W)));
  y0 = max(0, (int)ceilf(fmaxf(ly, -1.0f)));
  y1 = min(H - 1, (int)floorf(fminf(hy, (float)H)));
  return x0 <= x1 && y0 <= y1;
}

// Deterministic OIT backward (fixed-point gradient sums, composite.cu): the
// part of a Gaussian's quantum exponents that depends on its record alone,
// written by the projection into the record's spare words 13 and 14 (float
// 12 is ey).  The bounds on a (warp block, Gaussian) partial of each
// component k factor as c_k x V (k < 6; V the view's bound on |dL/dalpha|
// terms) or c_k x hmax (k >= 6) with
//   c_0 = 64 (|a| ex + |b| ey), c_1 = 64 (|b| ex + |c| ey), c_2 = 32 ex^2,
//   c_3 = 64 ex ey, c_4 = 32 ey^2, c_5 = c_6.. = 64
// (conic a, b, c; extents ex, ey).  With n partials at most (tiles of the
// rectangle x warp blocks per tile), the quantum exponent is
// x(c_k) + x(V or hmax) - (62 - ceil(log2 n)), x(b) = the least integer
// with b < 2^x (fixed_expo_above); the first and last terms are the
// pre-exponent p_k, stored as p_k + 128 in a byte (clamped to [0, 255]:
// raising p only coarsens the quantum).  Word 13: p_0..p_3; word 14: p_4,
// p_5 (= p_6..p_9), 0, kFixedPreTag (records written otherwise lack the tag
// and have the pre-exponents recomputed by whoever reads them).
constexpr uint32_t kFixedPreTag = 0x5Au;

// The least x >= -126 with b < 2^x, for b >= 0 (b >= 2^128, inf or NaN -> 129).
__device__ __forceinline__ int fixed_expo_above(float b) {
  const int E = (int)((__float_as_uint(b) >> 23) & 0xffu);
  return E == 0 ? -126 : E - 126;
}

__device__ __forceinline__ uint2 fixed_pre_exponents(float mx, float my, float ca, float cb,
                                                     float cc, float ex, float ey, int W, int H,
                                                     int tw, int th) {
  int n = 1, x0, x1, y0, y1;
  if (record_rect(mx, my, ex, ey, W, H, x0, x1, y0, y1))
    n = (x1 / tw - x0 / tw + 1) * (y1 / th - y0 / th + 1) * (tw * th / 32);
  const int off = (n > 1 ? 32 - __clz(n - 1) : 0) - 62 + 128;  // ceil(log2 n) - 62, biased
  // explicit roundings: every reader of an untagged record gets the same bits
  const float ax = fabsf(ex), ay = fabsf(ey);
  float c[5];
  c[0] = __fmul_rn(64.0f, __fmaf_rn(fabsf(ca), ax, __fmul_rn(fabsf(cb), ay)));
  c[1] = __fmul_rn(64.0f, __fmaf_rn(fabsf(cb), ax, __fmul_rn(fabsf(cc), ay)));
  c[2] = __fmul_rn(__fmul_rn(32.0f, ax), ax);
  c[3] = __fmul_rn(__fmul_rn(64.0f, ax), ay);
  c[4] = __fmul_rn(__fmul_rn(32.0f, ay), ay);
  uint32_t b[6];
#pragma unroll
  for (int k = 0; k < 5; ++k) b[k] = (uint32_t)min(max(fixed_expo_above(c[k]) + off, 0), 255);
  b[5] = (uint32_t)min(max(7 + off, 0), 255);  // x(64) = 7
  return make_uint2(b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24),
                    b[4] | (b[5] << 8) | (kFixedPreTag << 24));
}

__device__ __forceinline__ bool fixed_pre_tagged(uint32_t w14) { return (w14 >> 24) == kFixedPreTag; }

// Quantum exponents are clamped to [-120, 126] so that 2^-e and 2^e are
// normal floats (composite.cu derives the bounds behind them).
constexpr int kFixedEMin = -120, kFixedEMax = 126;

__device__ __forceinline__ int fixed_clamp_e(int e) { return min(max(e, kFixedEMin), kFixedEMax); }

// The quantum exponents of a Gaussian's ten components from its packed
// pre-exponents and the bounds V (components 0-5) and hmax (6-9).
__device__ __forceinline__ int fixed_pre_byte(uint32_t w, int k) {
  return (int)__byte_perm(w, 0u, 0x4440u + (uint32_t)k);  // byte k, zero-extended
}
__device__ __forceinline__ void fixed_exponents(uint2 pre, float V, float hm, int (&e)[10]) {
  const int xv = fixed_expo_above(V) - 128, xh = fixed_expo_above(hm) - 128;
#pragma unroll
  for (int k = 0; k < 4; ++k) e[k] = fixed_clamp_e(fixed_pre_byte(pre.x, k) + xv);
  e[4] = fixed_clamp_e(fixed_pre_byte(pre.y, 0) + xv);
  const int p5 = fixed_pre_byte(pre.y, 1);
  e[5] = fixed_clamp_e(p5 + xv);
  e[6] = e[7] = e[8] = e[9] = fixed_clamp_e(p5 + xh);
}

// The view's upstream bounds: with the fused L1 loss the forward's loss
// finalisation left them per unit dL/dloss in scalars[6..7] (scaled here by
// |dL/dloss|), with explicit upstream images upstream_max_kernel left the
// maxima themselves.
__device__ __forceinline__ void fixed_maxima(const ViewDev& v, const float* dloss, float& hm,
                                             float& sm) {
  const float f = v.fused && dloss ? fabsf(*dloss) : 1.0f;
  hm = __fmul_rn(v.scalars[6], f);
  sm = __fmul_rn(v.scalars[7], f);
}

// V = hmax (|r| + |g| + |b| + |d|) + smax, explicitly rounded (the walk and
// the conversion back compute it from the same record values).
__device__ __forceinline__ float fixed_v(float hm, float sm, float cr, float cg, float cb,
                                         float d) {
  return __fmaf_rn(hm, __fadd_rn(__fadd_rn(fabsf(cr), fabsf(cg)), __fadd_rn(fabsf(cb), fabsf(d))),
                   sm);
}

// A Gaussian's packed pre-exponents: from the record's words 13-14 where the
// projection wrote them, else recomputed from the record.
__device__ __forceinline__ uint2 fixed_pre(const ViewDev& v, const float4& E, float mx, float my,
                                           float ca, float cb, float cc, const float* ex_p) {
  const uint2 pre = make_uint2(__float_as_uint(E.y), __float_as_uint(E.z));
  if (fixed_pre_tagged(pre.y)) return pre;
  return fixed_pre_exponents(mx, my, ca, cb, cc, __ldg(ex_p), E.x, v.cam.W, v.cam.H, v.tw, v.th);
}

// A Gaussian's 2D gradient from its fixed-point sums: one rounding of each
// integer sum, then the exact power-of-two scale 2^e (the exponents
// recomputed from the record, as the backward walk computed them).
// ga = d/d(mx, my, conic a, conic b), gb = (conic c, sigma, r, g),
// gc = (b, depth, 0, 0), the layout of grad2d.
__device__ __forceinline__ void fixed_grad2d(const ViewDev& v, int i, const float* dloss,
                                             float4& ga, float4& gb, float4& gc) {
  const float4* rr = v.rec + 4 * (size_t)i;
  const float4 A = rr[0], C = rr[2];
  const uint2 pre = fixed_pre(v, rr[3], A.x, A.y, rr[1].x, rr[1].y, rr[1].z, &rr[2].w);
  float hm, sm;
  fixed_maxima(v, dloss, hm, sm);
  int e[10];
  fixed_exponents(pre, fixed_v(hm, sm, C.x, C.y, C.z, A.z), hm, e);
  const longlong2* s = reinterpret_cast<const longlong2*>(v.grad_fixed + 10 * (size_t)i);
  float g[10];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const longlong2 t = s[k];
    g[2 * k] = __fmul_rn(__ll2float_rn(t.x), __int_as_float((127 + e[2 * k]) << 23));
    g[2 * k + 1] = __fmul_rn(__ll2float_rn(t.y), __int_as_float((127 + e[2 * k + 1]) << 23));
  }
  ga = make_float4(g[0], g[1], g[2], g[3]);
  gb = make_float4(g[4], g[5], g[6], g[7]);
  gc = make_float4(g[8], g[9], 0.f, 0.f);
}

// q = dx (a dx + 2b dy) + (c dy) dy with explicit roundings (identical on the
// oracle's FP32 decision path).  b2 = 2 b.
__device__ __forceinline__ float quad_form(float a, float b2, float c, float dx, float dy) {
  const float s2 = __fmaf_rn(a, dx, __fmul_rn(b2, dy));
  const float s3 = __fmul_rn(__fmul_rn(c, dy), dy);
  return __fmaf_rn(dx, s2, s3);
}

__device__ __forceinline__ float depth_threshold(float Dt, float eps) {
  return Dt > 0.0f ? __fadd_rn(Dt, eps) : __int_as_float(0x7f800000);
}

__device__ __forceinline__ unsigned long long key_of(float d, uint32_t idx) {
  return ((unsigned long long)__float_as_uint(d) << 32) | idx;
}

// Binning CTAs take bin_chunks(M) consecutive chunks of 256 Gaussians each,
// and one range per (CTA, bin) is reserved.  Every CTA stages a word per bin,
// so CTAs should be few, but enough to fill the 148 SMs: about 600 (four per
// SM) once M passes 600 * 256, at most 8 chunks per CTA.
__host__ __device__ constexpr int bin_chunks(int M) {
  return M / (256 * 600) < 1 ? 1 : (M / (256 * 600) > 8 ? 8 : M / (256 * 600));
}
__host__ __device__ constexpr int bin_blocks(int M) {
  return (M + 256 * bin_chunks(M) - 1) / (256 * bin_chunks(M));
}

// Binning: after every thread of the block has added its Gaussians' super-tiles
// to the shared histogram s_hist, reserve one range per nonzero super-tile with
// one global atomic; the block's base inside super-tile s goes to
// block_base[block][s].  With fixed_order the block writes its counts there
// instead, and block_prefix_kernel turns them into bases in block order.
__device__ __forceinline__ void reserve_block_ranges(uint32_t* s_hist, int nsup,
                                                     uint32_t* __restrict__ sup_count,
                                                     uint32_t* __restrict__ block_base,
                                                     int fixed_order) {
  __syncthreads();
  if (fixed_order) {
    for (int s = threadIdx.x; s < nsup; s += blockDim.x)
      block_base[(size_t)blockIdx.x * nsup + s] = s_hist[s];
    return;
  }
  // eight bins per thread in flight: the atomics' round trips overlap
  constexpr int U = 8;
  for (int s0 = threadIdx.x; s0 < nsup; s0 += U * blockDim.x) {
    uint32_t base[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + u * blockDim.x;
      const uint32_t h = s < nsup ? s_hist[s] : 0u;
      base[u] = h ? atomicAdd(sup_count + s, h) : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + u * blockDim.x;
      if (s < nsup) block_base[(size_t)blockIdx.x * nsup + s] = base[u];
    }
  }
}

// Programmatic dependent launch.  The kernels of one iteration (projection,
// binning, composites, loss, backward passes, Adam) are launched with
// launch_chained, so that a kernel's launch is processed while its
// predecessor on the stream completes, and every such kernel starts with
// chain_wait(): it waits (griddepcontrol.wait) until the predecessor has
// completed and its memory is visible, before reading anything.  No kernel
// triggers its dependents early (griddepcontrol.launch_dependents at CTA
// start measured 1.4% slower per iteration in CUDA graphs: the waiting CTAs
// held SM slots); outside a programmatic dependency the wait does nothing.
__device__ __forceinline__ void chain_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                           cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// status word helpers
__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, 0, code); }

}  // namespace gps
