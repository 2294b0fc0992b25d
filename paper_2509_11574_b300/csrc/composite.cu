// Second rendering pass, hybrid blend, fused L1 loss and their adjoints.
//
// Forward (Eq. 1-4; Table 7 variant): one CTA per tile, one thread per pixel.
// Each tile's Gaussian list is sorted by depth, so the list is cut once at the
// first Gaussian at or behind max over the tile of D_t + eps (every pixel would
// cull it and all that follow), and each warp leaves a staged batch as soon as
// the next Gaussian is at or behind its own pixels' maximum threshold.  Batches
// of records are staged in shared memory and read as broadcasts.
//
// Backward, order-independent mode: the adjoint of Eq. 4 needs only per-pixel
// final values (N = 1 + W_G, C*, D*), not the order of the Gaussians, so the
// CTA transposes the work: each lane owns one Gaussian of the tile list and
// walks the tile's pixels (staged in shared memory, read as broadcasts),
// accumulating its 10 gradient terms privately - no shuffles.  One vector
// atomic per (tile, Gaussian) pair, or a plain store into the pair's slot in
// deterministic mode.
//
// Backward, alpha mode: per-pixel reverse walk of the list with the
// transmittance recomputed by division from the stored T_end, warp-shuffle
// reduction of each Gaussian's terms, then one shared-memory partial per warp.
#include <cuda_runtime.h>

#include "gps_common.cuh"

namespace gps {

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_min_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Instrumented runs: evaluation counters in the view scalars (uint64 after 8 floats).
__device__ __forceinline__ void add_counters(const ViewDev& v, int slot, unsigned tested,
                                             unsigned counted) {
  unsigned long long a = tested, b = counted;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    unsigned long long* c = reinterpret_cast<unsigned long long*>(v.scalars + 8);
    atomicAdd(c + slot, a);
    atomicAdd(c + slot + 1, b);
  }
}

// First position in [lo, hi) whose depth bits are >= bits(thr); thr > 0.
__device__ __forceinline__ uint32_t depth_cut(const unsigned long long* __restrict__ keys,
                                              uint32_t lo, uint32_t hi, float thr) {
  if (!(thr > 0.0f)) return lo;
  const uint32_t tb = __float_as_uint(thr);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((uint32_t)(keys[mid] >> 32) < tb) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The same cut computed by the whole CTA in two rounds of independent loads
// (a binary search is a chain of dependent ones): round 1 samples every
// step-th key, round 2 scans the one step that holds the cut.  All NT threads
// call it; lists longer than NT^2 fall back to the binary search.
template <int NT>
__device__ __forceinline__ uint32_t depth_cut_block(const unsigned long long* __restrict__ keys,
                                                   uint32_t lo, uint32_t hi, float thr) {
  const uint32_t n = hi - lo;
  if (!(thr > 0.0f) || n == 0) return lo;
  if (n > (uint32_t)NT * NT) return depth_cut(keys, lo, hi, thr);
  const uint32_t tb = __float_as_uint(thr);
  const uint32_t step = (n + NT - 1) / NT;
  const uint32_t p1 = lo + threadIdx.x * step;
  const bool below1 = p1 < hi && (uint32_t)(keys[p1] >> 32) < tb;
  const uint32_t c1 = (uint32_t)__syncthreads_count(below1);  // samples before the cut
  if (c1 == 0) return lo;
  const uint32_t a = lo + (c1 - 1) * step + 1, b = min(hi, lo + c1 * step);
  const uint32_t p2 = a + threadIdx.x;
  const bool below2 = p2 < b && (uint32_t)(keys[p2] >> 32) < tb;
  return a + (uint32_t)__syncthreads_count(below2);
}

template <int NT>
__device__ __forceinline__ float block_max(float v, float* s_tmp) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) s_tmp[w] = v;
  __syncthreads();
  float r = s_tmp[0];
#pragma unroll
  for (int k = 1; k < NT / 32; ++k) r = fmaxf(r, s_tmp[k]);
  return r;
}

// alpha = sigma exp(-q / 2) = 2^(log2(sigma) - q log2(e) / 2): one FMA on the
// staged log2(sigma) and the hardware base-2 exponential (ex2.approx, relative
// error about 2^-22, far inside the 1e-4 parity tolerance).  The counting
// decision never looks at alpha: it is taken on q.
constexpr float kHalfLog2e = 0.72134752044448170368f;  // log2(e) / 2
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float alpha_of(float q, float log2_sigma) {
  return ex2_approx(fmaf(q, -kHalfLog2e, log2_sigma));
}

// 1 / x by the hardware reciprocal (rcp.approx, within 1 ulp over the whole
// range): the alpha backward's 1 / (1 - alpha) with 1 - alpha in [0.01, 1].
// The correctly rounded rcp.rn took about 15 instructions with two branches
// against one here.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Does the support {q <= qmax} of a Gaussian centred at (mx, my) meet the
// rectangle [x0, x1] x [y0, y1]?  The minimum of the convex quadratic q over
// the rectangle is 0 if the centre lies inside, else it lies on an edge, at
// the stationary point of the edge's 1D quadratic clamped to the edge.
// Conservative (relative 1e-2 and absolute 1e-2 slack over FP32 rounding):
// used only to skip work, never to decide whether a pixel counts.
__device__ __forceinline__ bool ellipse_meets_rect(float mx, float my, float a, float b, float c,
                                                   float qmax, float x0, float x1, float y0,
                                                   float y1) {
  const float lx = x0 - mx, hx = x1 - mx, ly = y0 - my, hy = y1 - my;
  if (lx <= 0.f && hx >= 0.f && ly <= 0.f && hy >= 0.f) return true;
  float qmin = INFINITY;
  // approximate reciprocals: they only place the stationary point, and q there
  // is flat in the placement (error second order, inside the slack below)
  const float ic = __fdividef(1.0f, c), ia = __fdividef(1.0f, a);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float dx = e ? hx : lx;
    const float dy = fminf(fmaxf(-b * dx * ic, ly), hy);
    qmin = fminf(qmin, a * dx * dx + 2.0f * b * dx * dy + c * dy * dy);
    const float ey = e ? hy : ly;
    const float ex = fminf(fmaxf(-b * ey * ia, lx), hx);
    qmin = fminf(qmin, a * ex * ex + 2.0f * b * ex * ey + c * ey * ey);
  }
  return qmin <= qmax * 1.01f + 0.01f;
}

// ------------------------------------------------------------------ forward
// (the backward kernels' layout) Warp w covers the 8 x 4 pixel block
// (w % (TW/8), w / (TW/8)) of the tile, lane l its pixel (l % 8, l / 8).
template <int TW>
__device__ __forceinline__ void warp_block(int warp, int lane, int& ox, int& oy, int& lx, int& ly) {
  constexpr int BX = TW / 8;
  ox = (warp % BX) * 8;
  oy = (warp / BX) * 4;
  lx = ox + (lane & 7);
  ly = oy + (lane >> 3);
}

// OIT forward (Eq. 1-4) with two pixels per lane.  One CTA per tile; warp w
// covers the 8 x 8 pixel block (w % (TW/8), w / (TW/8)) of the tile, lane l
// the pixels (2 (l % 4), l / 4) and (2 (l % 4) + 1, l / 4) of it.  Per batch
// of staged records each warp compacts, 32 at a time with ballots, the
// Gaussians whose conservative rectangle meets its block and that lie in
// front of its largest depth threshold, then walks them with broadcast
// reads.  Each staged record is read once for both pixels of a lane, which
// share the dy terms of q.  Branch-free: a pixel where a Gaussian does not
// count adds alpha = 0 (exactly the same sums), so the warp never splits on
// the decision.
template <int TW, int TH, bool INSTR>
__global__ void __launch_bounds__(TW* TH / 2) composite_fwd_oit2_kernel(
    const __grid_constant__ ViewBatch vb, float eps, int has_tgt, int sorted) {
  chain_wait();
  constexpr int NTT = TW * TH / 2;  // threads
  constexpr int NW = NTT / 32;
  constexpr int NB = 2 * NTT;       // staged entries per batch
  constexpr int BX = TW / 8;
  __shared__ float4 s_a[NB], s_b[NB], s_c[NB];
  __shared__ float2 s_e[NB];
  __shared__ uint8_t s_list[NW][NB];
  __shared__ float s_tmp[NW * 4];
  const int slot = batch_slot(vb.tile_start, vb.n, blockIdx.x);
  const ViewDev& v = vb.v[vb.order[slot]];
  const int tile = tile_of(v, blockIdx.x - vb.tile_start[slot]);
  const int W = v.cam.W, H = v.cam.H;
  const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ox = (warp % BX) * 8, oy = (warp / BX) * 8;
  // lane (c, r) = (lane & 3, lane >> 2) owns pixels (2c, r) and (2c + 1, r)
  // of the warp's 8 x 8 block: one row, so the dy terms of q are shared
  const int px0 = tx * TW + ox + 2 * (lane & 3), px1 = px0 + 1;
  const int py = ty * TH + oy + (lane >> 2);
  const bool in0 = px0 < W && py < H, in1 = px1 < W && py < H;
  const long long npx = (long long)W * H;
  const long long pix0 = (long long)py * W + px0, pix1 = pix0 + 1;
  // C_t is read only at the end (fewer live registers in the list walk)
  float dt[2] = {0.f, 0.f};
  if (in0) dt[0] = __ldg(v.Dt + pix0);
  if (in1) dt[1] = __ldg(v.Dt + pix1);
  const float thr0 = in0 ? depth_threshold(dt[0], eps) : -INFINITY;
  const float thr1 = in1 ? depth_threshold(dt[1], eps) : -INFINITY;
  const uint2 r = v.tile_ranges[tile];
  uint32_t gi_next0 = r.x + tid < r.y ? (uint32_t)v.keys[r.x + tid] : 0u;
  uint32_t gi_next1 = r.x + NTT + tid < r.y ? (uint32_t)v.keys[r.x + NTT + tid] : 0u;
  const float wthr = warp_max(fmaxf(thr0, thr1));
  const float bthr = block_max<NTT>(fmaxf(thr0, thr1), s_tmp);
  // sorted lists end at the first Gaussian behind every pixel of the tile; an
  // unsorted list (per-Gaussian schedule) is walked to its end
  const bool srt = sorted && v.sorted;  // this view's lists are depth-sorted
  const uint32_t end = srt ? depth_cut_block<NTT>(v.keys, r.x, r.y, bthr) : r.y;
  const float bx0 = (float)(tx * TW + ox), bx1 = bx0 + 7.0f;
  const float by0 = (float)(ty * TH + oy), by1 = by0 + 7.0f;
  const float fpx0 = (float)px0, fpx1 = (float)px1, fpy = (float)py;
  float acc[2][5] = {{0.f, 0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f, 0.f}};  // r, g, b, W_G, Z
  bool wdone = wthr == -INFINITY;
  unsigned n_tested = 0, n_counted = 0;
  for (uint32_t b = r.x; b < end; b += NB) {
    __syncthreads();
    if (__syncthreads_and(wdone)) break;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t k = b + h * NTT + tid;
      const uint32_t gi = h ? gi_next1 : gi_next0;
      const uint32_t kn = k + NB;
      const uint32_t nxt = kn < r.y ? (uint32_t)v.keys[kn] : 0u;
      if (h) gi_next1 = nxt; else gi_next0 = nxt;
      if (k < end) {
        const float4* rr = v.rec + 4 * (size_t)gi;
        float4 A = rr[0], B = rr[1];
        const float4 C = rr[2];
        A.w = __log2f(A.w);  // log2 sigma, see alpha_of
        B.y = 2.0f * B.y;    // 2 b, exact
        const int e = h * NTT + tid;
        s_a[e] = A;
        s_b[e] = B;
        s_c[e] = C;
        s_e[e] = make_float2(C.w, rr[3].x);
      }
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)NB, end - b);
    int cnt = 0;
    if (!wdone) {
      for (int j0 = 0; j0 < nb; j0 += 32) {
        const int j = j0 + lane;
        bool stop = false, ok = false;
        if (j < nb) {
          const float4 A = s_a[j];
          const float2 E = s_e[j];
          stop = srt && A.z >= wthr;
          ok = A.z < wthr && A.x + E.x >= bx0 && A.x - E.x <= bx1 && A.y + E.y >= by0 &&
               A.y - E.y <= by1;
          if (ok) {
            const float4 B = s_b[j];
            ok = ellipse_meets_rect(A.x, A.y, B.x, 0.5f * B.y, B.z, B.w, bx0, bx1, by0, by1);
          }
        }
        const unsigned sb = __ballot_sync(0xffffffffu, stop);
        unsigned ob = __ballot_sync(0xffffffffu, ok);
        if (sb) ob &= (sb & (0u - sb)) - 1u;  // keep the entries before the first stop
        if ((ob >> lane) & 1u) s_list[warp][cnt + __popc(ob & ((1u << lane) - 1u))] = (uint8_t)j;
        cnt += __popc(ob);
        if (sb) {
          wdone = true;
          break;
        }
      }
    }
    __syncwarp();
#pragma unroll 4
    for (int t = 0; t < cnt; ++t) {
      const int j = s_list[warp][t];
      const float4 A = s_a[j], B = s_b[j];
      const float4 C = s_c[j];
      // quad_form's roundings, its dy terms computed once for the row
      const float dy = __fsub_rn(fpy, A.y);
      const float t1 = __fmul_rn(B.y, dy);
      const float s3 = __fmul_rn(__fmul_rn(B.z, dy), dy);
      const float dx0 = __fsub_rn(fpx0, A.x), dx1 = __fsub_rn(fpx1, A.x);
      const float q0 = __fmaf_rn(dx0, __fmaf_rn(B.x, dx0, t1), s3);
      const float q1 = __fmaf_rn(dx1, __fmaf_rn(B.x, dx1, t1), s3);
      const bool c0 = q0 <= B.w && A.z < thr0, c1 = q1 <= B.w && A.z < thr1;
      if (INSTR) {
        n_tested += in0 + in1;
        n_counted += c0 + c1;
      }
      const float a0 = c0 ? alpha_of(q0, A.w) : 0.0f;
      const float a1 = c1 ? alpha_of(q1, A.w) : 0.0f;
      acc[0][0] = fmaf(a0, C.x, acc[0][0]);
      acc[0][1] = fmaf(a0, C.y, acc[0][1]);
      acc[0][2] = fmaf(a0, C.z, acc[0][2]);
      acc[0][3] += a0;
      acc[0][4] = fmaf(a0, A.z, acc[0][4]);
      acc[1][0] = fmaf(a1, C.x, acc[1][0]);
      acc[1][1] = fmaf(a1, C.y, acc[1][1]);
      acc[1][2] = fmaf(a1, C.z, acc[1][2]);
      acc[1][3] += a1;
      acc[1][4] = fmaf(a1, A.z, acc[1][4]);
    }
  }
  if (INSTR) add_counters(v, 0, n_tested, n_counted);
  float lr = 0.f, ld = 0.f, nv = 0.f, um = 0.f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const bool in = h ? in1 : in0;
    const long long pix = h ? pix1 : pix0;
    float ct[3] = {0.f, 0.f, 0.f};
    if (in)
      for (int c = 0; c < 3; ++c) ct[c] = ld_col(v.Ct, c * npx + pix, v.prec);
    const float iN = 1.0f / (1.0f + acc[h][3]);
    const float o0 = (ct[0] + acc[h][0]) * iN;
    const float o1 = (ct[1] + acc[h][1]) * iN;
    const float o2 = (ct[2] + acc[h][2]) * iN;
    const float od = (dt[h] + acc[h][4]) * iN;
    if (in) {
      v.pix_a[pix] = make_float4(o0, o1, o2, od);
      v.pix_b[pix] = make_float4(acc[h][3], __uint_as_float(r.x), 0.f, 0.f);
      if (v.out_rgb) {
        st_col(v.out_rgb, pix, v.prec, o0);
        st_col(v.out_rgb, npx + pix, v.prec, o1);
        st_col(v.out_rgb, 2 * npx + pix, v.prec, o2);
      }
      if (v.out_depth) v.out_depth[pix] = od;
      if (v.out_weight) v.out_weight[pix] = acc[h][3];
      if (has_tgt) {
        const float dk = __ldg(v.Dtgt + pix);
        if (dk > 0.0f && dt[h] > 0.0f) {
          lr += fabsf(o0 - ld_col(v.Ctgt, pix, v.prec)) +
                fabsf(o1 - ld_col(v.Ctgt, npx + pix, v.prec)) +
                fabsf(o2 - ld_col(v.Ctgt, 2 * npx + pix, v.prec));
          ld += fabsf(od - dk);
          nv += 1.0f;
          // for the deterministic backward's quanta: the fused loss's
          // |dL/dalpha| term of this pixel is at most this x max(1/3, |lambda|)
          // x |dL/dloss| / N_valid
          um = fmaxf(um, (fabsf(o0) + fabsf(o1) + fabsf(o2) + fabsf(od)) * iN);
        }
      }
    }
  }
  if (has_tgt) {
    lr = warp_sum(lr);
    ld = warp_sum(ld);
    nv = warp_sum(nv);
    um = warp_max(um);
    __syncthreads();
    if (lane == 0) {
      s_tmp[warp * 4 + 0] = lr;
      s_tmp[warp * 4 + 1] = ld;
      s_tmp[warp * 4 + 2] = nv;
      s_tmp[warp * 4 + 3] = um;
    }
    __syncthreads();
    if (tid == 0) {
      float a = 0.f, bsum = 0.f, c = 0.f, w = 0.f;
      for (int k = 0; k < NW; ++k) {
        a += s_tmp[k * 4];
        bsum += s_tmp[k * 4 + 1];
        c += s_tmp[k * 4 + 2];
        w = fmaxf(w, s_tmp[k * 4 + 3]);
      }
      v.tile_partials[tile] = make_float4(a, bsum, c, w);
    }
  }
}

// The "with sort" forward (Table 7 reading: front to back, alpha clamped
// to 0.99, a pixel stops before T (1 - alpha) < 1e-4, C* = sum c alpha T +
// T_end C_t) with two pixels per lane, laid out as in composite_fwd_oit2_kernel
// (warp w the 8 x 8 block, lane (c, r) the pixels (2c, r), (2c + 1, r)).  The
// blend is branch-free: an entry that does not count, or reaches a finished
// pixel, or would end it, adds alpha T = 0 and leaves T as it is, so each
// pixel takes exactly the steps of the sequential blend (its T_end and last
// entry are what the backward's reverse walk starts from).
template <int TW, int TH, bool INSTR>
__global__ void __launch_bounds__(TW* TH / 2) composite_fwd_alpha2_kernel(
    const __grid_constant__ ViewBatch vb, float eps, int has_tgt) {
  chain_wait();
  constexpr int NTT = TW * TH / 2;  // threads
  constexpr int NW = NTT / 32;
  constexpr int NB = 2 * NTT;       // staged entries per batch
  constexpr int BX = TW / 8;
  __shared__ float4 s_a[NB], s_b[NB], s_c[NB];
  __shared__ float2 s_e[NB];
  __shared__ uint8_t s_list[NW][NB];
  __shared__ float s_tmp[NW * 3];
  const int slot = batch_slot(vb.tile_start, vb.n, blockIdx.x);
  const ViewDev& v = vb.v[vb.order[slot]];
  const int tile = tile_of(v, blockIdx.x - vb.tile_start[slot]);
  const int W = v.cam.W, H = v.cam.H;
  const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ox = (warp % BX) * 8, oy = (warp / BX) * 8;
  const int px0 = tx * TW + ox + 2 * (lane & 3), px1 = px0 + 1;
  const int py = ty * TH + oy + (lane >> 2);
  const bool in0 = px0 < W && py < H, in1 = px1 < W && py < H;
  const long long npx = (long long)W * H;
  const long long pix0 = (long long)py * W + px0, pix1 = pix0 + 1;
  float dt[2] = {0.f, 0.f};
  if (in0) dt[0] = __ldg(v.Dt + pix0);
  if (in1) dt[1] = __ldg(v.Dt + pix1);
  const float thr0 = in0 ? depth_threshold(dt[0], eps) : -INFINITY;
  const float thr1 = in1 ? depth_threshold(dt[1], eps) : -INFINITY;
  const uint2 r = v.tile_ranges[tile];
  uint32_t gi_next0 = r.x + tid < r.y ? (uint32_t)v.keys[r.x + tid] : 0u;
  uint32_t gi_next1 = r.x + NTT + tid < r.y ? (uint32_t)v.keys[r.x + NTT + tid] : 0u;
  const float wthr = warp_max(fmaxf(thr0, thr1));
  const float bthr = block_max<NTT>(fmaxf(thr0, thr1), s_tmp);
  // the lists are depth-sorted: they end at the first Gaussian behind every
  // pixel of the tile
  const uint32_t end = depth_cut_block<NTT>(v.keys, r.x, r.y, bthr);
  const float bx0 = (float)(tx * TW + ox), bx1 = bx0 + 7.0f;
  const float by0 = (float)(ty * TH + oy), by1 = by0 + 7.0f;
  const float fpx0 = (float)px0, fpx1 = (float)px1, fpy = (float)py;
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};  // r, g, b, depth
  float T[2] = {1.0f, 1.0f};
  uint32_t last[2] = {r.x, r.x};
  bool done0 = !in0, done1 = !in1;
  bool wdone = wthr == -INFINITY;
  unsigned n_tested = 0, n_counted = 0;
  for (uint32_t b = r.x; b < end; b += NB) {
    __syncthreads();
    wdone = wdone || __all_sync(0xffffffffu, done0 && done1);
    if (__syncthreads_and(wdone)) break;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t k = b + h * NTT + tid;
      const uint32_t gi = h ? gi_next1 : gi_next0;
      const uint32_t kn = k + NB;
      const uint32_t nxt = kn < r.y ? (uint32_t)v.keys[kn] : 0u;
      if (h) gi_next1 = nxt; else gi_next0 = nxt;
      if (k < end) {
        const float4* rr = v.rec + 4 * (size_t)gi;
        float4 A = rr[0], B = rr[1];
        const float4 C = rr[2];
        A.w = __log2f(A.w);  // log2 sigma, see alpha_of
        B.y = 2.0f * B.y;    // 2 b, exact
        const int e = h * NTT + tid;
        s_a[e] = A;
        s_b[e] = B;
        s_c[e] = C;
        s_e[e] = make_float2(C.w, rr[3].x);
      }
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)NB, end - b);
    int cnt = 0;
    if (!wdone) {
      for (int j0 = 0; j0 < nb; j0 += 32) {
        const int j = j0 + lane;
        bool stop = false, ok = false;
        if (j < nb) {
          const float4 A = s_a[j];
          const float2 E = s_e[j];
          stop = A.z >= wthr;
          ok = A.x + E.x >= bx0 && A.x - E.x <= bx1 && A.y + E.y >= by0 && A.y - E.y <= by1;
          if (ok) {
            const float4 B = s_b[j];
            ok = ellipse_meets_rect(A.x, A.y, B.x, 0.5f * B.y, B.z, B.w, bx0, bx1, by0, by1);
          }
        }
        const unsigned sb = __ballot_sync(0xffffffffu, stop);
        unsigned ob = __ballot_sync(0xffffffffu, ok);
        if (sb) ob &= (sb & (0u - sb)) - 1u;  // keep the entries before the first stop
        if ((ob >> lane) & 1u) s_list[warp][cnt + __popc(ob & ((1u << lane) - 1u))] = (uint8_t)j;
        cnt += __popc(ob);
        if (sb) {
          wdone = true;
          break;
        }
      }
    }
    __syncwarp();
    for (int t = 0; t < cnt; ++t) {
      const int j = s_list[warp][t];
      const float4 A = s_a[j], B = s_b[j];
      const float4 C = s_c[j];
      const float dy = __fsub_rn(fpy, A.y);
      const float t1 = __fmul_rn(B.y, dy);
      const float s3 = __fmul_rn(__fmul_rn(B.z, dy), dy);
      const float dx0 = __fsub_rn(fpx0, A.x), dx1 = __fsub_rn(fpx1, A.x);
      const float q0 = __fmaf_rn(dx0, __fmaf_rn(B.x, dx0, t1), s3);
      const float q1 = __fmaf_rn(dx1, __fmaf_rn(B.x, dx1, t1), s3);
      const bool c0 = q0 <= B.w && A.z < thr0, c1 = q1 <= B.w && A.z < thr1;
      if (INSTR) {
        n_tested += in0 + in1;
        n_counted += c0 + c1;
      }
      const uint32_t idx = b + (uint32_t)j + 1u;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool live = (h ? c1 : c0) && !(h ? done1 : done0);
        const float a = live ? fminf(alpha_of(h ? q1 : q0, A.w), kAlphaMax) : 0.0f;
        const float test = T[h] * (1.0f - a);
        const bool stop = live && test < kTMin;
        if (h) done1 = done1 || stop; else done0 = done0 || stop;
        const float aT = stop ? 0.0f : a * T[h];
        acc[h][0] = fmaf(C.x, aT, acc[h][0]);
        acc[h][1] = fmaf(C.y, aT, acc[h][1]);
        acc[h][2] = fmaf(C.z, aT, acc[h][2]);
        acc[h][3] = fmaf(A.z, aT, acc[h][3]);
        const bool step = live && !stop;
        T[h] = step ? test : T[h];
        last[h] = step ? idx : last[h];
      }
    }
  }
  if (INSTR) add_counters(v, 0, n_tested, n_counted);
  float lr = 0.f, ld = 0.f, nv = 0.f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const bool in = h ? in1 : in0;
    const long long pix = h ? pix1 : pix0;
    float ct[3] = {0.f, 0.f, 0.f};
    if (in)
      for (int c = 0; c < 3; ++c) ct[c] = ld_col(v.Ct, c * npx + pix, v.prec);
    const float o0 = acc[h][0] + T[h] * ct[0];
    const float o1 = acc[h][1] + T[h] * ct[1];
    const float o2 = acc[h][2] + T[h] * ct[2];
    const float od = acc[h][3] + T[h] * dt[h];
    if (in) {
      v.pix_a[pix] = make_float4(o0, o1, o2, od);
      v.pix_b[pix] = make_float4(T[h], __uint_as_float(last[h]), 0.f, 0.f);
      if (v.out_rgb) {
        st_col(v.out_rgb, pix, v.prec, o0);
        st_col(v.out_rgb, npx + pix, v.prec, o1);
        st_col(v.out_rgb, 2 * npx + pix, v.prec, o2);
      }
      if (v.out_depth) v.out_depth[pix] = od;
      if (v.out_weight) v.out_weight[pix] = 1.0f - T[h];
      if (has_tgt) {
        const float dk = __ldg(v.Dtgt + pix);
        if (dk > 0.0f && dt[h] > 0.0f) {
          lr += fabsf(o0 - ld_col(v.Ctgt, pix, v.prec)) +
                fabsf(o1 - ld_col(v.Ctgt, npx + pix, v.prec)) +
                fabsf(o2 - ld_col(v.Ctgt, 2 * npx + pix, v.prec));
          ld += fabsf(od - dk);
          nv += 1.0f;
        }
      }
    }
  }
  if (has_tgt) {
    lr = warp_sum(lr);
    ld = warp_sum(ld);
    nv = warp_sum(nv);
    __syncthreads();
    if (lane == 0) {
      s_tmp[warp * 3 + 0] = lr;
      s_tmp[warp * 3 + 1] = ld;
      s_tmp[warp * 3 + 2] = nv;
    }
    __syncthreads();
    if (tid == 0) {
      float a = 0.f, bsum = 0.f, c = 0.f;
      for (int k = 0; k < NW; ++k) {
        a += s_tmp[k * 3];
        bsum += s_tmp[k * 3 + 1];
        c += s_tmp[k * 3 + 2];
      }
      v.tile_partials[tile] = make_float4(a, bsum, c, 0.f);
    }
  }
}

// Per-view loss from the tile partial sums, summed in a fixed order: each
// thread adds a strided subset, then a fixed shuffle tree and warp order.
// scalars: [0] view loss, [1] sum |C* - C|, [2] sum |D* - D|, [3] N_valid,
// and for the deterministic OIT backward's quanta, bounds per unit
// |dL/dloss| on the fused loss's upstream terms: [6] >= |dL/dC*| / (1 + W),
// |dL/dD*| / (1 + W) = max(1/3, |lambda|) / N_valid, [7] >= |dL/dalpha|'s
// sum term (max(1/3, |lambda|) / N_valid x the forward's per-pixel maximum
// of (|C*| + |D*|) / (1 + W)); both carry a factor 1 + 2^-10 for the FP32
// rounding of the backward's products.  The views' losses are summed in view
// order into *loss (overwritten when `first`, else added).
__global__ void __launch_bounds__(256) finalize_loss_kernel(const __grid_constant__ ViewBatch vb,
                                                            float lambda_depth, float* loss,
                                                            int first) {
  chain_wait();
  __shared__ float s[4][8];
  float total = 0.f;
  for (int k = 0; k < vb.n; ++k) {
    const ViewDev& v = vb.v[k];
    const int ntiles = v.tiles_x * v.tiles_y;
    float a = 0.f, b = 0.f, c = 0.f, u = 0.f;
    for (int t = threadIdx.x; t < ntiles; t += 256) {
      const float4 p = v.tile_partials[t];
      a += p.x;
      b += p.y;
      c += p.z;
      u = fmaxf(u, p.w);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    u = warp_max(u);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      s[0][w] = a;
      s[1][w] = b;
      s[2][w] = c;
      s[3][w] = u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float sa = 0.f, sb = 0.f, n = 0.f, um = 0.f;
      for (int q = 0; q < 8; ++q) {
        sa += s[0][q];
        sb += s[1][q];
        n += s[2][q];
        um = fmaxf(um, s[3][q]);
      }
      const float L = n > 0.f ? sa / (3.0f * n) + lambda_depth * sb / n : 0.0f;
      const float hb = n > 0.f ? fmaxf(1.0f / 3.0f, fabsf(lambda_depth)) / n * (1.0f + 0x1p-10f)
                               : 0.0f;
      v.scalars[0] = L;
      v.scalars[1] = sa;
      v.scalars[2] = sb;
      v.scalars[3] = n;
      v.scalars[6] = hb;
      v.scalars[7] = hb * um;
      total = k == 0 ? L : total + L;
    }
  }
  if (threadIdx.x == 0 && loss) *loss = first ? total : *loss + total;
}

// Upstream gradient of one pixel (already scaled).
__device__ __forceinline__ void upstream(const ViewDev& v, long long pix, long long npx,
                                         const float4& st, float dt, int fused, float lambda,
                                         float scale, float& g0, float& g1, float& g2,
                                         float& gD) {
  if (fused) {
    const float dk = __ldg(v.Dtgt + pix);
    if (dk > 0.0f && dt > 0.0f) {
      const float s3 = scale * (1.0f / 3.0f);
      const float r0 = st.x - ld_col(v.Ctgt, pix, v.prec);
      const float r1 = st.y - ld_col(v.Ctgt, npx + pix, v.prec);
      const float r2 = st.z - ld_col(v.Ctgt, 2 * npx + pix, v.prec), rd = st.w - dk;
      g0 = r0 > 0.f ? s3 : (r0 < 0.f ? -s3 : 0.f);
      g1 = r1 > 0.f ? s3 : (r1 < 0.f ? -s3 : 0.f);
      g2 = r2 > 0.f ? s3 : (r2 < 0.f ? -s3 : 0.f);
      const float sl = lambda * scale;
      gD = rd > 0.f ? sl : (rd < 0.f ? -sl : 0.f);
    } else {
      g0 = g1 = g2 = gD = 0.f;
    }
  } else {
    g0 = v.g_rgb ? __ldg(v.g_rgb + pix) : 0.f;
    g1 = v.g_rgb ? __ldg(v.g_rgb + npx + pix) : 0.f;
    g2 = v.g_rgb ? __ldg(v.g_rgb + 2 * npx + pix) : 0.f;
    gD = v.g_depth ? __ldg(v.g_depth + pix) : 0.f;
  }
}

__device__ __forceinline__ float loss_scale(const ViewDev& v, int fused, const float* dloss) {
  if (!fused) return 1.0f;
  const float nv = v.scalars[3];
  return (nv > 0.f ? 1.0f / nv : 0.f) * (dloss ? *dloss : 1.0f);
}

// Deterministic mode: the pair_grads slot of the pair (tile (tx, ty),
// Gaussian gi): the Gaussian's first slot (pair_base) + the tile's row-major
// index inside the Gaussian's tile rectangle (from its record: centre mx, my,
// extents ex, ey).
__device__ __forceinline__ long long pair_slot(const ViewDev& v, uint32_t gi, int tx, int ty,
                                               float mx, float my, float ex, float ey) {
  int x0, x1, y0, y1;
  record_rect(mx, my, ex, ey, v.cam.W, v.cam.H, x0, x1, y0, y1);
  const int tx0 = x0 / v.tw, tx1 = x1 / v.tw, ty0 = y0 / v.th;
  return (long long)v.pair_base[gi] + (long long)(ty - ty0) * (tx1 - tx0 + 1) + (tx - tx0);
}

__device__ __forceinline__ void zero_slot(const ViewDev& v, long long slot) {
  if (slot < v.pair_slots) {
    float4* o = v.pair_grads + 3 * slot;
    o[0] = o[1] = o[2] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ----------------------------------------- deterministic fixed-point sums
// Deterministic mode (OIT blend, tile schedule) runs the carry-over backward,
// whose (warp block, Gaussian) partials reach a Gaussian in an order that
// varies from run to run.  Each partial is therefore added as a 64-bit
// integer in units of 2^e[k] for component k: integer addition is
// associative, so the sum is the same whatever the order, and converting
// back to float is one rounding.  e[k] comes from a bound b_k on the
// magnitude of any partial of that component of that Gaussian, from its
// record and the view's upstream bounds (hmax >= |h| of every pixel's
// dL/dC* / N, dL/dD* / N; smax >= |sv|):
//   a counted pixel has alpha <= sigma <= 1, |dx| <= ext_x, |dy| <= ext_y;
//   with V = hmax (|r| + |g| + |b| + |d|) + smax >= |dL/dalpha|, over a warp
//   block's 32 pixels |m_0..3| <= 32 hmax, |m4| <= 32 V sigma,
//   |m5| <= 32 V ext_x, |m6| <= 32 V ext_y, |m7| <= 32 V ext_x^2,
//   |m8| <= 32 V ext_x ext_y, |m9| <= 32 V ext_y^2, and grad2d_of's
//   combinations follow; the bounds carry a factor 2 for the FP32 rounding
//   of the partial and of the bound itself.
// The bounds factor as (record term c_k) x (V or hmax); the projection
// stores the record terms' exponents with the partial count in the record
// (fixed_pre_exponents), and the walk and the conversion back add the
// exponent of V or hmax.  With at most n = (tiles of the Gaussian's
// rectangle) x (warps per tile) partials, 2^e[k] > b_k 2^-(62 - ceil(log2 n))
// keeps every partial below 2^(62 - ceil(log2 n)) quanta and every sum below
// 2^62: no overflow.  The quantum is about 2^-56 of the bound at the room
// workload's sizes.  e is clamped to [-120, 126] so that 2^-e and 2^e are
// normal floats (raising e only coarsens the quantum; lowering it to 126
// happens only for bounds above 2^(188 - ceil(log2 n)), where any finite
// FP32 partial is still below 2^2 quanta).
// Add a (warp block, Gaussian gi) partial g to gi's fixed-point sums.  The
// integer q = floor(g 2^-e) is formed from the float's fields: g = s m
// 2^(E - 150) with the sign s and the 24-bit significand m, so q =
// floor(s m 2^39 / 2^(189 + e - E)), one arithmetic right shift of s m 2^39
// (the bound keeps E - 150 - e <= 38, so the shift is at least 1; an error
// below one quantum, the same in every run; shifts past 63 leave the sign).
// A component that is zero adds nothing and issues no atomic.  (Integer
// shifts: a float to 64-bit integer conversion per component measured
// 3.7 us slower per backward.)
__device__ __forceinline__ long long fixed_shr(long long x, int n) {
  long long r;
  asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(n));  // n > 63 acts as 64
  return r;
}
__device__ __forceinline__ void fixed_add(const ViewDev& v, uint32_t gi, const float (&g)[10],
                                          const int (&e)[10]) {
  unsigned long long* o = reinterpret_cast<unsigned long long*>(v.grad_fixed + 10 * (size_t)gi);
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const int bits = __float_as_int(g[k]);
    const int amt = e[k] + 189 - (int)(((unsigned)bits >> 23) & 0xffu);
    const int sm = (bits < 0 ? -1 : 1) * ((bits & 0x7fffff) | 0x800000);
    const long long q = fixed_shr((long long)((unsigned long long)((unsigned)sm << 7) << 32), amt);
    if (g[k] != 0.0f) atomicAdd(o + k, (unsigned long long)q);
  }
}

// The upstream maxima of the views with explicit upstream images
// (scalars[6] = hmax, scalars[7] = smax, zero on entry), from the same
// per-pixel terms the backward stages; views with the fused loss have their
// bounds from the forward.  Block row blockIdx.y: view; the blocks stride
// over the pixels, reduce in shared memory and add one atomic maximum per
// block (one atomic per warp, all on the same two words, took 19 us at
// 640 x 480).
__global__ void __launch_bounds__(256) upstream_max_kernel(const __grid_constant__ ViewBatch vb,
                                                           float eps, float lambda,
                                                           const float* dloss) {
  chain_wait();
  __shared__ float s_m[2][8];
  const ViewDev& v = vb.v[blockIdx.y];
  if (v.fused) return;
  const long long npx = (long long)v.cam.W * v.cam.H;
  const float scale = loss_scale(v, v.fused, dloss);
  float hm = 0.f, sm = 0.f;
  for (long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x; pix < npx;
       pix += (long long)gridDim.x * blockDim.x) {
    const float4 st = v.pix_a[pix];
    const float iN = 1.0f / (1.0f + v.pix_b[pix].x);
    const float dt = __ldg(v.Dt + pix);
    float g0, g1, g2, gD;
    upstream(v, pix, npx, st, dt, v.fused, lambda, scale, g0, g1, g2, gD);
    hm = fmaxf(hm, fmaxf(fmaxf(fabsf(g0 * iN), fabsf(g1 * iN)), fmaxf(fabsf(g2 * iN), fabsf(gD * iN))));
    sm = fmaxf(sm, fabsf((g0 * st.x + g1 * st.y + g2 * st.z + gD * st.w) * iN));
  }
  hm = warp_max(hm);
  sm = warp_max(sm);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_m[0][w] = hm;
    s_m[1][w] = sm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      hm = fmaxf(hm, s_m[0][k]);
      sm = fmaxf(sm, s_m[1][k]);
    }
    // non-negative floats order as their bit patterns
    atomicMax(reinterpret_cast<unsigned*>(v.scalars + 6), __float_as_uint(hm));
    atomicMax(reinterpret_cast<unsigned*>(v.scalars + 7), __float_as_uint(sm));
  }
}

// Fixed-point sums -> grad2d (float) for calls whose projection adjoint
// does not read the sums itself.  Block row blockIdx.y: view.
__global__ void __launch_bounds__(256) fixed_to_grad2d_kernel(const __grid_constant__ ViewBatch vb,
                                                              int M, const float* dloss) {
  chain_wait();
  const ViewDev& v = vb.v[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  float4 ga, gb, gc;
  fixed_grad2d(v, i, dloss, ga, gb, gc);
  float4* o = v.grad2d + 3 * (size_t)i;
  o[0] = ga;
  o[1] = gb;
  o[2] = gc;
}

// 2D gradient g of a (tile, Gaussian gi) pair: deterministic mode writes it
// into the pair's slot (skipped beyond the slot capacity), else adds it to
// grad2d with vector atomics.
__device__ __forceinline__ void store_grad2d(const ViewDev& v, int deterministic, long long slot,
                                             uint32_t gi, const float (&g)[10]) {
  const float4 a = make_float4(g[0], g[1], g[2], g[3]);
  const float4 b = make_float4(g[4], g[5], g[6], g[7]);
  const float4 c = make_float4(g[8], g[9], 0.f, 0.f);
  if (deterministic) {
    if (slot >= v.pair_slots) return;
    float4* o = v.pair_grads + 3 * slot;
    o[0] = a;
    o[1] = b;
    o[2] = c;
  } else {
    float4* o = v.grad2d + 3 * (size_t)gi;
    atomicAdd(o, a);
    atomicAdd(o + 1, b);
    atomicAdd(reinterpret_cast<float2*>(o + 2), make_float2(c.x, c.y));
  }
}

// ------------------------------------------------------- backward, OIT mode
// A lane's Gaussian in the OIT backward's pixel walk.
struct BwdGauss {
  float mx, my, d, lns, sig, ca, b2, cc, qmax, cr, cg, cb;
  uint32_t gi;
  int kx0, kx1, ky0, ky1;  // its rectangle inside the block (instrumented runs)
};

// Staged record (A, B with B.y = 2 b, C, E = extents) -> lane registers.
template <bool INSTR>
__device__ __forceinline__ BwdGauss bwd_gauss(const float4& A, const float4& B, const float4& C,
                                              const float2& E, uint32_t gi, float bx0, float by0) {
  BwdGauss G;
  G.mx = A.x; G.my = A.y; G.d = A.z; G.sig = A.w; G.lns = __log2f(A.w);
  G.ca = B.x; G.b2 = B.y; G.cc = B.z; G.qmax = B.w;
  G.cr = C.x; G.cg = C.y; G.cb = C.z;
  G.gi = gi;
  G.kx0 = 8; G.kx1 = -1; G.ky0 = 4; G.ky1 = -1;
  if (INSTR) {
    G.kx0 = max(0, (int)ceilf(G.mx - E.x - bx0));
    G.kx1 = min(7, (int)floorf(G.mx + E.x - bx0));
    G.ky0 = max(0, (int)ceilf(G.my - E.y - by0));
    G.ky1 = min(3, (int)floorf(G.my + E.y - by0));
  }
  return G;
}

// An idle lane: q >= 0 > qmax, so it adds alpha = 0 everywhere.
__device__ __forceinline__ BwdGauss bwd_idle() {
  BwdGauss G;
  G.mx = G.my = G.d = G.lns = 0.f;
  G.sig = 1.f;
  G.ca = G.b2 = G.cc = 0.f;
  G.qmax = -1.f;
  G.cr = G.cg = G.cb = 0.f;
  G.gi = 0u;
  G.kx0 = 8; G.kx1 = -1; G.ky0 = 4; G.ky1 = -1;
  return G;
}

// The lane's Gaussian over the warp's 8 x 4 pixel block (pixels blk ..
// blk + 31 of s_h / s_s, row-major), unrolled and branch-free: a pixel
// outside the support fails q <= qmax and adds alpha = 0 (cheaper than
// bounding each lane's loop by its rectangle).  m = (sum alpha h (4),
// sum v, sum v dx, sum v dy, sum v dx^2, sum v dx dy, sum v dy^2) with
// v = dL/dalpha * alpha.
template <bool INSTR>
__device__ __forceinline__ void bwd_walk(const BwdGauss& G, bool has, int blk, float bx0, float by0,
                                         const float4* s_h, const float2* s_s, float (&m)[10],
                                         unsigned& n_tested, unsigned& n_counted) {
  float dcr = 0.f, dcg = 0.f, dcb = 0.f, dd = 0.f, sa = 0.f;
  float sx = 0.f, sy = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f;
#pragma unroll 2
  for (int ky = 0; ky < 4; ++ky) {
    const float dy = __fsub_rn(by0 + (float)ky, G.my);
    // the dy terms of quad_form, hoisted out of the row (same roundings)
    const float t1 = __fmul_rn(G.b2, dy);
    const float s3 = __fmul_rn(__fmul_rn(G.cc, dy), dy);
    // row sums of v, v dx, v dx^2; the dy moments follow per row
    float ra = 0.f, rx = 0.f, rxx = 0.f;
#pragma unroll
    for (int kx = 0; kx < 8; ++kx) {
      const int p = blk + ky * 8 + kx;
      const float2 ss = s_s[p];
      const float dx = __fsub_rn(bx0 + (float)kx, G.mx);
      const float q = __fmaf_rn(dx, __fmaf_rn(G.ca, dx, t1), s3);
      const bool counted = q <= G.qmax && G.d < ss.y;
      if (INSTR) {
        n_tested += has && kx >= G.kx0 && kx <= G.kx1 && ky >= G.ky0 && ky <= G.ky1;
        n_counted += counted;
      }
      const float4 hh = s_h[p];
      const float al = counted ? alpha_of(q, G.lns) : 0.0f;
      dcr = fmaf(al, hh.x, dcr);
      dcg = fmaf(al, hh.y, dcg);
      dcb = fmaf(al, hh.z, dcb);
      dd = fmaf(al, hh.w, dd);
      const float dLda = fmaf(hh.x, G.cr, fmaf(hh.y, G.cg, fmaf(hh.z, G.cb, fmaf(hh.w, G.d, -ss.x))));
      const float vv = dLda * al;
      ra += vv;
      const float tx_ = vv * dx;
      rx += tx_;
      rxx = fmaf(tx_, dx, rxx);
    }
    sa += ra;
    sx += rx;
    sxx += rxx;
    sy = fmaf(ra, dy, sy);
    sxy = fmaf(rx, dy, sxy);
    syy = fmaf(ra * dy, dy, syy);
  }
  m[0] = dcr; m[1] = dcg; m[2] = dcb; m[3] = dd; m[4] = sa;
  m[5] = sx; m[6] = sy; m[7] = sxx; m[8] = sxy; m[9] = syy;
}

// 2D gradient of a Gaussian from its summed moments m (see bwd_walk):
// d/d(mx, my, conic a, b, c, sigma, r, g, b, d); dL/dsigma = sum dL/dalpha G
// = (sum dL/dalpha alpha) / sigma.
__device__ __forceinline__ void grad2d_of(const float (&m)[10], float ca, float cb, float cc,
                                          float sig, float (&g)[10]) {
  g[0] = ca * m[5] + cb * m[6];
  g[1] = cb * m[5] + cc * m[6];
  g[2] = -0.5f * m[7];
  g[3] = -m[8];
  g[4] = -0.5f * m[9];
  g[5] = m[4] / sig;
  g[6] = m[0]; g[7] = m[1]; g[8] = m[2]; g[9] = m[3];
}

// list entries staged per round of the OIT backward (per-warp partials of
// NW x NB x 10 floats stay within 20 KB of shared memory)
template <int NT>
struct BwdBatch {
  static constexpr int value = NT >= 256 ? 64 : (NT >= 128 ? 128 : 64);
};

// OIT backward: warp w owns the same 8 x 4 pixel block as in the forward.  Per
// staged batch, each warp compacts the Gaussians whose rectangle overlaps its
// block (depth order, cut at the block's threshold); lanes take one Gaussian
// each and walk the block's pixels (shared-memory broadcasts), accumulating
// 10 moments privately.  Per-warp partials are summed over warps in a fixed
// order and turned into the 2D gradient of the (tile, Gaussian) pair.
template <int TW, int TH, bool INSTR>
__global__ void __launch_bounds__(TW* TH) composite_bwd_oit_kernel(const __grid_constant__ ViewBatch vb,
                                                                   float eps, float lambda,
                                                                   const float* dloss,
                                                                   int deterministic, int sorted) {
  chain_wait();
  constexpr int NT = TW * TH;
  constexpr int NW = NT / 32;
  constexpr int NB = BwdBatch<NT>::value;
  constexpr int NMW = NB / 32;  // mask words per warp
  __shared__ float4 s_h[NT];
  __shared__ float2 s_s[NT];
  __shared__ float4 s_a[NB], s_b[NB], s_c[NB];
  __shared__ float2 s_e[NB];
  __shared__ float s_part[NW][NB][10];
  __shared__ uint32_t s_mask[NW][NMW];
  __shared__ uint8_t s_list[NW][NB];
  __shared__ float s_tmp[NW];
  const int slot = batch_slot(vb.tile_start, vb.n, blockIdx.x);
  const ViewDev& v = vb.v[vb.order[slot]];
  const int tile = tile_of(v, blockIdx.x - vb.tile_start[slot]);
  const int fused = v.fused;
  const int W = v.cam.W, H = v.cam.H;
  const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int ox, oy, lx, ly;
  warp_block<TW>(warp, lane, ox, oy, lx, ly);
  const int px = tx * TW + lx, py = ty * TH + ly;
  const bool inside = px < W && py < H;
  const long long npx = (long long)W * H, pix = (long long)py * W + px;
  const float scale = loss_scale(v, fused, dloss);
  float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
  float sv = 0.f, thr = -INFINITY;
  if (inside) {
    const float4 st = v.pix_a[pix];
    const float iN = 1.0f / (1.0f + v.pix_b[pix].x);
    const float dt = __ldg(v.Dt + pix);
    float g0, g1, g2, gD;
    upstream(v, pix, npx, st, dt, fused, lambda, scale, g0, g1, g2, gD);
    h = make_float4(g0 * iN, g1 * iN, g2 * iN, gD * iN);
    sv = (g0 * st.x + g1 * st.y + g2 * st.z + gD * st.w) * iN;
    if (g0 != 0.f || g1 != 0.f || g2 != 0.f || gD != 0.f) thr = depth_threshold(dt, eps);
  }
  s_h[tid] = h;
  s_s[tid] = make_float2(sv, thr);
  const uint2 r = v.tile_ranges[tile];
  uint32_t gi_next = tid < NB && r.x + tid < r.y ? (uint32_t)v.keys[r.x + tid] : 0u;
  const float wthr = warp_max(thr);
  const float bthr = block_max<NT>(thr, s_tmp);
  // a depth-sorted list ends at the first Gaussian behind every pixel of the
  // tile; an unsorted one is walked to its end, each warp skipping the
  // Gaussians behind all of its pixels
  const bool srt = sorted && v.sorted;  // this view's lists are depth-sorted
  const uint32_t end = srt ? depth_cut_block<NT>(v.keys, r.x, r.y, bthr) : r.y;
  const float bx0 = (float)(tx * TW + ox), bx1 = bx0 + 7.0f;
  const float by0 = (float)(ty * TH + oy), by1 = by0 + 3.0f;
  const int blk = warp * 32;  // this warp's pixels in s_h / s_s
  bool wdone = wthr == -INFINITY;
  unsigned n_tested = 0, n_counted = 0;
  for (uint32_t b = r.x; b < end; b += NB) {
    __syncthreads();
    if (__syncthreads_and(wdone)) break;
    const uint32_t gi = gi_next;
    if (tid < NB) gi_next = b + NB + tid < r.y ? (uint32_t)v.keys[b + NB + tid] : 0u;
    if (tid < NB && b + tid < end) {
      const float4* rr = v.rec + 4 * (size_t)gi;
      float4 B = rr[1];
      const float4 C = rr[2];
      B.y = 2.0f * B.y;
      s_a[tid] = rr[0];
      s_b[tid] = B;
      s_c[tid] = C;
      s_e[tid] = make_float2(C.w, rr[3].x);
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)NB, end - b);
    int cnt = 0;
    if (lane < NMW) s_mask[warp][lane] = 0u;
    __syncwarp();
    if (!wdone) {
      for (int j0 = 0; j0 < nb; j0 += 32) {
        const int j = j0 + lane;
        bool stop = false, ok = false;
        if (j < nb) {
          const float4 A = s_a[j];
          const float2 E = s_e[j];
          stop = srt && A.z >= wthr;
          ok = A.z < wthr && A.x + E.x >= bx0 && A.x - E.x <= bx1 && A.y + E.y >= by0 &&
               A.y - E.y <= by1;
          if (ok) {
            const float4 B = s_b[j];
            ok = ellipse_meets_rect(A.x, A.y, B.x, 0.5f * B.y, B.z, B.w, bx0, bx1, by0, by1);
          }
        }
        const unsigned sb = __ballot_sync(0xffffffffu, stop);
        unsigned ob = __ballot_sync(0xffffffffu, ok);
        if (sb) ob &= (sb & (0u - sb)) - 1u;
        if ((ob >> lane) & 1u) s_list[warp][cnt + __popc(ob & ((1u << lane) - 1u))] = (uint8_t)j;
        cnt += __popc(ob);
        if (lane == 0) s_mask[warp][j0 >> 5] = ob;
        if (sb) {
          wdone = true;
          break;
        }
      }
    }
    __syncwarp();
    for (int c0 = 0; c0 < cnt; c0 += 32) {
      const int t = c0 + lane;
      const bool has = t < cnt;
      const int j = has ? s_list[warp][t] : 0;
      const BwdGauss G = has ? bwd_gauss<INSTR>(s_a[j], s_b[j], s_c[j], s_e[j], 0u, bx0, by0)
                             : bwd_idle();
      float m[10];
      bwd_walk<INSTR>(G, has, blk, bx0, by0, s_h, s_s, m, n_tested, n_counted);
      if (has) {
        float* o = s_part[warp][j];
#pragma unroll
        for (int c = 0; c < 10; ++c) o[c] = m[c];
      }
    }
    __syncthreads();
    // fixed-order sum over warps, one gradient per (tile, Gaussian) pair
    for (int t = tid; t < nb; t += NT) {
      float m[10];
#pragma unroll
      for (int c = 0; c < 10; ++c) m[c] = 0.f;
      bool any = false;
      for (int w2 = 0; w2 < NW; ++w2) {
        if ((s_mask[w2][t >> 5] >> (t & 31)) & 1u) {
          any = true;
#pragma unroll
          for (int c = 0; c < 10; ++c) m[c] += s_part[w2][t][c];
        }
      }
      if (any || deterministic) {
        const float4 A = s_a[t], B = s_b[t];
        const float2 E = s_e[t];
        const uint32_t gi = (uint32_t)v.keys[b + t];
        float g[10];
        grad2d_of(m, B.x, 0.5f * B.y, B.z, A.w, g);
        store_grad2d(v, deterministic,
                     deterministic ? pair_slot(v, gi, tx, ty, A.x, A.y, E.x, E.y) : 0, gi, g);
      }
    }
  }
  if (INSTR) add_counters(v, 2, n_tested, n_counted);
  if (deterministic) {
    // pairs behind the depth cut contribute nothing; give their slots zeros
    for (uint32_t k = end + tid; k < r.y; k += NT) {
      const uint32_t gi = (uint32_t)v.keys[k];
      const float4 A = v.rec[4 * (size_t)gi], C = v.rec[4 * (size_t)gi + 2];
      zero_slot(v, pair_slot(v, gi, tx, ty, A.x, A.y, C.w, v.rec[4 * (size_t)gi + 3].x));
    }
  }
}

// Sort-free OIT backward, not deterministic.  As composite_bwd_oit_kernel,
// but a warp walks only full groups of 32 Gaussians: the culled Gaussians
// that do not fill a group wait in their lanes' registers for the next
// staged batch (one partial group per warp and tile, at its end), and each
// lane adds its Gaussian's block gradient to grad2d with vector atomics, so
// no per-warp partials are combined in shared memory.
template <int NT>
struct BwdCarryBatch {
  static constexpr int value = NT >= 128 ? 256 : 128;
};

template <bool INSTR, bool FIXED>
__device__ __forceinline__ void bwd_flush(const ViewDev& v, const BwdGauss& G, bool has, int blk,
                                          float bx0, float by0, const float4* s_h,
                                          const float2* s_s, const float* dloss,
                                          unsigned& n_tested, unsigned& n_counted) {
  float m[10], g[10];
  bwd_walk<INSTR>(G, has, blk, bx0, by0, s_h, s_s, m, n_tested, n_counted);
  if (has) {
    grad2d_of(m, G.ca, 0.5f * G.b2, G.cc, G.sig, g);
    if constexpr (FIXED) {
      // the pre-exponents are read back here (an L2 hit: the batch staged
      // the record) rather than carried through the walk in registers
      const float4* rr = v.rec + 4 * (size_t)G.gi;
      const uint2 pre = fixed_pre(v, __ldg(rr + 3), G.mx, G.my, G.ca, 0.5f * G.b2, G.cc, &rr[2].w);
      float hm, sm;
      fixed_maxima(v, dloss, hm, sm);
      int e[10];
      fixed_exponents(pre, fixed_v(hm, sm, G.cr, G.cg, G.cb, G.d), hm, e);
      fixed_add(v, G.gi, g, e);
    } else {
      store_grad2d(v, 0, 0u, G.gi, g);
    }
  }
}

// FIXED: deterministic mode's fixed-point sums (a separate instantiation, so
// that the default walk carries none of their code).
template <int TW, int TH, bool INSTR, bool FIXED>
__global__ void __launch_bounds__(TW* TH)
    composite_bwd_oit_carry_kernel(const __grid_constant__ ViewBatch vb, float eps, float lambda,
                                   const float* dloss) {
  chain_wait();
  constexpr int NT = TW * TH;
  constexpr int NB = BwdCarryBatch<NT>::value;
  constexpr int NW = NT / 32;
  constexpr int KPT = NB / NT;  // entries staged per thread
  static_assert(KPT >= 1 && KPT * NT == NB, "a batch is a whole number of entries per thread");
  __shared__ float4 s_h[NT];
  __shared__ float2 s_s[NT];
  __shared__ float4 s_a[NB], s_b[NB], s_c[NB];
  __shared__ float2 s_e[NB];
  __shared__ uint32_t s_gi[NB];
  __shared__ uint8_t s_list[NW][NB];
  const int slot = batch_slot(vb.tile_start, vb.n, blockIdx.x);
  const ViewDev& v = vb.v[vb.order[slot]];
  const int tile = tile_of(v, blockIdx.x - vb.tile_start[slot]);
  const int fused = v.fused;
  const int W = v.cam.W, H = v.cam.H;
  const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int ox, oy, lx, ly;
  warp_block<TW>(warp, lane, ox, oy, lx, ly);
  const int px = tx * TW + lx, py = ty * TH + ly;
  const bool inside = px < W && py < H;
  const long long npx = (long long)W * H, pix = (long long)py * W + px;
  const float scale = loss_scale(v, fused, dloss);
  float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
  float sv = 0.f, thr = -INFINITY;
  if (inside) {
    const float4 st = v.pix_a[pix];
    const float iN = 1.0f / (1.0f + v.pix_b[pix].x);
    const float dt = __ldg(v.Dt + pix);
    float g0, g1, g2, gD;
    upstream(v, pix, npx, st, dt, fused, lambda, scale, g0, g1, g2, gD);
    h = make_float4(g0 * iN, g1 * iN, g2 * iN, gD * iN);
    sv = (g0 * st.x + g1 * st.y + g2 * st.z + gD * st.w) * iN;
    if (g0 != 0.f || g1 != 0.f || g2 != 0.f || gD != 0.f) thr = depth_threshold(dt, eps);
  }
  s_h[tid] = h;
  s_s[tid] = make_float2(sv, thr);
  const uint2 r = v.tile_ranges[tile];
  uint32_t gi_next[KPT];
#pragma unroll
  for (int u = 0; u < KPT; ++u)
    gi_next[u] = r.x + u * NT + tid < r.y ? (uint32_t)v.keys[r.x + u * NT + tid] : 0u;
  const float wthr = warp_max(thr);
  const bool wdone = wthr == -INFINITY;  // no pixel of the warp has a gradient
  if (__syncthreads_and(wdone)) return;
  const float bx0 = (float)(tx * TW + ox), bx1 = bx0 + 7.0f;
  const float by0 = (float)(ty * TH + oy), by1 = by0 + 3.0f;
  const int blk = warp * 32;
  unsigned n_tested = 0, n_counted = 0;
  int pend = 0;  // lanes [0, pend) hold culled Gaussians waiting for a full group
  BwdGauss G = bwd_idle();
  for (uint32_t b = r.x; b < r.y; b += NB) {
    __syncthreads();  // the previous batch's records are no longer read
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
      const int k = u * NT + tid;
      const uint32_t gi = gi_next[u];
      gi_next[u] = b + NB + k < r.y ? (uint32_t)v.keys[b + NB + k] : 0u;
      if (b + k < r.y) {
        const float4* rr = v.rec + 4 * (size_t)gi;
        float4 B = rr[1];
        const float4 C = rr[2];
        B.y = 2.0f * B.y;
        s_a[k] = rr[0];
        s_b[k] = B;
        s_c[k] = C;
        s_e[k] = make_float2(C.w, rr[3].x);
        s_gi[k] = gi;
      }
    }
    __syncthreads();
    if (wdone) continue;
    const int nb = (int)min((uint32_t)NB, r.y - b);
    int cnt = 0;
    for (int j0 = 0; j0 < nb; j0 += 32) {
      const int j = j0 + lane;
      bool ok = false;
      if (j < nb) {
        const float4 A = s_a[j];
        const float2 E = s_e[j];
        ok = A.z < wthr && A.x + E.x >= bx0 && A.x - E.x <= bx1 && A.y + E.y >= by0 &&
             A.y - E.y <= by1;
        if (ok) {
          const float4 B = s_b[j];
          ok = ellipse_meets_rect(A.x, A.y, B.x, 0.5f * B.y, B.z, B.w, bx0, bx1, by0, by1);
        }
      }
      const unsigned ob = __ballot_sync(0xffffffffu, ok);
      if (ok) s_list[warp][cnt + __popc(ob & ((1u << lane) - 1u))] = (uint8_t)j;
      cnt += __popc(ob);
    }
    __syncwarp();
    // full groups: the waiting lanes keep their Gaussians, the others load
    int t0 = 0;
    while (pend + cnt - t0 >= 32) {
      if (lane >= pend) {
        const int j = s_list[warp][t0 + lane - pend];
        G = bwd_gauss<INSTR>(s_a[j], s_b[j], s_c[j], s_e[j], s_gi[j], bx0, by0);
      }
      bwd_flush<INSTR, FIXED>(v, G, true, blk, bx0, by0, s_h, s_s, dloss, n_tested, n_counted);
      t0 += 32 - pend;
      pend = 0;
    }
    // the rest waits
    if (lane >= pend && lane < pend + cnt - t0) {
      const int j = s_list[warp][t0 + lane - pend];
      G = bwd_gauss<INSTR>(s_a[j], s_b[j], s_c[j], s_e[j], s_gi[j], bx0, by0);
    }
    pend += cnt - t0;
  }
  if (pend > 0) {
    const bool has = lane < pend;
    if (!has) G = bwd_idle();
    bwd_flush<INSTR, FIXED>(v, G, has, blk, bx0, by0, s_h, s_s, dloss, n_tested, n_counted);
  }
  if (INSTR) add_counters(v, 2, n_tested, n_counted);
}

// ----------------------------------------------------- backward, alpha mode
// Transposing butterfly over a warp: the warp's sums of 10 per-lane values
// in 12 shuffles (a separate reduction per value takes 50).  At each level a
// lane keeps part of the values it carries, sends the rest to its partner
// and adds what the partner sent for its own part: 10 -> 5 (xor 16), 5 -> 3
// or 2 (xor 8), -> 2 or 1 (xor 4), -> 1 (xor 2), then the pair adds (xor 1).
// Returns the lane's sum and sets comp to its component (-1: none); lanes 2m
// and 2m + 1 hold the same one.  The order of the additions is fixed.
__device__ __forceinline__ float warp_sum10(const float (&v)[10], int lane, int& comp) {
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
  float a[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float r = __shfl_xor_sync(0xffffffffu, h4 ? v[i] : v[5 + i], 16);
    a[i] = (h4 ? v[5 + i] : v[i]) + r;
  }
  // h3 = 0 keeps a0..a2, h3 = 1 keeps a3, a4
  float b[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float send = h3 ? a[i] : (i < 2 ? a[3 + i] : 0.f);
    const float r = __shfl_xor_sync(0xffffffffu, send, 8);
    b[i] = h3 ? (i < 2 ? a[3 + i] + r : 0.f) : a[i] + r;
  }
  // h2 = 0 keeps b0, b1, h2 = 1 keeps b2
  float c[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h2 ? b[i] : (i == 0 ? b[2] : 0.f);
    const float r = __shfl_xor_sync(0xffffffffu, send, 4);
    c[i] = h2 ? (i == 0 ? b[2] + r : 0.f) : b[i] + r;
  }
  float d = (h1 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h1 ? c[0] : c[1], 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  const int ai = h3 ? (h2 ? -1 : 3 + (h1 ? 1 : 0)) : (h2 ? (h1 ? -1 : 2) : (h1 ? 1 : 0));
  comp = ai < 0 ? -1 : ai + (h4 ? 5 : 0);
  return d;
}

// list entries staged per round of the alpha backward (per-warp partials of
// NW x NB x 10 floats stay within 20 KB of shared memory)
template <int NT>
struct AlphaBatch {
  static constexpr int value = NT >= 256 ? 64 : NT;
};

// The front-to-back (alpha) backward: each pixel walks its list from its
// last contributing entry back to the first, undoing the forward's
// transmittance, T_j = T_{j+1} / (1 - alpha_j), and carrying the colour and
// depth composited behind j.  A warp owns an 8 x 4 pixel block and walks only
// the entries of the batch that can reach it (conservative ellipse test, in
// front of its depth threshold, before its last contributing entry): the
// skipped ones leave every pixel of the block unchanged.  Per entry the
// warp's 10 gradient sums come from warp_sum10, per (tile, Gaussian) pair
// the warps' sums are added in warp order.
template <int TW, int TH>
__global__ void __launch_bounds__(TW* TH) composite_bwd_alpha_kernel(const __grid_constant__ ViewBatch vb,
                                                                     float eps, float lambda,
                                                                     const float* dloss,
                                                                     int deterministic) {
  chain_wait();
  constexpr int NT = TW * TH;
  constexpr int NW = NT / 32;
  constexpr int NB = AlphaBatch<NT>::value;
  constexpr int NM = NB / 32;
  static_assert(NB <= NT && NM * 32 == NB, "one staged entry per thread at most");
  __shared__ float4 s_a[NB], s_b[NB], s_c[NB];
  __shared__ float2 s_e[NB];
  __shared__ float s_l2[NB];  // log2 sigma, as staged by the forward
  __shared__ uint32_t s_gi[NB];
  __shared__ float s_part[NW][NB][10];
  __shared__ uint32_t s_mask[NW][NM];
  __shared__ float s_tmp[NW];
  const int slot = batch_slot(vb.tile_start, vb.n, blockIdx.x);
  const ViewDev& v = vb.v[vb.order[slot]];
  const int tile = tile_of(v, blockIdx.x - vb.tile_start[slot]);
  const int fused = v.fused;
  const int W = v.cam.W, H = v.cam.H;
  const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int ox, oy, lx, ly;
  warp_block<TW>(warp, lane, ox, oy, lx, ly);
  const int px = tx * TW + lx, py = ty * TH + ly;
  const bool inside = px < W && py < H;
  const long long npx = (long long)W * H, pix = (long long)py * W + px;
  const float scale = loss_scale(v, fused, dloss);
  const uint2 r = v.tile_ranges[tile];
  // P: the upstream gradient dotted with the colour and depth composited
  // behind the current entry (T_end (C_t, D_t) at the start), so that
  // dL/dalpha_j = (g . c_j) T_j - P / (1 - alpha_j) and P grows by
  // (g . c_j) alpha_j T_j as the walk passes j
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, gD = 0.f, T = 1.f, thr = -INFINITY, P = 0.f;
  uint32_t mylast = r.x;
  if (inside) {
    const float4 st = v.pix_a[pix];
    const float4 sb = v.pix_b[pix];
    const float dt = __ldg(v.Dt + pix);
    upstream(v, pix, npx, st, dt, fused, lambda, scale, g0, g1, g2, gD);
    T = sb.x;
    mylast = min(max(__float_as_uint(sb.y), r.x), r.y);  // stays inside this tile's list
    thr = depth_threshold(dt, eps);
    P = T * (g0 * ld_col(v.Ct, pix, v.prec) + g1 * ld_col(v.Ct, npx + pix, v.prec) +
             g2 * ld_col(v.Ct, 2 * npx + pix, v.prec) + gD * dt);
    if (g0 == 0.f && g1 == 0.f && g2 == 0.f && gD == 0.f) mylast = r.x;
  }
  const float fpx = (float)px, fpy = (float)py;
  const float maxlast = block_max<NT>((float)(mylast - r.x), s_tmp);
  const uint32_t top = r.x + (uint32_t)maxlast;
  // this warp's block, last entry and depth threshold
  const float bx0 = (float)(tx * TW + ox), bx1 = bx0 + 7.0f;
  const float by0 = (float)(ty * TH + oy), by1 = by0 + 3.0f;
  const uint32_t wlast = __reduce_max_sync(0xffffffffu, mylast);
  const float wthr = warp_max(thr);
  for (uint32_t hi = top; hi > r.x; hi = hi > r.x + NB ? hi - NB : r.x) {
    const uint32_t lo = hi > r.x + NB ? hi - NB : r.x;
    const int nb = (int)(hi - lo);
    __syncthreads();
    if (tid < nb) {
      const uint32_t gi = (uint32_t)v.keys[lo + tid];
      const float4* rr = v.rec + 4 * (size_t)gi;
      float4 B = rr[1];
      B.y = 2.0f * B.y;
      const float4 A0 = rr[0], C = rr[2];
      s_a[tid] = A0;
      s_b[tid] = B;
      s_c[tid] = C;
      s_e[tid] = make_float2(C.w, rr[3].x);
      s_gi[tid] = gi;
      s_l2[tid] = __log2f(A0.w);
    }
    __syncthreads();
    // the batch's entries this warp walks
    uint32_t msk[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const int j = m * 32 + lane;
      bool ok = false;
      if (j < nb && lo + j < wlast) {
        const float4 A = s_a[j];
        const float2 E = s_e[j];
        ok = A.z < wthr && A.x + E.x >= bx0 && A.x - E.x <= bx1 && A.y + E.y >= by0 &&
             A.y - E.y <= by1;
        if (ok) {
          const float4 B = s_b[j];
          ok = ellipse_meets_rect(A.x, A.y, B.x, 0.5f * B.y, B.z, B.w, bx0, bx1, by0, by1);
        }
      }
      msk[m] = __ballot_sync(0xffffffffu, ok);
    }
#pragma unroll
    for (int m = NM - 1; m >= 0; --m) {
      uint32_t mm = msk[m], keep = 0u;
      while (mm) {
        const int jj = 31 - __clz(mm);
        mm &= ~(1u << jj);
        const int j = m * 32 + jj;
        float gv[10];
#pragma unroll
        for (int c = 0; c < 10; ++c) gv[c] = 0.f;
        bool contrib = false;
        if (lo + j < mylast) {
          const float4 A = s_a[j], B = s_b[j];
          const float dx = __fsub_rn(fpx, A.x), dy = __fsub_rn(fpy, A.y);
          const float q = quad_form(B.x, B.y, B.z, dx, dy);
          if (q <= B.w && A.z < thr) {
            const float4 C = s_c[j];
            // the forward's alpha, bit for bit, so that T_j = T_{j+1} / (1 - alpha_j)
            // undoes what the forward multiplied in
            const float raw = alpha_of(q, s_l2[j]);
            const bool clamped = raw > kAlphaMax;
            const float a = fminf(raw, kAlphaMax);
            const float ia = rcp_approx(1.0f - a);
            const float Tj = T * ia;
            const float aT = a * Tj;
            gv[6] = g0 * aT;
            gv[7] = g1 * aT;
            gv[8] = g2 * aT;
            gv[9] = gD * aT;
            const float gc = g0 * C.x + g1 * C.y + g2 * C.z + gD * A.z;
            const float dLda = gc * Tj - P * ia;
            P = fmaf(gc, aT, P);
            T = Tj;
            if (!clamped) {
              const float vv = dLda * a;
              const float cb = 0.5f * B.y;
              gv[0] = vv * (B.x * dx + cb * dy);
              gv[1] = vv * (cb * dx + B.z * dy);
              gv[2] = -0.5f * vv * dx * dx;
              gv[3] = -vv * dx * dy;
              gv[4] = -0.5f * vv * dy * dy;
              gv[5] = __fdividef(dLda * raw, A.w);  // dL/dsigma = dL/dalpha * G, G = alpha / sigma
            }
            contrib = true;
          }
        }
        if (__any_sync(0xffffffffu, contrib)) {
          int comp;
          const float t = warp_sum10(gv, lane, comp);
          if (comp >= 0 && !(lane & 1)) s_part[warp][j][comp] = t;
          keep |= 1u << jj;
        }
      }
      if (lane == 0) s_mask[warp][m] = keep;
    }
    __syncthreads();
    // fixed-order sum over the warps that walked the entry, then one write
    // per (tile, Gaussian) pair
    if (tid < nb) {
      float g[10];
#pragma unroll
      for (int c = 0; c < 10; ++c) g[c] = 0.f;
      bool any = false;
      for (int w = 0; w < NW; ++w) {
        if ((s_mask[w][tid >> 5] >> (tid & 31)) & 1u) {
          any = true;
#pragma unroll
          for (int c = 0; c < 10; ++c) g[c] += s_part[w][tid][c];
        }
      }
      if (any || deterministic) {
        long long ps = 0;
        if (deterministic) {
          const uint32_t gi = s_gi[tid];
          ps = pair_slot(v, gi, tx, ty, s_a[tid].x, s_a[tid].y, s_e[tid].x, s_e[tid].y);
        }
        store_grad2d(v, deterministic, ps, s_gi[tid], g);
      }
    }
  }
  if (deterministic) {
    for (uint32_t k = top + tid; k < r.y; k += NT) {
      const uint32_t gi = (uint32_t)v.keys[k];
      const float4 A = v.rec[4 * (size_t)gi], C = v.rec[4 * (size_t)gi + 2];
      zero_slot(v, pair_slot(v, gi, tx, ty, A.x, A.y, C.w, v.rec[4 * (size_t)gi + 3].x));
    }
  }
}

// The alpha backward, not deterministic: the walk of composite_bwd_alpha_kernel
// with the per-entry warp reduction replaced by a transpose through shared
// memory.  Each warp gathers the entries that can reach its 8 x 4 block, in
// walk order, into groups of 16; for a group,
//   1. pixel lanes walk its entries in order (the per-pixel transmittance
//      and composited colour behind each entry are sequential) and leave,
//      per (pixel, entry), w = (alpha T_j, dL/dalpha alpha) (zero where the
//      entry does not count, and the second zero where alpha is clamped) in
//      shared memory;
//   2. two lanes per entry (rows 0-1 and 2-3 of the block) walk the pixels
//      and sum, from w and each pixel's upstream gradient, the moments of
//      grad2d_of (as the OIT backward does); the pair adds its halves and the
//      entry's Gaussian's block gradient goes to grad2d with vector atomics.
// w is stored at [pixel][entry ^ (pixel mod 16)], so both phases touch
// distinct banks.
constexpr int kAlphaGroup = 16;

template <int NT>
struct AlphaCarryBatch {
  static constexpr int value = NT >= 256 ? 64 : 2 * NT;
};

template <int TW, int TH>
__global__ void __launch_bounds__(TW* TH)
    composite_bwd_alpha_carry_kernel(const __grid_constant__ ViewBatch vb, float eps, float lambda,
                                     const float* dloss) {
  chain_wait();
  constexpr int NT = TW * TH;
  constexpr int NW = NT / 32;
  constexpr int NB = AlphaCarryBatch<NT>::value;
  constexpr int NM = NB / 32;
  constexpr int G = kAlphaGroup;
  constexpr int KPT = (NB + NT - 1) / NT;  // entries staged per thread
  static_assert(NM * 32 == NB && KPT * NT >= NB, "whole chunks of 32 entries");
  __shared__ float4 s_a[NB], s_b[NB], s_c[NB];
  __shared__ float2 s_e[NB];
  __shared__ uint32_t s_gi[NB];
  __shared__ float4 s_pg[NT];  // each pixel's upstream gradient, by warp block
  // groups: (mx, my, d, log2 sigma), (a, 2b, c, qmax), (r, g, b, sigma), (list index, gi)
  __shared__ float4 s_ga[NW][G], s_gb[NW][G], s_gc[NW][G];
  __shared__ uint2 s_gk[NW][G];
  __shared__ float2 s_w[NW][32][G];
  __shared__ float s_tmp[NW];
  const int slot = batch_slot(vb.tile_start, vb.n, blockIdx.x);
  const ViewDev& v = vb.v[vb.order[slot]];
  const int tile = tile_of(v, blockIdx.x - vb.tile_start[slot]);
  const int fused = v.fused;
  const int W = v.cam.W, H = v.cam.H;
  const int tx = tile % v.tiles_x, ty = tile / v.tiles_x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int ox, oy, lx, ly;
  warp_block<TW>(warp, lane, ox, oy, lx, ly);
  const int px = tx * TW + lx, py = ty * TH + ly;
  const bool inside = px < W && py < H;
  const long long npx = (long long)W * H, pix = (long long)py * W + px;
  const float scale = loss_scale(v, fused, dloss);
  const uint2 r = v.tile_ranges[tile];
  // P: the upstream gradient dotted with the colour and depth composited
  // behind the current entry (T_end (C_t, D_t) at the start), so that
  // dL/dalpha_j = (g . c_j) T_j - P / (1 - alpha_j) and P grows by
  // (g . c_j) alpha_j T_j as the walk passes j
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, gD = 0.f, T = 1.f, thr = -INFINITY, P = 0.f;
  uint32_t mylast = r.x;
  if (inside) {
    const float4 st = v.pix_a[pix];
    const float4 sb = v.pix_b[pix];
    const float dt = __ldg(v.Dt + pix);
    upstream(v, pix, npx, st, dt, fused, lambda, scale, g0, g1, g2, gD);
    T = sb.x;
    mylast = min(max(__float_as_uint(sb.y), r.x), r.y);  // stays inside this tile's list
    thr = depth_threshold(dt, eps);
    P = T * (g0 * ld_col(v.Ct, pix, v.prec) + g1 * ld_col(v.Ct, npx + pix, v.prec) +
             g2 * ld_col(v.Ct, 2 * npx + pix, v.prec) + gD * dt);
    if (g0 == 0.f && g1 == 0.f && g2 == 0.f && gD == 0.f) mylast = r.x;
  }
  s_pg[tid] = make_float4(g0, g1, g2, gD);
  const float maxlast = block_max<NT>((float)(mylast - r.x), s_tmp);
  const uint32_t top = r.x + (uint32_t)maxlast;
  const float bx0 = (float)(tx * TW + ox), bx1 = bx0 + 7.0f;
  const float by0 = (float)(ty * TH + oy), by1 = by0 + 3.0f;
  const uint32_t wlast = __reduce_max_sync(0xffffffffu, mylast);
  const float wthr = warp_max(thr);
  float4* __restrict__ ga = s_ga[warp];
  float4* __restrict__ gb = s_gb[warp];
  float4* __restrict__ gc = s_gc[warp];
  uint2* __restrict__ gk = s_gk[warp];
  float2(*__restrict__ w)[G] = s_w[warp];
  const float4* __restrict__ pg = s_pg + warp * 32;
  const int ge = lane & (G - 1), half = lane >> 4;  // phase 2: entry, rows 2 half .. 2 half + 1

  // one group of n entries: phase 1 (pixel lanes), then phase 2 (entry lanes)
  auto run_group = [&](int n) {
    __syncwarp();
    const float fpx = (float)px, fpy = (float)py;
    const int sw = lane & (G - 1);
    // branch-free: an entry that does not count takes alpha = 0, which
    // leaves T (T / 1) and the sums behind it (+ 0) exactly as they are
#pragma unroll 4
    for (int e = 0; e < n; ++e) {
      const float4 A = ga[e], B = gb[e], C = gc[e];
      const uint2 K = gk[e];
      const float dx = __fsub_rn(fpx, A.x), dy = __fsub_rn(fpy, A.y);
      const float q = quad_form(B.x, B.y, B.z, dx, dy);
      const bool counted = K.x < mylast && q <= B.w && A.z < thr;
      // the forward's alpha, bit for bit (see composite_bwd_alpha_kernel)
      const float raw = alpha_of(q, A.w);
      const float a = counted ? fminf(raw, kAlphaMax) : 0.0f;
      const float ia = rcp_approx(1.0f - a);
      const float Tj = T * ia;
      const float aT = a * Tj;
      const float gc = g0 * C.x + g1 * C.y + g2 * C.z + gD * A.z;
      const float dLda = gc * Tj - P * ia;
      P = fmaf(gc, aT, P);
      T = Tj;
      const float vv = counted && !(raw > kAlphaMax) ? dLda * a : 0.0f;
      w[lane][e ^ sw] = make_float2(aT, vv);
    }
    __syncwarp();
    const float4 A = ga[ge];
    float dcr = 0.f, dcg = 0.f, dcb = 0.f, dd = 0.f, sa = 0.f;
    float sx = 0.f, sy = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f;
#pragma unroll
    for (int k2 = 0; k2 < 2; ++k2) {
      const int ky = 2 * half + k2;
      const float dy = __fsub_rn(by0 + (float)ky, A.y);
      float ra = 0.f, rx = 0.f, rxx = 0.f;
#pragma unroll
      for (int kx = 0; kx < 8; ++kx) {
        const int p = ky * 8 + kx;
        const float2 wv = w[p][ge ^ (p & (G - 1))];
        const float4 hh = pg[p];
        dcr = fmaf(wv.x, hh.x, dcr);
        dcg = fmaf(wv.x, hh.y, dcg);
        dcb = fmaf(wv.x, hh.z, dcb);
        dd = fmaf(wv.x, hh.w, dd);
        const float dx = __fsub_rn(bx0 + (float)kx, A.x);
        ra += wv.y;
        const float tx_ = wv.y * dx;
        rx += tx_;
        rxx = fmaf(tx_, dx, rxx);
      }
      sa += ra;
      sx += rx;
      sxx += rxx;
      sy = fmaf(ra, dy, sy);
      sxy = fmaf(rx, dy, sxy);
      syy = fmaf(ra * dy, dy, syy);
    }
    float m[10] = {dcr, dcg, dcb, dd, sa, sx, sy, sxx, sxy, syy};
#pragma unroll
    for (int c = 0; c < 10; ++c) m[c] += __shfl_xor_sync(0xffffffffu, m[c], 16);
    if (half == 0 && ge < n) {
      const float4 B = gb[ge], C = gc[ge];
      float g[10];
      grad2d_of(m, B.x, 0.5f * B.y, B.z, C.w, g);
      store_grad2d(v, 0, 0, gk[ge].y, g);
    }
    __syncwarp();
  };

  int cnt = 0;  // entries in this warp's open group
  // batches from the back of the list; a last round without entries runs
  // the open group (one call site keeps the kernel's code small)
  // the first batch's keys (the next batch's are fetched while this one is
  // walked)
  uint32_t gi_next[KPT];
  {
    const uint32_t lo0 = top > r.x + NB ? top - NB : r.x;
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
      const uint32_t k = lo0 + u * NT + tid;
      gi_next[u] = u * NT + tid < NB && k < top ? (uint32_t)v.keys[k] : 0u;
    }
  }
  for (uint32_t hi = top;; hi = hi > r.x + NB ? hi - NB : r.x) {
    const bool flush = hi <= r.x;
    const uint32_t lo = hi > r.x + NB ? hi - NB : r.x;
    const int nb = (int)(hi - lo);
    const uint32_t lo2 = lo > r.x + NB ? lo - NB : r.x;  // the next batch: [lo2, lo)
    __syncthreads();
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
      const int t = u * NT + tid;
      const uint32_t gi = gi_next[u];
      gi_next[u] = t < NB && lo2 + t < lo ? (uint32_t)v.keys[lo2 + t] : 0u;
      if (t < nb) {
        const float4* rr = v.rec + 4 * (size_t)gi;
        float4 B = rr[1];
        B.y = 2.0f * B.y;
        const float4 C = rr[2];
        s_a[t] = rr[0];
        s_b[t] = B;
        s_c[t] = C;
        s_e[t] = make_float2(C.w, rr[3].x);
        s_gi[t] = gi;
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int m = flush ? 0 : NM - 1; m >= 0; --m) {
      const int j = m * 32 + lane;
      bool ok = false;
      if (j < nb && lo + j < wlast) {
        const float4 A = s_a[j];
        const float2 E = s_e[j];
        ok = A.z < wthr && A.x + E.x >= bx0 && A.x - E.x <= bx1 && A.y + E.y >= by0 &&
             A.y - E.y <= by1;
        if (ok) {
          const float4 B = s_b[j];
          ok = ellipse_meets_rect(A.x, A.y, B.x, 0.5f * B.y, B.z, B.w, bx0, bx1, by0, by1);
        }
      }
      uint32_t mask = __ballot_sync(0xffffffffu, ok);
      while (mask || (flush && cnt > 0)) {
        // the highest (G - cnt) entries of the mask join the group, highest first
        uint32_t take = mask;
        for (int extra = __popc(mask) - (G - cnt); extra > 0; --extra) take &= take - 1u;
        if ((take >> lane) & 1u) {
          const int e = cnt + __popc(take >> lane) - 1;
          const float4 A = s_a[j], B = s_b[j], C = s_c[j];
          ga[e] = make_float4(A.x, A.y, A.z, __log2f(A.w));
          gb[e] = B;
          gc[e] = make_float4(C.x, C.y, C.z, A.w);
          gk[e] = make_uint2(lo + j, s_gi[j]);
        }
        cnt += __popc(take);
        mask &= ~take;
        if (cnt == G || flush) {
          run_group(cnt);
          cnt = 0;
        }
      }
    }
    if (flush) break;
  }
}

// Deterministic mode, before the backward: the first pair_grads slot of each
// Gaussian, its rectangle's tile count after those of the Gaussians placed
// before it (warp prefix sums, one atomic per warp on the view's counter,
// scalars[5], zero on entry).  The placement varies with the atomics' order;
// the sums do not, as each Gaussian's slots are summed in its own tile order.
// If the forward overflowed the pair capacity, some lists lost pairs whose
// slots nothing writes: then the Gaussian's slots are zeroed here first.
__global__ void __launch_bounds__(256) pair_base_kernel(const __grid_constant__ ViewBatch vb,
                                                        int M, const int* status) {
  chain_wait();
  const ViewDev& v = vb.v[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
  int cnt = 0;
  if (i < M) {
    const float4 A = v.rec[4 * (size_t)i], C = v.rec[4 * (size_t)i + 2];
    int x0, x1, y0, y1;
    if (record_rect(A.x, A.y, C.w, v.rec[4 * (size_t)i + 3].x, v.cam.W, v.cam.H, x0, x1, y0, y1))
      cnt = (x1 / v.tw - x0 / v.tw + 1) * (y1 / v.th - y0 / v.th + 1);
  }
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(reinterpret_cast<uint32_t*>(v.scalars + 5), (uint32_t)incl);
  base = __shfl_sync(0xffffffffu, base, 31);
  if (i >= M) return;
  const uint32_t first = base + (uint32_t)(incl - cnt);
  v.pair_base[i] = first;
  if (*status == GPS_ERR_CAPACITY)
    for (int k = 0; k < cnt; ++k) zero_slot(v, (long long)first + k);
}

// Deterministic mode: per Gaussian, sum its pair slots in row-major tile
// order (contiguous from pair_base).  Block row blockIdx.y: view.
__global__ void __launch_bounds__(256) gather_pair_grads_kernel(const __grid_constant__ ViewBatch vb,
                                                                int M) {
  chain_wait();
  const ViewDev& v = vb.v[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const float4 A = v.rec[4 * (size_t)i], C = v.rec[4 * (size_t)i + 2], E = v.rec[4 * (size_t)i + 3];
  float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0;
  int x0, x1, y0, y1;
  if (record_rect(A.x, A.y, C.w, E.x, v.cam.W, v.cam.H, x0, x1, y0, y1)) {
    const int cnt = (x1 / v.tw - x0 / v.tw + 1) * (y1 / v.th - y0 / v.th + 1);
    const long long first = v.pair_base[i];
    for (int k = 0; k < cnt && first + k < v.pair_slots; ++k) {
      const float4* p = v.pair_grads + 3 * (first + k);
      const float4 a = p[0], b = p[1], c = p[2];
      s0.x += a.x; s0.y += a.y; s0.z += a.z; s0.w += a.w;
      s1.x += b.x; s1.y += b.y; s1.z += b.z; s1.w += b.w;
      s2.x += c.x; s2.y += c.y;
    }
  }
  float4* o = v.grad2d + 3 * (size_t)i;
  o[0] = s0;
  o[1] = s1;
  o[2] = s2;
}

// ------------------------------------------- backward, per-Gaussian schedule
// The paper's sort-free backward (Sec. 3.1, App. B): threads work per
// Gaussian, over the pixels its support can reach, and accumulate its
// gradient privately, so no atomics are needed.  Here one warp takes one
// (view, Gaussian) and walks the Gaussian's pixel rectangle in groups of 32
// pixels (every lane runs the same number of iterations whatever the
// Gaussian's size: the fixed-size groups of App. B), then reduces its 10
// moments with shuffles in a fixed order and writes the 2D gradient once.
//
// Per pixel it needs dL/dC* / N, dL/dD* / N, sum dL/d(C*, D*) (C*, D*) / N and
// the depth threshold (-inf for pixels without gradient), precomputed here:
__global__ void __launch_bounds__(256) bwd_pixel_terms_kernel(const __grid_constant__ ViewBatch vb,
                                                              float eps, float lambda,
                                                              const float* dloss) {
  chain_wait();
  const ViewDev& v = vb.v[blockIdx.y];
  const int W = v.cam.W, H = v.cam.H;
  const long long npx = (long long)W * H;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npx) return;
  const float scale = loss_scale(v, v.fused, dloss);
  const float4 st = v.pix_a[pix];
  const float iN = 1.0f / (1.0f + v.pix_b[pix].x);
  const float dt = __ldg(v.Dt + pix);
  float g0, g1, g2, gD;
  upstream(v, pix, npx, st, dt, v.fused, lambda, scale, g0, g1, g2, gD);
  const float sv = (g0 * st.x + g1 * st.y + g2 * st.z + gD * st.w) * iN;
  const bool any = g0 != 0.f || g1 != 0.f || g2 != 0.f || gD != 0.f;
  v.pix_g[2 * pix] = make_float4(g0 * iN, g1 * iN, g2 * iN, gD * iN);
  v.pix_g[2 * pix + 1] = make_float4(sv, any ? depth_threshold(dt, eps) : -INFINITY, 0.f, 0.f);
}

template <bool INSTR>
__global__ void __launch_bounds__(256) composite_bwd_per_gaussian_kernel(
    const __grid_constant__ ViewBatch vb, int M) {
  chain_wait();
  const ViewDev& v = vb.v[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gi = blockIdx.x * 8 + warp;
  if (gi >= M) return;  // warp-uniform
  const float4* rr = v.rec + 4 * (size_t)gi;
  const float4 A = rr[0], B = rr[1], C = rr[2], E = rr[3];
  float4* o = v.grad2d + 3 * (size_t)gi;
  int x0, x1, y0, y1;
  if (!record_rect(A.x, A.y, C.w, E.x, v.cam.W, v.cam.H, x0, x1, y0, y1)) {
    if (lane == 0) o[0] = o[1] = o[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const int W = v.cam.W, w = x1 - x0 + 1, n = w * (y1 - y0 + 1);
  const float inv_w = 1.0f / (float)w;
  const float mx = A.x, my = A.y, d = A.z, lns = __log2f(A.w);
  const float ca = B.x, b2 = 2.0f * B.y, cc = B.z, qmax = B.w;
  float m[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  unsigned n_tested = 0, n_counted = 0;
  for (int p = lane; p < n; p += 32) {
    // pixel p of the rectangle, row-major (a float quotient, corrected)
    int ky = __float2int_rd(((float)p + 0.5f) * inv_w);
    int kx = p - ky * w;
    if (kx < 0) { --ky; kx += w; }
    if (kx >= w) { ++ky; kx -= w; }
    const int x = x0 + kx, y = y0 + ky;
    const long long pix = (long long)y * W + x;
    const float4 hh = v.pix_g[2 * pix];
    const float2 ss = *reinterpret_cast<const float2*>(v.pix_g + 2 * pix + 1);
    const float dx = __fsub_rn((float)x, mx), dy = __fsub_rn((float)y, my);
    const float q = quad_form(ca, b2, cc, dx, dy);
    const bool counted = q <= qmax && d < ss.y;
    if (INSTR) {
      ++n_tested;
      n_counted += counted;
    }
    const float al = counted ? alpha_of(q, lns) : 0.0f;
    m[0] = fmaf(al, hh.x, m[0]);
    m[1] = fmaf(al, hh.y, m[1]);
    m[2] = fmaf(al, hh.z, m[2]);
    m[3] = fmaf(al, hh.w, m[3]);
    const float dLda = fmaf(hh.x, C.x, fmaf(hh.y, C.y, fmaf(hh.z, C.z, fmaf(hh.w, d, -ss.x))));
    const float vv = dLda * al;
    m[4] += vv;
    const float tx = vv * dx, ty = vv * dy;
    m[5] += tx;
    m[6] += ty;
    m[7] = fmaf(tx, dx, m[7]);
    m[8] = fmaf(tx, dy, m[8]);
    m[9] = fmaf(ty, dy, m[9]);
  }
  if (INSTR) add_counters(v, 2, n_tested, n_counted);
#pragma unroll
  for (int c = 0; c < 10; ++c) m[c] = warp_sum(m[c]);
  if (lane == 0) {
    const float cb = B.y;
    o[0] = make_float4(ca * m[5] + cb * m[6], cb * m[5] + cc * m[6], -0.5f * m[7], -m[8]);
    o[1] = make_float4(-0.5f * m[9], m[4] / A.w, m[0], m[1]);
    o[2] = make_float4(m[2], m[3], 0.f, 0.f);
  }
}

cudaError_t launch_composite_bwd_per_gaussian(const ViewBatch& vb, int M, float eps, float lambda,
                                              const float* dloss, int instr, cudaStream_t st) {
  int max_px = 0;
  for (int k = 0; k < vb.n; ++k) max_px = max(max_px, vb.v[k].cam.W * vb.v[k].cam.H);
  launch_chained(bwd_pixel_terms_kernel, dim3((max_px + 255) / 256, vb.n), dim3(256), 0, st,
      vb, eps, lambda, dloss);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || M <= 0) return e;
  if (instr)
    launch_chained(composite_bwd_per_gaussian_kernel<true>, dim3((M + 7) / 8, vb.n), dim3(256), 0, st,
        vb, M);
  else
    launch_chained(composite_bwd_per_gaussian_kernel<false>, dim3((M + 7) / 8, vb.n), dim3(256), 0, st,
        vb, M);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
template <int TW, int TH>
static cudaError_t fwd_tw(const ViewBatch& vb, float eps, int mode, int has_tgt, int instr,
                          int sorted, cudaStream_t st) {
  const int items = vb.tile_start[vb.n];
  if (items <= 0) return cudaSuccess;
  if (mode == GPS_BLEND_OIT) {
    if (instr)
      launch_chained(composite_fwd_oit2_kernel<TW, TH, true>, dim3(items), dim3(TW * TH / 2), 0, st,
          vb, eps, has_tgt, sorted);
    else
      launch_chained(composite_fwd_oit2_kernel<TW, TH, false>, dim3(items), dim3(TW * TH / 2), 0, st,
          vb, eps, has_tgt, sorted);
  } else {
    if (instr)
      launch_chained(composite_fwd_alpha2_kernel<TW, TH, true>, dim3(items), dim3(TW * TH / 2), 0, st,
          vb, eps, has_tgt);
    else
      launch_chained(composite_fwd_alpha2_kernel<TW, TH, false>, dim3(items), dim3(TW * TH / 2), 0, st,
          vb, eps, has_tgt);
  }
  return cudaGetLastError();
}

template <int TW, int TH>
static cudaError_t bwd_tw(const ViewBatch& vb, float eps, float lambda, const float* dloss, int mode,
                          int det, int instr, int sorted, cudaStream_t st) {
  const int items = vb.tile_start[vb.n];
  if (items <= 0) return cudaSuccess;
  // the carry-over walk: sort-free lists, or deterministic mode's fixed-point sums
  if (mode == GPS_BLEND_OIT && ((!det && !sorted) || vb.v[0].grad_fixed)) {
    const bool fixed = vb.v[0].grad_fixed != nullptr;
    if (instr && fixed)
      launch_chained(composite_bwd_oit_carry_kernel<TW, TH, true, true>, dim3(items), dim3(TW * TH),
          0, st, vb, eps, lambda, dloss);
    else if (instr)
      launch_chained(composite_bwd_oit_carry_kernel<TW, TH, true, false>, dim3(items), dim3(TW * TH),
          0, st, vb, eps, lambda, dloss);
    else if (fixed)
      launch_chained(composite_bwd_oit_carry_kernel<TW, TH, false, true>, dim3(items), dim3(TW * TH),
          0, st, vb, eps, lambda, dloss);
    else
      launch_chained(composite_bwd_oit_carry_kernel<TW, TH, false, false>, dim3(items), dim3(TW * TH),
          0, st, vb, eps, lambda, dloss);
  } else if (mode == GPS_BLEND_OIT) {
    if (instr)
      launch_chained(composite_bwd_oit_kernel<TW, TH, true>, dim3(items), dim3(TW * TH), 0, st,
          vb, eps, lambda, dloss, det, sorted);
    else
      launch_chained(composite_bwd_oit_kernel<TW, TH, false>, dim3(items), dim3(TW * TH), 0, st,
          vb, eps, lambda, dloss, det, sorted);
  } else if (det) {
    launch_chained(composite_bwd_alpha_kernel<TW, TH>, dim3(items), dim3(TW * TH), 0, st,
        vb, eps, lambda, dloss, det);
  } else {
    launch_chained(composite_bwd_alpha_carry_kernel<TW, TH>, dim3(items), dim3(TW * TH), 0, st,
        vb, eps, lambda, dloss);
  }
  return cudaGetLastError();
}

cudaError_t launch_composite_fwd(const ViewBatch& vb, int tw, int th, float eps, int mode,
                                 int has_tgt, int instr, int sorted, cudaStream_t st) {
  if (tw == 16 && th == 16) return fwd_tw<16, 16>(vb, eps, mode, has_tgt, instr, sorted, st);
  if (tw == 16 && th == 8) return fwd_tw<16, 8>(vb, eps, mode, has_tgt, instr, sorted, st);
  if (tw == 8 && th == 8) return fwd_tw<8, 8>(vb, eps, mode, has_tgt, instr, sorted, st);
  if (tw == 32 && th == 8) return fwd_tw<32, 8>(vb, eps, mode, has_tgt, instr, sorted, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_composite_bwd(const ViewBatch& vb, int tw, int th, float eps, float lambda,
                                 const float* dloss, int mode, int det, int instr, int sorted,
                                 cudaStream_t st) {
  if (tw == 16 && th == 16) return bwd_tw<16, 16>(vb, eps, lambda, dloss, mode, det, instr, sorted, st);
  if (tw == 16 && th == 8) return bwd_tw<16, 8>(vb, eps, lambda, dloss, mode, det, instr, sorted, st);
  if (tw == 8 && th == 8) return bwd_tw<8, 8>(vb, eps, lambda, dloss, mode, det, instr, sorted, st);
  if (tw == 32 && th == 8) return bwd_tw<32, 8>(vb, eps, lambda, dloss, mode, det, instr, sorted, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_finalize_loss(const ViewBatch& vb, float lambda, float* loss, int first,
                                 cudaStream_t st) {
  launch_chained(finalize_loss_kernel, dim3(1), dim3(256), 0, st, vb, lambda, loss, first);
  return cudaGetLastError();
}

cudaError_t launch_pair_base(const ViewBatch& vb, int M, const int* status, cudaStream_t st) {
  launch_chained(pair_base_kernel, dim3((M + 255) / 256, vb.n), dim3(256), 0, st, vb, M, status);
  return cudaGetLastError();
}

cudaError_t launch_upstream_max(const ViewBatch& vb, float eps, float lambda, const float* dloss,
                                cudaStream_t st) {
  int max_px = 0;
  for (int k = 0; k < vb.n; ++k) max_px = max(max_px, vb.v[k].cam.W * vb.v[k].cam.H);
  // about two blocks per SM, each striding over its view's pixels
  const int blocks = max(1, min((max_px + 255) / 256, 296));
  launch_chained(upstream_max_kernel, dim3(blocks, vb.n), dim3(256), 0, st, vb, eps, lambda, dloss);
  return cudaGetLastError();
}

cudaError_t launch_fixed_to_grad2d(const ViewBatch& vb, int M, const float* dloss,
                                   cudaStream_t st) {
  launch_chained(fixed_to_grad2d_kernel, dim3((M + 255) / 256, vb.n), dim3(256), 0, st, vb, M,
                 dloss);
  return cudaGetLastError();
}

cudaError_t launch_gather_pair_grads(const ViewBatch& vb, int M, cudaStream_t st) {
  launch_chained(gather_pair_grads_kernel, dim3((M + 255) / 256, vb.n), dim3(256), 0, st, vb, M);
  return cudaGetLastError();
}

}  // namespace gps
