// Projection of 3D Gaussians to 2D conics (Sec. 3.1, "following 3DGS") and its
// adjoint.  One thread per Gaussian; parameters are read once (56 B) and one
// 64-byte record is written.  The forward also builds its block's histogram of
// super-tiles touched and reserves the block's ranges (first half of the binning).
#include <cuda_runtime.h>

#include <cmath>

#include "adam.cuh"
#include "gps_common.cuh"
#include "sh.cuh"

namespace gps {

cudaError_t launch_adam_step_advance(int* device_step, cudaStream_t st);  // adam.cu

struct Params {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* logits;
  const float* rgb;
  const float* sh;  // [M][K][3], K = sh_coeffs(sh_degree); null when sh_degree = 0
  int sh_degree;
};

// SH rows of a block's Gaussians are staged in shared memory: the global
// rows (3K floats, 12 K bytes) are read and written with consecutive threads
// on consecutive floats, and each thread then works on its own row at an odd
// word stride, which keeps the per-thread accesses free of bank conflicts.
template <int DEG>
struct ShRows {
  static constexpr int K = sh_coeffs(DEG);
  static constexpr int K3 = 3 * K;
  static constexpr int STRIDE = K3 | 1;
};

constexpr int kProjThreads = 256;  // block size of both projection kernels

// rows [base, base + n) of a [M][K3] array -> s[r * STRIDE + c].  Each thread
// issues its K3 loads before the first store, so they are in flight together.
template <int DEG>
__device__ __forceinline__ void stage_rows(const float* __restrict__ g, long long base, int n,
                                           float* s) {
  using R = ShRows<DEG>;
  const float* src = g + base * R::K3;
  const int total = n * R::K3;
  float v[R::K3];
#pragma unroll
  for (int j = 0; j < R::K3; ++j) {
    const int e = j * kProjThreads + threadIdx.x;
    v[j] = e < total ? __ldg(src + e) : 0.0f;
  }
#pragma unroll
  for (int j = 0; j < R::K3; ++j) {
    const int e = j * kProjThreads + threadIdx.x;
    const int r = e / R::K3;
    if (e < total) s[r * R::STRIDE + (e - r * R::K3)] = v[j];
  }
}

// dst rows [base, base + n) += s rows, loads batched as in stage_rows.
template <int DEG>
__device__ __forceinline__ void add_rows(float* __restrict__ g, long long base, int n,
                                         const float* s) {
  using R = ShRows<DEG>;
  float* dst = g + base * R::K3;
  const int total = n * R::K3;
  float v[R::K3];
#pragma unroll
  for (int j = 0; j < R::K3; ++j) {
    const int e = j * kProjThreads + threadIdx.x;
    v[j] = e < total ? dst[e] : 0.0f;
  }
#pragma unroll
  for (int j = 0; j < R::K3; ++j) {
    const int e = j * kProjThreads + threadIdx.x;
    const int r = e / R::K3;
    if (e < total) dst[e] = v[j] + s[r * R::STRIDE + (e - r * R::K3)];
  }
}

// Colour of Gaussian i seen from the camera centre (Sec. 3.1, SH of degree
// DEG over rgb); f: its coefficient row (K3 floats).
template <int DEG>
__device__ __forceinline__ float3 view_colour(const Params& P, int i, const Cam& c,
                                              const float* f) {
  const float* col = P.rgb + 3 * (size_t)i;
  float3 out = make_float3(col[0], col[1], col[2]);
  if constexpr (DEG > 0) {
    const float* p = P.means + 3 * (size_t)i;
    const float vx = p[0] - c.t[0], vy = p[1] - c.t[1], vz = p[2] - c.t[2];
    const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
    float Y[kShMaxCoeffs];
    sh_eval(DEG, vx * inv, vy * inv, vz * inv, Y);
#pragma unroll
    for (int k = 0; k < ShRows<DEG>::K; ++k) {
      out.x += Y[k] * f[3 * k];
      out.y += Y[k] * f[3 * k + 1];
      out.z += Y[k] * f[3 * k + 2];
    }
  }
  return out;
}

// Adjoint of view_colour given dL/dc = g: adds Y_k(d) g to the coefficient
// gradient row dsh and returns the mean's gradient through the direction,
// (I - d d^T) / |v| sum_k grad Y_k (f_k . g).
template <int DEG>
__device__ __forceinline__ float3 view_colour_adjoint(const Params& P, int i, const Cam& c,
                                                      float3 g, const float* f, float* dsh) {
  const float* p = P.means + 3 * (size_t)i;
  const float vx = p[0] - c.t[0], vy = p[1] - c.t[1], vz = p[2] - c.t[2];
  const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
  const float dx = vx * inv, dy = vy * inv, dz = vz * inv;
  float Y[kShMaxCoeffs], w[kShMaxCoeffs];
  sh_eval(DEG, dx, dy, dz, Y);
#pragma unroll
  for (int k = 0; k < kShMaxCoeffs; ++k) {
    if (k < ShRows<DEG>::K) {
      dsh[3 * k] += Y[k] * g.x;
      dsh[3 * k + 1] += Y[k] * g.y;
      dsh[3 * k + 2] += Y[k] * g.z;
      w[k] = f[3 * k] * g.x + f[3 * k + 1] * g.y + f[3 * k + 2] * g.z;
    } else {
      w[k] = 0.0f;
    }
  }
  const float3 gd = sh_grad_dot(DEG, dx, dy, dz, w);
  const float dot = gd.x * dx + gd.y * dy + gd.z * dz;
  return make_float3((gd.x - dx * dot) * inv, (gd.y - dy * dot) * inv, (gd.z - dz * dot) * inv);
}

struct ProjState {
  bool vis;
  float qn[4], qnorm, Rg[9], s[3], Sig[6];  // Sig: xx, xy, xz, yy, yz, zz
  float tc[3], txp, typ;
  bool clx, cly;
  float T[6], S2xx, S2xy, S2yy, det, ca, cb, cc, mx, my, sig, qmax, ex, ey;
};

__device__ __forceinline__ void project_gaussian(const Params& P, int i, const Cam& c, float near_,
                                                 ProjState& o) {
  o.vis = false;
  const float4 q = *reinterpret_cast<const float4*>(P.quats + 4 * (size_t)i);
  o.qnorm = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float inv = 1.0f / o.qnorm;
  const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  o.qn[0] = w; o.qn[1] = x; o.qn[2] = y; o.qn[3] = z;
  float* Rg = o.Rg;
  Rg[0] = 1.f - 2.f * (y * y + z * z); Rg[1] = 2.f * (x * y - w * z); Rg[2] = 2.f * (x * z + w * y);
  Rg[3] = 2.f * (x * y + w * z); Rg[4] = 1.f - 2.f * (x * x + z * z); Rg[5] = 2.f * (y * z - w * x);
  Rg[6] = 2.f * (x * z - w * y); Rg[7] = 2.f * (y * z + w * x); Rg[8] = 1.f - 2.f * (x * x + y * y);
  const float* ls = P.log_scales + 3 * (size_t)i;
  o.s[0] = expf(ls[0]); o.s[1] = expf(ls[1]); o.s[2] = expf(ls[2]);
  const float s0 = o.s[0] * o.s[0], s1 = o.s[1] * o.s[1], s2 = o.s[2] * o.s[2];
  // Sigma = Rg diag(s^2) Rg^T (symmetric, 6 entries)
  o.Sig[0] = Rg[0] * Rg[0] * s0 + Rg[1] * Rg[1] * s1 + Rg[2] * Rg[2] * s2;
  o.Sig[1] = Rg[0] * Rg[3] * s0 + Rg[1] * Rg[4] * s1 + Rg[2] * Rg[5] * s2;
  o.Sig[2] = Rg[0] * Rg[6] * s0 + Rg[1] * Rg[7] * s1 + Rg[2] * Rg[8] * s2;
  o.Sig[3] = Rg[3] * Rg[3] * s0 + Rg[4] * Rg[4] * s1 + Rg[5] * Rg[5] * s2;
  o.Sig[4] = Rg[3] * Rg[6] * s0 + Rg[4] * Rg[7] * s1 + Rg[5] * Rg[8] * s2;
  o.Sig[5] = Rg[6] * Rg[6] * s0 + Rg[7] * Rg[7] * s1 + Rg[8] * Rg[8] * s2;
  const float* p = P.means + 3 * (size_t)i;
  const float d0 = p[0] - c.t[0], d1 = p[1] - c.t[1], d2 = p[2] - c.t[2];
  o.tc[0] = c.R[0] * d0 + c.R[3] * d1 + c.R[6] * d2;
  o.tc[1] = c.R[1] * d0 + c.R[4] * d1 + c.R[7] * d2;
  o.tc[2] = c.R[2] * d0 + c.R[5] * d1 + c.R[8] * d2;
  o.sig = 1.0f / (1.0f + expf(-P.logits[i]));
  const float tz = o.tc[2];
  if (!(tz > near_)) return;
  const float limx = 1.3f * ((float)c.W / (2.0f * c.fx)), limy = 1.3f * ((float)c.H / (2.0f * c.fy));
  const float rx = o.tc[0] / tz, ry = o.tc[1] / tz;
  o.clx = rx < -limx || rx > limx;
  o.cly = ry < -limy || ry > limy;
  o.txp = fminf(limx, fmaxf(-limx, rx)) * tz;
  o.typ = fminf(limy, fmaxf(-limy, ry)) * tz;
  const float itz = 1.0f / tz;
  const float J00 = c.fx * itz, J02 = -c.fx * o.txp * itz * itz;
  const float J11 = c.fy * itz, J12 = -c.fy * o.typ * itz * itz;
  // T = J W, W[k][j] = R[j][k]: T[a][j] = sum_k J[a][k] R[j*3+k]
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    o.T[j] = J00 * c.R[j * 3 + 0] + J02 * c.R[j * 3 + 2];
    o.T[3 + j] = J11 * c.R[j * 3 + 1] + J12 * c.R[j * 3 + 2];
  }
  const float* T = o.T;
  const float* S = o.Sig;
  // U = T Sigma (2x3)
  float U[6];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    U[a * 3 + 0] = T[a * 3 + 0] * S[0] + T[a * 3 + 1] * S[1] + T[a * 3 + 2] * S[2];
    U[a * 3 + 1] = T[a * 3 + 0] * S[1] + T[a * 3 + 1] * S[3] + T[a * 3 + 2] * S[4];
    U[a * 3 + 2] = T[a * 3 + 0] * S[2] + T[a * 3 + 1] * S[4] + T[a * 3 + 2] * S[5];
  }
  o.S2xx = U[0] * T[0] + U[1] * T[1] + U[2] * T[2] + 0.3f;
  o.S2xy = U[0] * T[3] + U[1] * T[4] + U[2] * T[5];
  o.S2yy = U[3] * T[3] + U[4] * T[4] + U[5] * T[5] + 0.3f;
  o.det = o.S2xx * o.S2yy - o.S2xy * o.S2xy;
  if (!(o.det > 0.0f)) return;
  const float idet = 1.0f / o.det;
  o.ca = o.S2yy * idet;
  o.cb = -o.S2xy * idet;
  o.cc = o.S2xx * idet;
  o.mx = c.fx * o.tc[0] * itz + c.cx;
  o.my = c.fy * o.tc[1] * itz + c.cy;
  if (!(o.sig >= kAlphaMin)) return;
  o.qmax = 2.0f * logf(255.0f * o.sig);
  o.ex = __fadd_rn(__fmul_rn(sqrtf(__fmul_rn(o.qmax, o.S2xx)), kExtRel), kExtAbs);
  o.ey = __fadd_rn(__fmul_rn(sqrtf(__fmul_rn(o.qmax, o.S2yy)), kExtRel), kExtAbs);
  int x0, x1, y0, y1;
  if (!record_rect(o.mx, o.my, o.ex, o.ey, c.W, c.H, x0, x1, y0, y1)) return;
  o.vis = isfinite(o.mx) && isfinite(o.my) && isfinite(o.ca) && isfinite(o.cb) && isfinite(o.cc);
}

// K3 for Gaussian i: its record, and its bins added to the block histogram.
template <int DEG>
__device__ __forceinline__ void project_one(const Params& P, int i, float near_, const ViewDev& v,
                                            const float* s_row, uint32_t* s_hist) {
  const Cam cam = v.cam;
  ProjState o;
  project_gaussian(P, i, cam, near_, o);
  float4* r = v.rec + 4 * (size_t)i;
  if (!o.vis) {
    // (a culled Gaussian adds no partials: its fixed-point quanta are moot)
    const uint2 pre = v.grad_fixed ? make_uint2(0u, kFixedPreTag << 24) : make_uint2(0u, 0u);
    r[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    r[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    r[2] = make_float4(0.f, 0.f, 0.f, -1.0f);
    r[3] = make_float4(-1.0f, __uint_as_float(pre.x), __uint_as_float(pre.y), 0.f);
    return;
  }
  const float3 col = view_colour<DEG>(P, i, cam, s_row);
  // deterministic OIT backward: the record's part of the fixed-point quanta
  const uint2 pre = v.grad_fixed ? fixed_pre_exponents(o.mx, o.my, o.ca, o.cb, o.cc, o.ex, o.ey,
                                                       cam.W, cam.H, v.tw, v.th)
                                 : make_uint2(0u, 0u);
  r[0] = make_float4(o.mx, o.my, o.tc[2], o.sig);
  r[1] = make_float4(o.ca, o.cb, o.cc, o.qmax);
  r[2] = make_float4(col.x, col.y, col.z, o.ex);
  r[3] = make_float4(o.ey, __uint_as_float(pre.x), __uint_as_float(pre.y), 0.f);
  int x0, x1, y0, y1;
  record_rect(o.mx, o.my, o.ex, o.ey, cam.W, cam.H, x0, x1, y0, y1);
  for (int sy = y0 >> v.bin_sy; sy <= (y1 >> v.bin_sy); ++sy)
    for (int sx = x0 >> v.bin_sx; sx <= (x1 >> v.bin_sx); ++sx)
      atomicAdd(s_hist + sy * v.sup_x + sx, 1u);
}

// K3: records, plus the block's bin histogram and range reservation (first
// half of the binning; bins are super-tiles or tiles).  Block row blockIdx.y
// projects for view blockIdx.y of the batch; a block takes bin_chunks(M)
// chunks of 256 Gaussians.  sup_count must be zero on entry.
// Shared memory: the bin histogram (max_nsup words, rounded up to an even
// count) and, with DEG > 0, the chunk's SH rows.
template <int DEG>
__global__ void __launch_bounds__(256) project_kernel(Params P, int M, float near_, int hist_words,
                                                      const __grid_constant__ ViewBatch vb) {
  chain_wait();
  extern __shared__ uint32_t s_hist[];
  float* s_f = reinterpret_cast<float*>(s_hist + hist_words);
  const ViewDev& v = vb.v[blockIdx.y];
  const int nsup = v.sup_x * v.sup_y;
  for (int s = threadIdx.x; s < nsup; s += blockDim.x) s_hist[s] = 0;
  const int chunks = bin_chunks(M);
  for (int ch = 0; ch < chunks; ++ch) {
    const long long base = ((long long)blockIdx.x * chunks + ch) * blockDim.x;
    if constexpr (DEG > 0) {
      if (ch > 0) __syncthreads();  // the previous chunk's rows are read
      if (base < M) stage_rows<DEG>(P.sh, base, (int)min((long long)blockDim.x, M - base), s_f);
    }
    if (DEG > 0 || ch == 0) __syncthreads();
    if (base + threadIdx.x < M)
      project_one<DEG>(P, (int)(base + threadIdx.x), near_, v,
                       s_f + threadIdx.x * ShRows<DEG>::STRIDE, s_hist);
  }
  reserve_block_ranges(s_hist, nsup, v.sup_count, v.block_base, v.fixed_order);
}

// Parameter gradients of one Gaussian, summed over the views of a batch.
struct ParamGrad {
  float mean[3], ls[3], q[4], logit, rgb[3];
};

// K8 for one view: the adjoint of the projection of Gaussian i,
// given its 2D gradient (d/d(mx, my, conic_a, conic_b, conic_c, sigma, r, g,
// b, d), already scaled) and the forward state o of the same view; the
// result is added to `acc`.
__device__ __forceinline__ void project_adjoint(const ProjState& o, const Cam& cam, float4 ga,
                                                float4 gb, float4 gc, ParamGrad& acc) {
  const float g_mx = ga.x, g_my = ga.y, g_ca = ga.z, g_cb = ga.w, g_cc = gb.x, g_sig = gb.y;
  const float g_r = gb.z, g_g = gb.w, g_b = gc.x, g_d = gc.y;
  acc.rgb[0] += g_r;
  acc.rgb[1] += g_g;
  acc.rgb[2] += g_b;
  acc.logit += g_sig * o.sig * (1.0f - o.sig);
  // conic = inverse(Sigma2): dS2 = -C Gs C, Gs = [[g_ca, g_cb/2], [g_cb/2, g_cc]]
  const float C00 = o.ca, C01 = o.cb, C11 = o.cc;
  const float G00 = g_ca, G01 = 0.5f * g_cb, G11 = g_cc;
  const float t00 = C00 * G00 + C01 * G01, t01 = C00 * G01 + C01 * G11;
  const float t10 = C01 * G00 + C11 * G01, t11 = C01 * G01 + C11 * G11;
  const float dS00 = -(t00 * C00 + t01 * C01), dS01 = -(t00 * C01 + t01 * C11);
  const float dS11 = -(t10 * C01 + t11 * C11);
  const float* T = o.T;
  const float* S = o.Sig;
  // dT = 2 dS2 T Sigma ; dSigma = T^T dS2 T
  float TS[6];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    TS[a * 3 + 0] = T[a * 3 + 0] * S[0] + T[a * 3 + 1] * S[1] + T[a * 3 + 2] * S[2];
    TS[a * 3 + 1] = T[a * 3 + 0] * S[1] + T[a * 3 + 1] * S[3] + T[a * 3 + 2] * S[4];
    TS[a * 3 + 2] = T[a * 3 + 0] * S[2] + T[a * 3 + 1] * S[4] + T[a * 3 + 2] * S[5];
  }
  float dT[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dT[j] = 2.0f * (dS00 * TS[j] + dS01 * TS[3 + j]);
    dT[3 + j] = 2.0f * (dS01 * TS[j] + dS11 * TS[3 + j]);
  }
  // V = dS2 T (2x3); dSigma = T^T V (symmetric 3x3 as 6 entries)
  float V[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    V[j] = dS00 * T[j] + dS01 * T[3 + j];
    V[3 + j] = dS01 * T[j] + dS11 * T[3 + j];
  }
  float dSig[9];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) dSig[k * 3 + l] = T[k] * V[l] + T[3 + k] * V[3 + l];
  // dJ[a][k] = sum_j dT[a][j] R[j][k]
  float dJ[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dJ[k] = dT[0] * cam.R[k] + dT[1] * cam.R[3 + k] + dT[2] * cam.R[6 + k];
    dJ[3 + k] = dT[3] * cam.R[k] + dT[4] * cam.R[3 + k] + dT[5] * cam.R[6 + k];
  }
  const float tz = o.tc[2], itz = 1.0f / tz, itz2 = itz * itz, itz3 = itz2 * itz;
  float dtx = 0.f, dty = 0.f, dtz = 0.f;
  dtz += dJ[0] * (-cam.fx * itz2) + dJ[4] * (-cam.fy * itz2) +
         dJ[2] * (2.0f * cam.fx * o.txp * itz3) + dJ[5] * (2.0f * cam.fy * o.typ * itz3);
  const float dtxp = dJ[2] * (-cam.fx * itz2), dtyp = dJ[5] * (-cam.fy * itz2);
  if (o.clx) dtz += dtxp * (o.txp * itz); else dtx += dtxp;
  if (o.cly) dtz += dtyp * (o.typ * itz); else dty += dtyp;
  dtx += g_mx * cam.fx * itz;
  dty += g_my * cam.fy * itz;
  dtz += -g_mx * cam.fx * o.tc[0] * itz2 - g_my * cam.fy * o.tc[1] * itz2 + g_d;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    acc.mean[r] += cam.R[r * 3 + 0] * dtx + cam.R[r * 3 + 1] * dty + cam.R[r * 3 + 2] * dtz;
  // Sigma = Mg Mg^T, Mg = Rg diag(s): dMg = 2 dSigma Mg; dRg = dMg diag(s); ds_b = sum_a dMg[a][b] Rg[a][b]
  const float* Rg = o.Rg;
  float dRg[9];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    float ds = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float dMg = 2.0f * (dSig[a * 3 + 0] * Rg[0 * 3 + b] + dSig[a * 3 + 1] * Rg[1 * 3 + b] +
                                dSig[a * 3 + 2] * Rg[2 * 3 + b]) * o.s[b];
      dRg[a * 3 + b] = dMg * o.s[b];
      ds += dMg * Rg[a * 3 + b];
    }
    acc.ls[b] += ds * o.s[b];
  }
  const float w = o.qn[0], x = o.qn[1], y = o.qn[2], z = o.qn[3];
  float dqn[4];
  dqn[0] = dRg[1] * (-2 * z) + dRg[2] * (2 * y) + dRg[3] * (2 * z) + dRg[5] * (-2 * x) +
           dRg[6] * (-2 * y) + dRg[7] * (2 * x);
  dqn[1] = dRg[1] * (2 * y) + dRg[2] * (2 * z) + dRg[3] * (2 * y) + dRg[4] * (-4 * x) +
           dRg[5] * (-2 * w) + dRg[6] * (2 * z) + dRg[7] * (2 * w) + dRg[8] * (-4 * x);
  dqn[2] = dRg[0] * (-4 * y) + dRg[1] * (2 * x) + dRg[2] * (2 * w) + dRg[3] * (2 * x) +
           dRg[5] * (2 * z) + dRg[6] * (-2 * w) + dRg[7] * (2 * z) + dRg[8] * (-4 * y);
  dqn[3] = dRg[0] * (-4 * z) + dRg[1] * (-2 * w) + dRg[2] * (2 * x) + dRg[3] * (2 * w) +
           dRg[4] * (-4 * z) + dRg[5] * (2 * y) + dRg[6] * (2 * x) + dRg[7] * (2 * y);
  const float dot = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
  const float iqn = 1.0f / o.qnorm;
#pragma unroll
  for (int k = 0; k < 4; ++k) acc.q[k] += (dqn[k] - o.qn[k] * dot) * iqn;
}

// K8: adjoint of the projection, summed over the batch's views in view order
// and accumulated (+=) into the parameter gradients once per Gaussian.  With
// DEG > 0 the block stages its Gaussians' SH rows and their gradient rows in
// shared memory (2 x 256 x STRIDE floats).  FIXED: the 2D gradients are
// read from deterministic mode's fixed-point sums (converted here, in the
// same arithmetic as fixed_to_grad2d_kernel) instead of grad2d.
template <int DEG, bool FIXED>
__global__ void __launch_bounds__(256, DEG == 0 ? 3 : 2) project_backward_kernel(Params P, int M, float near_,
                                                               const __grid_constant__ ViewBatch vb,
                                                               GpsGaussians grads,
                                                               const float* dloss) {
  chain_wait();
  extern __shared__ float s_sh[];
  using R = ShRows<DEG>;
  const long long base = (long long)blockIdx.x * blockDim.x;
  const int n_blk = (int)min((long long)blockDim.x, M - base);
  float* s_f = s_sh;
  float* s_g = s_sh + blockDim.x * R::STRIDE;
  if constexpr (DEG > 0) {
    stage_rows<DEG>(P.sh, base, n_blk, s_f);
#pragma unroll
    for (int j = 0; j < R::STRIDE; ++j) s_g[j * kProjThreads + threadIdx.x] = 0.0f;
    __syncthreads();
  }
  const int i = (int)base + threadIdx.x;
  ParamGrad a{};
  for (int k = 0; k < vb.n && i < M; ++k) {
    const Cam cam = vb.v[k].cam;
    ProjState o;
    project_gaussian(P, i, cam, near_, o);
    if (!o.vis) continue;
    float4 ga, gb, gc;
    if constexpr (FIXED) {
      fixed_grad2d(vb.v[k], i, dloss, ga, gb, gc);  // deterministic mode's sums
    } else {
      const float4* g2 = vb.v[k].grad2d + 3 * (size_t)i;
      ga = g2[0];
      gb = g2[1];
      gc = g2[2];
    }
    project_adjoint(o, cam, ga, gb, gc, a);
    if constexpr (DEG > 0) {
      const float3 gm = view_colour_adjoint<DEG>(P, i, cam, make_float3(gb.z, gb.w, gc.x),
                                                 s_f + threadIdx.x * R::STRIDE,
                                                 s_g + threadIdx.x * R::STRIDE);
      a.mean[0] += gm.x;
      a.mean[1] += gm.y;
      a.mean[2] += gm.z;
    }
  }
  // grads += a, through shared memory and coalesced over each group's
  // contiguous [256 x width] slice, all loads before the first store
  constexpr int kRow = kProjThreads + 1;
  __shared__ float s_grad[14 * kRow];
  {
    const float comp[14] = {a.mean[0], a.mean[1], a.mean[2], a.ls[0], a.ls[1], a.ls[2],
                            a.q[0],    a.q[1],    a.q[2],    a.q[3],  a.logit, a.rgb[0],
                            a.rgb[1],  a.rgb[2]};
#pragma unroll
    for (int q = 0; q < 14; ++q) s_grad[q * kRow + threadIdx.x] = comp[q];
  }
  __syncthreads();
  {
    float* const dst[5] = {grads.means, grads.log_scales, grads.quats, grads.opacity_logits,
                           grads.rgb};
    constexpr int width[5] = {3, 3, 4, 1, 3};
    constexpr int first[5] = {0, 3, 6, 10, 11};
    float gv[14];
    int q = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int j = 0; j < width[k]; ++j, ++q) {
        const int e = j * kProjThreads + threadIdx.x;
        if (e < n_blk * width[k]) gv[q] = dst[k][(size_t)base * width[k] + e];
      }
    q = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int j = 0; j < width[k]; ++j, ++q) {
        const int e = j * kProjThreads + threadIdx.x;
        if (e < n_blk * width[k]) {
          const int r = e / width[k], c = e - r * width[k];
          dst[k][(size_t)base * width[k] + e] = gv[q] + s_grad[(first[k] + c) * kRow + r];
        }
      }
  }
  if constexpr (DEG > 0) add_rows<DEG>(grads.sh_rest, base, n_blk, s_g);
}

// Adam state of the fused projection adjoint + Adam step: per group (means,
// log_scales, quats, opacity_logits, rgb, sh_rest) parameters (updated in
// place), moments and learning rate.
struct AdamFused {
  float* p[6];
  float* m[6];
  float* v[6];
  float lr[6];
  float b1, b2, eps;
  float bc1, inv_sbc2;    // 1 - b1^t and 1 / sqrt(1 - b2^t) when the step is known on the host
  const int* device_step; // else: step t = *device_step + 1
};

// K8 and Adam in one pass: as project_backward_kernel, but each Gaussian's
// parameter gradient (summed over the batch's views, zero if no view sees
// it) feeds adam_update directly instead of being added to a gradient array.
// With the gradient array zeroed before render_backward, the same FP32
// operations as render_backward followed by adam_step.  FIXED: as in
// project_backward_kernel.
template <int DEG, bool FIXED>
__global__ void __launch_bounds__(256, DEG == 0 ? 3 : 2) project_backward_adam_kernel(
    Params P, int M, float near_, const __grid_constant__ ViewBatch vb, AdamFused A,
    const float* dloss) {
  chain_wait();
  extern __shared__ float s_sh[];
  using R = ShRows<DEG>;
  const long long base = (long long)blockIdx.x * blockDim.x;
  const int n_blk = (int)min((long long)blockDim.x, M - base);
  float* s_f = s_sh;
  float* s_g = s_sh + blockDim.x * R::STRIDE;
  if constexpr (DEG > 0) {
    stage_rows<DEG>(P.sh, base, n_blk, s_f);
#pragma unroll
    for (int j = 0; j < R::STRIDE; ++j) s_g[j * kProjThreads + threadIdx.x] = 0.0f;
    __syncthreads();
  }
  const int i = (int)base + threadIdx.x;
  ParamGrad a{};
  for (int k = 0; k < vb.n && i < M; ++k) {
    const Cam cam = vb.v[k].cam;
    ProjState o;
    project_gaussian(P, i, cam, near_, o);
    if (!o.vis) continue;
    float4 ga, gb, gc;
    if constexpr (FIXED) {
      fixed_grad2d(vb.v[k], i, dloss, ga, gb, gc);  // deterministic mode's sums
    } else {
      const float4* g2 = vb.v[k].grad2d + 3 * (size_t)i;
      ga = g2[0];
      gb = g2[1];
      gc = g2[2];
    }
    project_adjoint(o, cam, ga, gb, gc, a);
    if constexpr (DEG > 0) {
      const float3 gm = view_colour_adjoint<DEG>(P, i, cam, make_float3(gb.z, gb.w, gc.x),
                                                 s_f + threadIdx.x * R::STRIDE,
                                                 s_g + threadIdx.x * R::STRIDE);
      a.mean[0] += gm.x;
      a.mean[1] += gm.y;
      a.mean[2] += gm.z;
    }
  }
  float bc1 = A.bc1, inv_sbc2 = A.inv_sbc2;
  if (A.device_step) adam_bias(*A.device_step + 1, A.b1, A.b2, bc1, inv_sbc2);
  // The block's 14 gradient components go through shared memory
  // (component-major, 257-float rows against bank conflicts), and the Adam
  // update then walks each group's contiguous [256 x width] slice with
  // consecutive threads on consecutive floats: coalesced, and the adjoint's
  // registers are free again.  The gradient is taken as render_backward
  // leaves it in a zeroed array: 0 + a.
  constexpr int kRow = kProjThreads + 1;
  __shared__ float s_grad[14 * kRow];
  {
    const float comp[14] = {a.mean[0], a.mean[1], a.mean[2], a.ls[0], a.ls[1], a.ls[2],
                            a.q[0],    a.q[1],    a.q[2],    a.q[3],  a.logit, a.rgb[0],
                            a.rgb[1],  a.rgb[2]};
#pragma unroll
    for (int q = 0; q < 14; ++q) s_grad[q * kRow + threadIdx.x] = 0.0f + comp[q];
  }
  __syncthreads();
  {
    constexpr int width[5] = {3, 3, 4, 1, 3};
    constexpr int first[5] = {0, 3, 6, 10, 11};  // first component of each group
    constexpr int NP = 14;
    float pr[NP], mr[NP], vr[NP];
    // all loads first (in flight together), then the updates and stores
    int q = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int j = 0; j < width[k]; ++j, ++q) {
        const int e = j * kProjThreads + threadIdx.x;
        if (e < n_blk * width[k]) {
          const size_t x = (size_t)base * width[k] + e;
          pr[q] = A.p[k][x];
          mr[q] = A.m[k][x];
          vr[q] = A.v[k][x];
        }
      }
    q = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float step_size = A.lr[k] / bc1;
#pragma unroll
      for (int j = 0; j < width[k]; ++j, ++q) {
        const int e = j * kProjThreads + threadIdx.x;
        if (e < n_blk * width[k]) {
          const int r = e / width[k], c = e - r * width[k];
          adam_update(pr[q], s_grad[(first[k] + c) * kRow + r], mr[q], vr[q], A.b1, A.b2, A.eps,
                      step_size, inv_sbc2);
          const size_t x = (size_t)base * width[k] + e;
          A.p[k][x] = pr[q];
          A.m[k][x] = mr[q];
          A.v[k][x] = vr[q];
        }
      }
    }
  }
  if constexpr (DEG > 0) {
    // the block's SH rows, coalesced as in add_rows, in chunks of CH floats
    // per thread whose loads are in flight together
    __syncthreads();
    const float step_size = A.lr[5] / bc1;
    const int total = n_blk * R::K3;
    constexpr int CH = 16;
#pragma unroll
    for (int j0 = 0; j0 < R::K3; j0 += CH) {
      float pr[CH], mr[CH], vr[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int e = (j0 + u) * kProjThreads + threadIdx.x;
        if (j0 + u < R::K3 && e < total) {
          const size_t x = (size_t)base * R::K3 + e;
          pr[u] = A.p[5][x];
          mr[u] = A.m[5][x];
          vr[u] = A.v[5][x];
        }
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int e = (j0 + u) * kProjThreads + threadIdx.x;
        if (j0 + u < R::K3 && e < total) {
          const int r = e / R::K3;
          const size_t x = (size_t)base * R::K3 + e;
          adam_update(pr[u], 0.0f + s_g[r * R::STRIDE + (e - r * R::K3)], mr[u], vr[u], A.b1,
                      A.b2, A.eps, step_size, inv_sbc2);
          A.p[5][x] = pr[u];
          A.m[5][x] = mr[u];
          A.v[5][x] = vr[u];
        }
      }
    }
  }
}

template <int DEG>
cudaError_t launch_project_t(const Params& P, int M, float near_, const ViewBatch& vb,
                             int max_nsup, cudaStream_t st) {
  const int hist_words = (max_nsup + 1) & ~1;
  const size_t smem =
      (size_t)hist_words * 4 + (DEG > 0 ? kProjThreads * ShRows<DEG>::STRIDE * 4 : 0);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        project_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  static_assert(kProjThreads == 256, "binning chunks hold 256 Gaussians");
  launch_chained(project_kernel<DEG>, dim3(bin_blocks(M), vb.n), dim3(kProjThreads), smem, st,
      P, M, near_, hist_words, vb);
  return cudaGetLastError();
}

template <int DEG, bool FIXED>
cudaError_t launch_project_backward_t(const Params& P, int M, float near_, const ViewBatch& vb,
                                      const GpsGaussians& grads, const float* dloss,
                                      cudaStream_t st) {
  const size_t smem = DEG > 0 ? 2 * kProjThreads * ShRows<DEG>::STRIDE * 4 : 0;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(project_backward_kernel<DEG, FIXED>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  launch_chained(project_backward_kernel<DEG, FIXED>, dim3((M + kProjThreads - 1) / kProjThreads),
                 dim3(kProjThreads), smem, st, P, M, near_, vb, grads, dloss);
  return cudaGetLastError();
}

template <int DEG, bool FIXED>
cudaError_t launch_project_backward_adam_t(const Params& P, int M, float near_,
                                           const ViewBatch& vb, const AdamFused& A,
                                           const float* dloss, cudaStream_t st) {
  const size_t smem = DEG > 0 ? 2 * kProjThreads * ShRows<DEG>::STRIDE * 4 : 0;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(project_backward_adam_kernel<DEG, FIXED>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  launch_chained(project_backward_adam_kernel<DEG, FIXED>,
                 dim3((M + kProjThreads - 1) / kProjThreads), dim3(kProjThreads), smem, st, P, M,
                 near_, vb, A, dloss);
  return cudaGetLastError();
}

template <bool FIXED>
cudaError_t launch_project_backward_adam_deg(const Params& P, int M, float near_,
                                             const ViewBatch& vb, const AdamFused& A,
                                             const float* dloss, cudaStream_t st) {
  switch (P.sh_degree) {
    case 1: return launch_project_backward_adam_t<1, FIXED>(P, M, near_, vb, A, dloss, st);
    case 2: return launch_project_backward_adam_t<2, FIXED>(P, M, near_, vb, A, dloss, st);
    case 3: return launch_project_backward_adam_t<3, FIXED>(P, M, near_, vb, A, dloss, st);
    default: return launch_project_backward_adam_t<0, FIXED>(P, M, near_, vb, A, dloss, st);
  }
}

template <bool FIXED>
cudaError_t launch_project_backward_deg(const Params& P, int M, float near_, const ViewBatch& vb,
                                        const GpsGaussians& grads, const float* dloss,
                                        cudaStream_t st) {
  switch (P.sh_degree) {
    case 1: return launch_project_backward_t<1, FIXED>(P, M, near_, vb, grads, dloss, st);
    case 2: return launch_project_backward_t<2, FIXED>(P, M, near_, vb, grads, dloss, st);
    case 3: return launch_project_backward_t<3, FIXED>(P, M, near_, vb, grads, dloss, st);
    default: return launch_project_backward_t<0, FIXED>(P, M, near_, vb, grads, dloss, st);
  }
}

// Fused projection adjoint + Adam (one batch of views); afterwards the device
// step counter advances when the step is read on the device.
cudaError_t launch_project_backward_adam(const GpsGaussians& g, float near_, const ViewBatch& vb,
                                         const GpsGaussians& Mo, const GpsGaussians& Vo,
                                         const GpsAdamHyper& h, int step, int* device_step,
                                         bool fixed_in, const float* dloss, cudaStream_t st) {
  const Params P{g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb, g.sh_rest, g.sh_degree};
  AdamFused A{};
  float* const pp[6] = {g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb, g.sh_rest};
  float* const mm[6] = {Mo.means, Mo.log_scales, Mo.quats, Mo.opacity_logits, Mo.rgb, Mo.sh_rest};
  float* const vv[6] = {Vo.means, Vo.log_scales, Vo.quats, Vo.opacity_logits, Vo.rgb, Vo.sh_rest};
  for (int k = 0; k < 6; ++k) {
    A.p[k] = pp[k];
    A.m[k] = mm[k];
    A.v[k] = vv[k];
    A.lr[k] = k < 5 ? h.lr[k] : h.lr_sh_rest;
  }
  A.b1 = h.beta1;
  A.b2 = h.beta2;
  A.eps = h.eps;
  if (step > 0) {
    A.bc1 = (float)(1.0 - std::pow((double)h.beta1, (double)step));
    A.inv_sbc2 = (float)(1.0 / std::sqrt(1.0 - std::pow((double)h.beta2, (double)step)));
    A.device_step = nullptr;
  } else {
    A.device_step = device_step;
  }
  cudaError_t e = fixed_in
                      ? launch_project_backward_adam_deg<true>(P, g.M, near_, vb, A, dloss, st)
                      : launch_project_backward_adam_deg<false>(P, g.M, near_, vb, A, dloss, st);
  if (e == cudaSuccess && step <= 0) e = launch_adam_step_advance(device_step, st);
  return e;
}

cudaError_t launch_project(const GpsGaussians& g, float near_, const ViewBatch& vb, int max_nsup,
                           cudaStream_t st) {
  const Params P{g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb, g.sh_rest, g.sh_degree};
  switch (g.sh_degree) {
    case 1: return launch_project_t<1>(P, g.M, near_, vb, max_nsup, st);
    case 2: return launch_project_t<2>(P, g.M, near_, vb, max_nsup, st);
    case 3: return launch_project_t<3>(P, g.M, near_, vb, max_nsup, st);
    default: return launch_project_t<0>(P, g.M, near_, vb, max_nsup, st);
  }
}

// fixed_in: the views' 2D gradients are deterministic mode's fixed-point
// sums, not yet converted into grad2d.
cudaError_t launch_project_backward(const GpsGaussians& g, float near_, const ViewBatch& vb,
                                    const GpsGaussians& grads, bool fixed_in, const float* dloss,
                                    cudaStream_t st) {
  const Params P{g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb, g.sh_rest, g.sh_degree};
  return fixed_in ? launch_project_backward_deg<true>(P, g.M, near_, vb, grads, dloss, st)
                  : launch_project_backward_deg<false>(P, g.M, near_, vb, grads, dloss, st);
}

}  // namespace gps
