// Projection of 3D Gaussians to 2D conics (Sec. 3.1, "following 3DGS") and its
// adjoint.  One thread per Gaussian; parameters are read once (56 B) and one
// 64-byte record is written.  The forward also builds its block's histogram of
// super-tiles touched and reserves the block's ranges (first half of the binning).
#include <cuda_runtime.h>

#include "gps_common.cuh"

namespace gps {

struct Params {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* logits;
  const float* rgb;
};

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

// K3: records, plus the block's super-tile histogram and range reservation
// (first half of the binning).  Block row blockIdx.y projects for view
// blockIdx.y of the batch.  sup_count must be zero on entry.
__global__ void __launch_bounds__(256) project_kernel(Params P, int M, float near_,
                                                      const __grid_constant__ ViewBatch vb) {
  extern __shared__ uint32_t s_hist[];
  const ViewDev& v = vb.v[blockIdx.y];
  const int sh = v.sup_shift, sup_x = v.sup_x, nsup = v.sup_x * v.sup_y;
  for (int s = threadIdx.x; s < nsup; s += blockDim.x) s_hist[s] = 0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) {
    const Cam cam = v.cam;
    ProjState o;
    project_gaussian(P, i, cam, near_, o);
    float4* r = v.rec + 4 * (size_t)i;
    if (!o.vis) {
      r[0] = make_float4(0.f, 0.f, 0.f, 0.f);
      r[1] = make_float4(0.f, 0.f, 0.f, 0.f);
      r[2] = make_float4(0.f, 0.f, 0.f, -1.0f);
      r[3] = make_float4(-1.0f, 0.f, 0.f, 0.f);
    } else {
      const float* col = P.rgb + 3 * (size_t)i;
      r[0] = make_float4(o.mx, o.my, o.tc[2], o.sig);
      r[1] = make_float4(o.ca, o.cb, o.cc, o.qmax);
      r[2] = make_float4(col[0], col[1], col[2], o.ex);
      r[3] = make_float4(o.ey, 0.f, 0.f, 0.f);
      int x0, x1, y0, y1;
      record_rect(o.mx, o.my, o.ex, o.ey, cam.W, cam.H, x0, x1, y0, y1);
      for (int sy = y0 >> sh; sy <= (y1 >> sh); ++sy)
        for (int sx = x0 >> sh; sx <= (x1 >> sh); ++sx)
          atomicAdd(s_hist + sy * sup_x + sx, 1u);
    }
  }
  reserve_block_ranges(s_hist, nsup, v.sup_count, v.block_base);
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
// and accumulated (+=) into the parameter gradients once per Gaussian.
__global__ void __launch_bounds__(256) project_backward_kernel(Params P, int M, float near_,
                                                               const __grid_constant__ ViewBatch vb,
                                                               GpsGaussians grads) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  ParamGrad a{};
  bool any = false;
  for (int k = 0; k < vb.n; ++k) {
    const Cam cam = vb.v[k].cam;
    ProjState o;
    project_gaussian(P, i, cam, near_, o);
    if (!o.vis) continue;
    const float4* g2 = vb.v[k].grad2d + 3 * (size_t)i;
    project_adjoint(o, cam, g2[0], g2[1], g2[2], a);
    any = true;
  }
  if (!any) return;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    grads.means[3 * (size_t)i + r] += a.mean[r];
    grads.log_scales[3 * (size_t)i + r] += a.ls[r];
    grads.rgb[3 * (size_t)i + r] += a.rgb[r];
  }
  float4* dq = reinterpret_cast<float4*>(grads.quats) + i;
  float4 q = *dq;
  q.x += a.q[0];
  q.y += a.q[1];
  q.z += a.q[2];
  q.w += a.q[3];
  *dq = q;
  grads.opacity_logits[i] += a.logit;
}

cudaError_t launch_project(const GpsGaussians& g, float near_, const ViewBatch& vb, int max_nsup,
                           cudaStream_t st) {
  Params P{g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb};
  const size_t smem = (size_t)max_nsup * sizeof(uint32_t);
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  project_kernel<<<dim3((g.M + 255) / 256, vb.n), 256, smem, st>>>(P, g.M, near_, vb);
  return cudaGetLastError();
}

cudaError_t launch_project_backward(const GpsGaussians& g, float near_, const ViewBatch& vb,
                                    const GpsGaussians& grads, cudaStream_t st) {
  Params P{g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb};
  project_backward_kernel<<<(g.M + 255) / 256, 256, 0, st>>>(P, g.M, near_, vb, grads);
  return cudaGetLastError();
}

}  // namespace gps
