// Adam over the parameter groups (App. C learning rates: the five of every set,
// plus the SH coefficients of degree >= 1 when present), torch.optim.Adam
// semantics, FP32 moments.  One launch covers all groups; each thread updates
// four consecutive floats with 16-byte loads where the group allows it.  The
// gradient is zeroed in the same pass (its write replaces the zero_grad pass).
// The update itself is adam_update (adam.cuh).
#include <cuda_runtime.h>

#include <cmath>

#include "adam.cuh"
#include "gps_common.cuh"
#include "sh.cuh"

namespace gps {

struct AdamGroup {
  float* p;
  float* g;
  float* m;
  float* v;
  long long n;
  float lr;
  int vec4;  // all four pointers 16-byte aligned
};

constexpr int kAdamGroups = 6;

struct AdamArgs {
  AdamGroup grp[kAdamGroups];
  long long first_block[kAdamGroups + 1];  // block offsets per group (empty groups: n = 0)
  float b1, b2, eps;
  float bc1, inv_sbc2;  // 1 - b1^t and 1 / sqrt(1 - b2^t) when the step is known on the host
  int* device_step; // else: step t = *device_step + 1
};

__global__ void __launch_bounds__(256) adam_kernel(AdamArgs a) {
  chain_wait();
  float bc1 = a.bc1, inv_sbc2 = a.inv_sbc2;
  if (a.device_step) adam_bias(*a.device_step + 1, a.b1, a.b2, bc1, inv_sbc2);
  const long long blk = blockIdx.x;
  int gidx = 0;
#pragma unroll
  for (int k = 1; k < kAdamGroups; ++k)
    if (blk >= a.first_block[k]) gidx = k;
  const AdamGroup& G = a.grp[gidx];
  const long long base = ((blk - a.first_block[gidx]) * 256 + threadIdx.x) * 4;
  if (base >= G.n) return;
  const float step_size = G.lr / bc1;
  const float b1 = a.b1, b2 = a.b2, eps = a.eps;
  if (G.vec4 && base + 4 <= G.n) {
    float4 p = *reinterpret_cast<float4*>(G.p + base);
    const float4 g = *reinterpret_cast<float4*>(G.g + base);
    float4 m = *reinterpret_cast<float4*>(G.m + base);
    float4 v = *reinterpret_cast<float4*>(G.v + base);
    adam_update(p.x, g.x, m.x, v.x, b1, b2, eps, step_size, inv_sbc2);
    adam_update(p.y, g.y, m.y, v.y, b1, b2, eps, step_size, inv_sbc2);
    adam_update(p.z, g.z, m.z, v.z, b1, b2, eps, step_size, inv_sbc2);
    adam_update(p.w, g.w, m.w, v.w, b1, b2, eps, step_size, inv_sbc2);
    *reinterpret_cast<float4*>(G.p + base) = p;
    *reinterpret_cast<float4*>(G.m + base) = m;
    *reinterpret_cast<float4*>(G.v + base) = v;
    *reinterpret_cast<float4*>(G.g + base) = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    for (long long k = base; k < min(base + 4, G.n); ++k) {
      float p = G.p[k], m = G.m[k], v = G.v[k];
      adam_update(p, G.g[k], m, v, b1, b2, eps, step_size, inv_sbc2);
      G.m[k] = m;
      G.v[k] = v;
      G.p[k] = p;
      G.g[k] = 0.0f;
    }
  }
}

__global__ void adam_step_advance_kernel(int* device_step) {
  chain_wait();
  *device_step += 1;
}

cudaError_t launch_adam_step_advance(int* device_step, cudaStream_t st) {
  launch_chained(adam_step_advance_kernel, dim3(1), dim3(1), 0, st, device_step);
  return cudaGetLastError();
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

cudaError_t launch_adam(const GpsGaussians& P, const GpsGaussians& Gr, const GpsGaussians& Mo,
                        const GpsGaussians& Vo, const GpsAdamHyper& h, int step, int* device_step,
                        cudaStream_t st) {
  AdamArgs a{};
  float* const pp[kAdamGroups] = {P.means, P.log_scales, P.quats, P.opacity_logits, P.rgb,
                                  P.sh_rest};
  float* const gg[kAdamGroups] = {Gr.means, Gr.log_scales, Gr.quats, Gr.opacity_logits, Gr.rgb,
                                  Gr.sh_rest};
  float* const mm[kAdamGroups] = {Mo.means, Mo.log_scales, Mo.quats, Mo.opacity_logits, Mo.rgb,
                                  Mo.sh_rest};
  float* const vv[kAdamGroups] = {Vo.means, Vo.log_scales, Vo.quats, Vo.opacity_logits, Vo.rgb,
                                  Vo.sh_rest};
  const int width[kAdamGroups] = {3, 3, 4, 1, 3, P.sh_degree > 0 ? 3 * sh_coeffs(P.sh_degree) : 0};
  long long blocks = 0;
  for (int k = 0; k < kAdamGroups; ++k) {
    AdamGroup& G = a.grp[k];
    G.p = pp[k];
    G.g = gg[k];
    G.m = mm[k];
    G.v = vv[k];
    G.n = (long long)P.M * width[k];
    G.lr = k < 5 ? h.lr[k] : h.lr_sh_rest;
    G.vec4 = aligned16(G.p) && aligned16(G.g) && aligned16(G.m) && aligned16(G.v);
    a.first_block[k] = blocks;
    blocks += (G.n + 1023) / 1024;
  }
  a.first_block[kAdamGroups] = blocks;
  a.b1 = h.beta1;
  a.b2 = h.beta2;
  a.eps = h.eps;
  if (step > 0) {
    a.bc1 = (float)(1.0 - std::pow((double)h.beta1, (double)step));
    a.inv_sbc2 = (float)(1.0 / std::sqrt(1.0 - std::pow((double)h.beta2, (double)step)));
    a.device_step = nullptr;
  } else {
    a.device_step = device_step;
  }
  if (blocks == 0) return cudaSuccess;
  launch_chained(adam_kernel, dim3((unsigned)blocks), dim3(256), 0, st, a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && step <= 0) e = launch_adam_step_advance(device_step, st);
  return e;
}

}  // namespace gps
