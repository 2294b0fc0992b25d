// Adam's per-parameter update (torch.optim.Adam semantics, FP32 moments),
// shared by adam_kernel and the fused projection-adjoint + Adam kernel so that
// both paths take the same FP32 operations:
//   m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2
//   p <- p - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)
#pragma once
#include <cuda_runtime.h>

namespace gps {

// 1 - b1^t and 1 / sqrt(1 - b2^t) for step t, with 1 - b^t = -expm1(t ln b)
// and ln b = log1p(b - 1): accurate for b near 1.
__device__ __forceinline__ void adam_bias(int t, float b1, float b2, float& bc1,
                                          float& inv_sbc2) {
  const float tf = (float)t;
  bc1 = -expm1f(tf * log1pf(b1 - 1.0f));
  inv_sbc2 = 1.0f / sqrtf(-expm1f(tf * log1pf(b2 - 1.0f)));
}

// step_size = lr / (1 - b1^t), inv_sbc2 = 1 / sqrt(1 - b2^t).  Every
// rounding is spelled out (no contraction left to the compiler), so the two
// kernels that inline it compute the same bits.  The bias correction of v
// is a product with the precomputed reciprocal and the step's quotient the
// fast reciprocal-multiply (__fdividef, within 2 ulp): together about 3e-7
// relative on the step, against the division-heavy form that made the
// update the larger part of the fused backward's instructions.
__device__ __forceinline__ void adam_update(float& p, float g, float& m, float& v, float b1,
                                            float b2, float eps, float step_size,
                                            float inv_sbc2) {
  m = __fmaf_rn(b1, m, __fmul_rn(1.0f - b1, g));
  v = __fmaf_rn(b2, v, __fmul_rn(__fmul_rn(1.0f - b2, g), g));
  const float den = __fmaf_rn(__fsqrt_rn(v), inv_sbc2, eps);
  p = __fsub_rn(p, __fmul_rn(step_size, __fdividef(m, den)));
}

}  // namespace gps
