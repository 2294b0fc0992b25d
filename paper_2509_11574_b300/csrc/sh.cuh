// View-dependent colour of a Gaussian from real spherical harmonics of degree
// 1..3 (Sec. 3.1: Gaussians carry SH colour "following 3DGS").  Internal header.
//
//   c = rgb + sum_k Y_k(d) f_k,   d = (p - o) / |p - o|,  k = (l, m), m = -l..l
//
// Y_k are the real orthonormal harmonics (Condon-Shortley phase), written as
// polynomials in the unit direction (x, y, z); their normalisation constants
// are sqrt((2l + 1) / (4 pi) (l - |m|)! / (l + |m|)!) times sqrt(2) for m != 0,
// folded into the polynomial coefficients below.
#pragma once
#include <cuda_runtime.h>

namespace gps {

constexpr int kShMaxCoeffs = 15;  // degree 3
__host__ __device__ constexpr int sh_coeffs(int degree) { return (degree + 1) * (degree + 1) - 1; }

// polynomial coefficients (the constants of the orthonormal basis)
constexpr float kSh1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kSh2a = 1.09254843059207907f;  // sqrt(15 / pi) / 2
constexpr float kSh2b = 0.31539156525252001f;  // sqrt(5 / pi) / 4
constexpr float kSh2c = 0.54627421529603954f;  // sqrt(15 / pi) / 4
constexpr float kSh3a = 0.59004358992664352f;  // sqrt(35 / (2 pi)) / 4
constexpr float kSh3b = 2.89061144264055405f;  // sqrt(105 / pi) / 2
constexpr float kSh3c = 0.45704579946446572f;  // sqrt(21 / (2 pi)) / 4
constexpr float kSh3d = 0.37317633259011540f;  // sqrt(7 / pi) / 4
constexpr float kSh3e = 1.44530572132027702f;  // sqrt(105 / pi) / 4

// Y[0 .. sh_coeffs(degree)) at the unit direction (x, y, z).
__device__ __forceinline__ void sh_eval(int degree, float x, float y, float z, float* Y) {
  Y[0] = -kSh1 * y;
  Y[1] = kSh1 * z;
  Y[2] = -kSh1 * x;
  if (degree < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[3] = kSh2a * x * y;
  Y[4] = -kSh2a * y * z;
  Y[5] = kSh2b * (2.0f * zz - xx - yy);
  Y[6] = -kSh2a * x * z;
  Y[7] = kSh2c * (xx - yy);
  if (degree < 3) return;
  Y[8] = -kSh3a * y * (3.0f * xx - yy);
  Y[9] = kSh3b * x * y * z;
  Y[10] = -kSh3c * y * (4.0f * zz - xx - yy);
  Y[11] = kSh3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
  Y[12] = -kSh3c * x * (4.0f * zz - xx - yy);
  Y[13] = kSh3e * z * (xx - yy);
  Y[14] = -kSh3a * x * (xx - 3.0f * yy);
}

// sum_k w[k] grad Y_k at (x, y, z), the gradient of each polynomial taken in
// R^3 (the caller projects it onto the sphere's tangent plane).
__device__ __forceinline__ float3 sh_grad_dot(int degree, float x, float y, float z,
                                              const float* w) {
  float gx = -kSh1 * w[2], gy = -kSh1 * w[0], gz = kSh1 * w[1];
  if (degree >= 2) {
    gx += kSh2a * y * w[3] - 2.0f * kSh2b * x * w[5] - kSh2a * z * w[6] + 2.0f * kSh2c * x * w[7];
    gy += kSh2a * x * w[3] - kSh2a * z * w[4] - 2.0f * kSh2b * y * w[5] - 2.0f * kSh2c * y * w[7];
    gz += -kSh2a * y * w[4] + 4.0f * kSh2b * z * w[5] - kSh2a * x * w[6];
  }
  if (degree >= 3) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += -6.0f * kSh3a * x * y * w[8] + kSh3b * y * z * w[9] + 2.0f * kSh3c * x * y * w[10] -
          6.0f * kSh3d * x * z * w[11] - kSh3c * (4.0f * zz - 3.0f * xx - yy) * w[12] +
          2.0f * kSh3e * x * z * w[13] - 3.0f * kSh3a * (xx - yy) * w[14];
    gy += -3.0f * kSh3a * (xx - yy) * w[8] + kSh3b * x * z * w[9] -
          kSh3c * (4.0f * zz - xx - 3.0f * yy) * w[10] - 6.0f * kSh3d * y * z * w[11] +
          2.0f * kSh3c * x * y * w[12] - 2.0f * kSh3e * y * z * w[13] + 6.0f * kSh3a * x * y * w[14];
    gz += kSh3b * x * y * w[9] - 8.0f * kSh3c * y * z * w[10] +
          kSh3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * w[11] - 8.0f * kSh3c * x * z * w[12] +
          kSh3e * (xx - yy) * w[13];
  }
  return make_float3(gx, gy, gz);
}

}  // namespace gps
