// Oracle (test infrastructure only): view-dependent colour from spherical
// harmonics, FP64.
//
// Sec. 3.1 gives every Gaussian spherical-harmonic colour coefficients
// "following 3DGS"; App. C sets their learning rates.  Reading used here: the
// colour seen from camera centre o is
//     c = rgb + sum_{l=1..D} sum_{m=-l..l} Y_lm(d) f_lm,   d = (p - o) / |p - o|,
// with Y_lm the real, orthonormal spherical harmonics built from the complex
// ones with the Condon-Shortley phase: Y_l0 = Y_l^0, Y_lm = sqrt(2) Re Y_l^m
// (m > 0), Y_l,-m = sqrt(2) Im Y_l^m (m > 0); coefficients stored per
// Gaussian in the order l = 1..D, m = -l..l, each an RGB triple.  The degree-0
// term is rgb itself (no +0.5 offset, no clamp at zero), as for degree 0.
//
// Each Y_lm is written below as its polynomial in the unit vector (x, y, z);
// the gradient of the colour with respect to the mean goes through the
// normalisation: dL/dp = (I - d d^T) / |p - o| * sum_lm (dY_lm/dd) (f_lm . dL/dc).
#include <cmath>
#include <cstddef>
#include <vector>

#include "mag.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

int sh_count(int degree) { return (degree + 1) * (degree + 1) - 1; }

// Y[k] for k = 0 .. sh_count(degree) - 1 and, when dY is non-null, the
// partial derivatives of each polynomial along x, y, z: dY[3k + 0..2].
void basis(int degree, double x, double y, double z, double* Y, double* dY) {
  const double c1 = std::sqrt(3.0 / (4.0 * kPi));
  const double c2a = 0.5 * std::sqrt(15.0 / kPi), c2b = 0.25 * std::sqrt(5.0 / kPi),
               c2c = 0.25 * std::sqrt(15.0 / kPi);
  const double c3a = 0.25 * std::sqrt(35.0 / (2.0 * kPi)), c3b = 0.5 * std::sqrt(105.0 / kPi),
               c3c = 0.25 * std::sqrt(21.0 / (2.0 * kPi)), c3d = 0.25 * std::sqrt(7.0 / kPi),
               c3e = 0.25 * std::sqrt(105.0 / kPi);
  double v[15], g[45] = {0};
  // l = 1: m = -1, 0, 1
  v[0] = -c1 * y;  g[0 * 3 + 1] = -c1;
  v[1] = c1 * z;   g[1 * 3 + 2] = c1;
  v[2] = -c1 * x;  g[2 * 3 + 0] = -c1;
  // l = 2
  v[3] = c2a * x * y;                     g[9] = c2a * y;  g[10] = c2a * x;
  v[4] = -c2a * y * z;                    g[13] = -c2a * z; g[14] = -c2a * y;
  v[5] = c2b * (2 * z * z - x * x - y * y);
  g[15] = -2 * c2b * x; g[16] = -2 * c2b * y; g[17] = 4 * c2b * z;
  v[6] = -c2a * x * z;                    g[18] = -c2a * z; g[20] = -c2a * x;
  v[7] = c2c * (x * x - y * y);           g[21] = 2 * c2c * x; g[22] = -2 * c2c * y;
  // l = 3
  v[8] = -c3a * y * (3 * x * x - y * y);
  g[24] = -6 * c3a * x * y; g[25] = -3 * c3a * (x * x - y * y);
  v[9] = c3b * x * y * z;
  g[27] = c3b * y * z; g[28] = c3b * x * z; g[29] = c3b * x * y;
  v[10] = -c3c * y * (4 * z * z - x * x - y * y);
  g[30] = 2 * c3c * x * y; g[31] = -c3c * (4 * z * z - x * x - 3 * y * y); g[32] = -8 * c3c * y * z;
  v[11] = c3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
  g[33] = -6 * c3d * x * z; g[34] = -6 * c3d * y * z; g[35] = c3d * (6 * z * z - 3 * x * x - 3 * y * y);
  v[12] = -c3c * x * (4 * z * z - x * x - y * y);
  g[36] = -c3c * (4 * z * z - 3 * x * x - y * y); g[37] = 2 * c3c * x * y; g[38] = -8 * c3c * x * z;
  v[13] = c3e * z * (x * x - y * y);
  g[39] = 2 * c3e * x * z; g[40] = -2 * c3e * y * z; g[41] = c3e * (x * x - y * y);
  v[14] = -c3a * x * (x * x - 3 * y * y);
  g[42] = -3 * c3a * (x * x - y * y); g[43] = 6 * c3a * x * y;
  const int K = sh_count(degree);
  for (int k = 0; k < K; ++k) {
    Y[k] = v[k];
    if (dY)
      for (int a = 0; a < 3; ++a) dY[3 * k + a] = g[3 * k + a];
  }
}


inline bool is_zero(double v) { return v == 0.0; }
inline bool is_zero(Mag m) { return m.v == 0.0; }

// Body of orc_sh_backward; T = double is the adjoint, T = Mag its magnitudes.
template <class T>
void sh_backward_t(int M, int degree, const double* means, const double* sh,
                   const double* centre, const T* dc, T* d_means, T* d_sh) {
  const int K = sh_count(degree);
  double Y[15], dY[45];
  for (int i = 0; i < M; ++i) {
    const T* g = dc + 3 * i;
    if (is_zero(g[0]) && is_zero(g[1]) && is_zero(g[2])) continue;
    double v[3], n2 = 0;
    for (int a = 0; a < 3; ++a) {
      v[a] = means[3 * i + a] - centre[a];
      n2 += v[a] * v[a];
    }
    const double n = std::sqrt(n2);
    const double d[3] = {v[0] / n, v[1] / n, v[2] / n};
    basis(degree, d[0], d[1], d[2], Y, dY);
    T gd[3] = {0.0, 0.0, 0.0};  // dL/dd (ambient)
    for (int k = 0; k < K; ++k) {
      const double* f = sh + ((size_t)i * K + k) * 3;
      T* df = d_sh + ((size_t)i * K + k) * 3;
      T w = 0.0;
      for (int ch = 0; ch < 3; ++ch) {
        df[ch] += Y[k] * g[ch];
        w += f[ch] * g[ch];
      }
      for (int a = 0; a < 3; ++a) gd[a] += dY[3 * k + a] * w;
    }
    const T dot = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
    for (int a = 0; a < 3; ++a) d_means[3 * i + a] += (gd[a] - d[a] * dot) / n;
  }
}

}  // namespace

extern "C" {

// Y [n][sh_count(degree)] at unit directions dirs [n][3].
void orc_sh_basis(int n, int degree, const double* dirs, double* Y) {
  const int K = sh_count(degree);
  for (int i = 0; i < n; ++i)
    basis(degree, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Y + (size_t)i * K, nullptr);
}

// Colour of each Gaussian seen from camera centre `centre`: out [M][3].
void orc_sh_colour(int M, int degree, const double* means, const double* rgb, const double* sh,
                   const double* centre, double* out) {
  const int K = sh_count(degree);
  double Y[15];
  for (int i = 0; i < M; ++i) {
    double v[3], n2 = 0;
    for (int a = 0; a < 3; ++a) {
      v[a] = means[3 * i + a] - centre[a];
      n2 += v[a] * v[a];
    }
    const double n = std::sqrt(n2);
    basis(degree, v[0] / n, v[1] / n, v[2] / n, Y, nullptr);
    for (int ch = 0; ch < 3; ++ch) {
      double c = rgb[3 * i + ch];
      for (int k = 0; k < K; ++k) c += Y[k] * sh[((size_t)i * K + k) * 3 + ch];
      out[3 * i + ch] = c;
    }
  }
}

// Adjoint of orc_sh_colour given dL/dc [M][3]: adds to d_means [M][3] and
// d_sh [M][K][3] (dL/drgb = dL/dc, left to the caller).
void orc_sh_backward(int M, int degree, const double* means, const double* sh,
                     const double* centre, const double* dc, double* d_means, double* d_sh) {
  sh_backward_t<double>(M, degree, means, sh, centre, dc, d_means, d_sh);
}

// The same adjoint in magnitude arithmetic (mag.h) from |dL/dc|: adds the
// magnitudes of its terms to d_means and d_sh.
void orc_sh_backward_mag(int M, int degree, const double* means, const double* sh,
                         const double* centre, const double* dc, double* d_means, double* d_sh) {
  const int K = sh_count(degree);
  std::vector<Mag> gm(3 * (size_t)M), dm(3 * (size_t)M), ds((size_t)M * K * 3);
  for (size_t k = 0; k < gm.size(); ++k) gm[k] = Mag(dc[k]);
  sh_backward_t<Mag>(M, degree, means, sh, centre, gm.data(), dm.data(), ds.data());
  for (size_t k = 0; k < dm.size(); ++k) d_means[k] += dm[k].v;
  for (size_t k = 0; k < ds.size(); ++k) d_sh[k] += ds[k].v;
}

}  // extern "C"
