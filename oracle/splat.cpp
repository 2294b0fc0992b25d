// Oracle (test infrastructure only): Gaussian projection, depth-culled hybrid
// compositing, L1 loss, analytic adjoints, tile binning and Adam, in FP64.
//
// What it computes, with the passage it follows:
//   * Gaussian set {p_i, sigma_i, r_i, s_i, SH_i} "following 3DGS" (Sec. 3.1); colour
//     is the degree-0 RGB only.
//   * projection to a 2D mean p^_i, covariance Sigma_2D and centre depth d_i
//     (Sec. 3.1, Eq. 3 and the sentence after it): EWA with the 3DGS 1.3x
//     frustum clamp of the Jacobian and a +0.3 px^2 dilation.
//   * order-independent, depth-culled accumulation (Eq. 1-3) and the hybrid
//     blend with W_t = 1 (Eq. 4); alpha < 1/255 counts as 0 (Sec. 3.1).
//   * the "with sort" variant of Table 7, read as 3DGS front-to-back alpha
//     compositing over the SDF colour (alpha <= 0.99, stop when T < 1e-4).
//   * colour L1 loss (Sec. 3.2.2, Eq. 6) averaged over valid pixels and channels,
//     plus an optional depth L1 term weighted by lambda_depth.
//   * the exact derivative of all of the above (hand-derived chain rule).
//   * Adam with per-group learning rates (App. C), torch semantics.
//
// Decisions that pick an integer (is Gaussian i counted at pixel x?) can be
// taken either in FP64 (the definition) or in FP32 from the FP32 values of a
// projected record - the precision of the CUDA kernels - so that a staged
// comparison sees identical decisions; the FP32 form is spelled out at
// `support_f32`.  Every accumulation is FP64.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <omp.h>

#include "mag.h"

namespace {

// projected record, FP64 (index names shared with the Python wrapper)
enum {
  R_MX = 0, R_MY, R_D, R_SIG, R_CA, R_CB, R_CC, R_QMAX, R_R, R_G, R_B, R_EX, R_EY, R_VIS,
  R_S2XX, R_S2YY, R_N
};
// per-Gaussian 2D gradient layout
enum { G_MX = 0, G_MY, G_CA, G_CB, G_CC, G_SIG, G_R, G_G, G_B, G_D, G_N };

struct Cam {
  double fx, fy, cx, cy;
  int W, H;
  const double* R;  // camera->world, row-major
  const double* t;  // camera centre
};

inline void rot_from_quat(const double* q, double* Rm) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  Rm[0] = 1 - 2 * (y * y + z * z); Rm[1] = 2 * (x * y - w * z);     Rm[2] = 2 * (x * z + w * y);
  Rm[3] = 2 * (x * y + w * z);     Rm[4] = 1 - 2 * (x * x + z * z); Rm[5] = 2 * (y * z - w * x);
  Rm[6] = 2 * (x * z - w * y);     Rm[7] = 2 * (y * z + w * x);     Rm[8] = 1 - 2 * (x * x + y * y);
}

// Intermediate quantities of one Gaussian's projection, kept for the adjoint.
struct Proj {
  bool vis;
  double qn[4], qnorm, Rg[9], s[3], Sig[9], tc[3], txp, typ;
  bool clx, cly;
  double J[6], T[6], S2[4], det, conic[3], mx, my, sig, qmax, ex, ey;
};

// Sec. 3.1: p^_i, Sigma_2D, d_i, following 3DGS (EWA splatting).
Proj project_one(const Cam& c, const double* p, const double* ls, const double* q,
                 double logit, double near_) {
  Proj P{};
  P.vis = false;
  P.qnorm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) P.qn[k] = q[k] / P.qnorm;
  rot_from_quat(P.qn, P.Rg);
  for (int k = 0; k < 3; ++k) P.s[k] = std::exp(ls[k]);
  // Sigma = R S S^T R^T
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0;
      for (int k = 0; k < 3; ++k) a += P.Rg[i * 3 + k] * P.s[k] * P.s[k] * P.Rg[j * 3 + k];
      P.Sig[i * 3 + j] = a;
    }
  // t = R_cw (p - c), R_cw = R^T
  double d[3] = {p[0] - c.t[0], p[1] - c.t[1], p[2] - c.t[2]};
  for (int i = 0; i < 3; ++i)
    P.tc[i] = c.R[0 * 3 + i] * d[0] + c.R[1 * 3 + i] * d[1] + c.R[2 * 3 + i] * d[2];
  P.sig = 1.0 / (1.0 + std::exp(-logit));
  if (!(P.tc[2] > near_)) return P;
  const double tz = P.tc[2];
  const double limx = 1.3 * (c.W / (2.0 * c.fx)), limy = 1.3 * (c.H / (2.0 * c.fy));
  double rx = P.tc[0] / tz, ry = P.tc[1] / tz;
  P.clx = rx < -limx || rx > limx;
  P.cly = ry < -limy || ry > limy;
  P.txp = std::min(limx, std::max(-limx, rx)) * tz;
  P.typ = std::min(limy, std::max(-limy, ry)) * tz;
  P.J[0] = c.fx / tz; P.J[1] = 0; P.J[2] = -c.fx * P.txp / (tz * tz);
  P.J[3] = 0; P.J[4] = c.fy / tz; P.J[5] = -c.fy * P.typ / (tz * tz);
  // T = J W, W = R_cw (row i of W = column i of R)
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0;
      for (int k = 0; k < 3; ++k) a += P.J[i * 3 + k] * c.R[j * 3 + k];
      P.T[i * 3 + j] = a;
    }
  // Sigma_2D = T Sigma T^T + 0.3 I
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double a = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) a += P.T[i * 3 + k] * P.Sig[k * 3 + l] * P.T[j * 3 + l];
      P.S2[i * 2 + j] = a + (i == j ? 0.3 : 0.0);
    }
  P.det = P.S2[0] * P.S2[3] - P.S2[1] * P.S2[2];
  if (!(P.det > 0.0)) return P;
  P.conic[0] = P.S2[3] / P.det;
  P.conic[1] = -P.S2[1] / P.det;
  P.conic[2] = P.S2[0] / P.det;
  P.mx = c.fx * P.tc[0] / tz + c.cx;
  P.my = c.fy * P.tc[1] / tz + c.cy;
  if (!(P.sig >= 1.0 / 255.0)) return P;
  // support {q <= qmax} is exactly the set where sigma exp(-q/2) >= 1/255
  P.qmax = 2.0 * std::log(255.0 * P.sig);
  P.ex = std::sqrt(P.qmax * P.S2[0]);
  P.ey = std::sqrt(P.qmax * P.S2[3]);
  if (P.mx + P.ex < 0 || P.mx - P.ex > c.W - 1 || P.my + P.ey < 0 || P.my - P.ey > c.H - 1)
    return P;
  P.vis = true;
  return P;
}

// FP32 form of the per-pixel decisions (the kernels' precision).  With
// dx = x - mx, dy = y - my in float:
//   q = fmaf(dx, fmaf(a, dx, (2b) dy), (c dy) dy)   (each product rounded to float)
//   counted  <=>  q <= qmax  and  d < thr,  thr = D_t + eps (float) or +inf if D_t <= 0.
inline bool support_f32(float mx, float my, float a, float b, float c, float qmax, int px,
                        int py) {
  float dx = (float)px - mx;
  float dy = (float)py - my;
  float b2 = 2.0f * b;
  float t1 = b2 * dy;
  float s2 = std::fmaf(a, dx, t1);
  float cd = c * dy;
  float s3 = cd * dy;
  float q = std::fmaf(dx, s2, s3);
  return q <= qmax;
}

struct Item {
  int id;
  double alpha, G, dx, dy;
};

// Front-to-back order: by depth (compared in float when the decisions are
// taken in FP32), ties by ascending index.
void sort_front_to_back(std::vector<Item>& its, const double* rec, int f32) {
  std::stable_sort(its.begin(), its.end(), [&](const Item& a, const Item& b) {
    double da = rec[(size_t)a.id * R_N + R_D], db = rec[(size_t)b.id * R_N + R_D];
    if (f32) {
      float fa = (float)da, fb = (float)db;
      if (fa != fb) return fa < fb;
    } else if (da != db) {
      return da < db;
    }
    return a.id < b.id;
  });
}

// Candidates of one pixel: every visible Gaussian whose bounding box (extent +
// 1 px) contains it, in index order.  `brute` = every visible Gaussian.
struct Lists {
  std::vector<std::vector<int>> cand;
};

Lists build_lists(int M, const double* rec, int W, int H, int brute, int x0, int x1, int y0,
                  int y1) {
  Lists L;
  L.cand.assign((size_t)W * H, {});
  for (int i = 0; i < M; ++i) {
    const double* r = rec + (size_t)i * R_N;
    if (r[R_VIS] == 0.0) continue;
    int ax, bx, ay, by;
    if (brute) {
      ax = 0; bx = W - 1; ay = 0; by = H - 1;
    } else {
      ax = (int)std::max(0.0, std::ceil(r[R_MX] - r[R_EX] - 1.0));
      bx = (int)std::min((double)W - 1, std::floor(r[R_MX] + r[R_EX] + 1.0));
      ay = (int)std::max(0.0, std::ceil(r[R_MY] - r[R_EY] - 1.0));
      by = (int)std::min((double)H - 1, std::floor(r[R_MY] + r[R_EY] + 1.0));
    }
    ax = std::max(ax, x0); bx = std::min(bx, x1);
    ay = std::max(ay, y0); by = std::min(by, y1);
    for (int y = ay; y <= by; ++y)
      for (int x = ax; x <= bx; ++x) L.cand[(size_t)y * W + x].push_back(i);
  }
  return L;
}

// One (pixel, Gaussian) counting decision (Eq. 1-3: alpha >= 1/255 and
// d < thr, thr = D_t + eps or +inf where the ray-cast missed) in FP64, and
// whether it lies within the error band of a single-precision evaluation
// (band: conic, mean, qmax, depth; see orc_envelope; null: never ambiguous):
// support ambiguous where |qmax - q| < qband = band[0] cn r^2 + 2 band[1] cn r
// + band[2] |qmax| (cn = |a| + 2|b| + |c|, r = |(dx, dy)|), depth where
// |d - thr| < band[3] thr; the pair is ambiguous where either test is near
// and the other passes or is near.
struct Decision {
  double q, G, alpha, dx, dy, qband;
  bool ref_in, ambiguous;
};

Decision classify(const double* r, int x, int y, double Dt, double eps, const double* band,
                  int f32 = 0) {
  const double thr = Dt > 0.0 ? Dt + eps : INFINITY;
  Decision d;
  d.dx = x - r[R_MX];
  d.dy = y - r[R_MY];
  d.q = r[R_CA] * d.dx * d.dx + 2.0 * r[R_CB] * d.dx * d.dy + r[R_CC] * d.dy * d.dy;
  d.G = std::exp(-0.5 * d.q);
  d.alpha = r[R_SIG] * d.G;
  if (f32) {
    const float tf = Dt > 0.0 ? (float)Dt + (float)eps : INFINITY;
    d.ref_in = support_f32((float)r[R_MX], (float)r[R_MY], (float)r[R_CA], (float)r[R_CB],
                           (float)r[R_CC], (float)r[R_QMAX], x, y) &&
               (float)r[R_D] < tf;
  } else {
    d.ref_in = d.alpha >= 1.0 / 255.0 && r[R_D] < thr;
  }
  d.qband = 0.0;
  d.ambiguous = false;
  if (band) {
    const double cn = std::fabs(r[R_CA]) + 2.0 * std::fabs(r[R_CB]) + std::fabs(r[R_CC]);
    const double r2 = d.dx * d.dx + d.dy * d.dy;
    d.qband = band[0] * cn * r2 + 2.0 * band[1] * cn * std::sqrt(r2) +
              band[2] * std::fabs(r[R_QMAX]);
    const bool in_s = d.q <= r[R_QMAX], near_s = std::fabs(r[R_QMAX] - d.q) < d.qband;
    const bool in_d = r[R_D] < thr,
               near_d = std::isfinite(thr) && std::fabs(r[R_D] - thr) < band[3] * thr;
    d.ambiguous = (near_s || near_d) && (in_s || near_s) && (in_d || near_d);
  }
  return d;
}

// SplitMix64 (Steele, Lea, Flood 2014): the diagnostic's coin per decision.
inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The Gaussians counted at pixel (x, y), sorted front to back by (d, index).
// f32 != 0: decisions in FP32 from the record's float values (see support_f32);
// otherwise alpha >= 1/255 and d < D_t + eps in FP64.
// flip (diagnostic only, nullable; 7 values: the 4 bands of `classify`, two
// unused, a seed): the decisions `classify` calls ambiguous are taken the
// other way (seed 0) or by a coin drawn from the seed, pixel and Gaussian -
// results a single-precision evaluation may reach.
std::vector<Item> counted(const std::vector<int>& cand, const double* rec, int x, int y,
                          double Dt, double eps, int f32, const double* flip = nullptr) {
  std::vector<Item> out;
  for (int i : cand) {
    const double* r = rec + (size_t)i * R_N;
    bool keep;
    const Decision d = classify(r, x, y, Dt, eps, flip);
    if (flip) {
      keep = d.ref_in;
      if (d.ambiguous) {
        const uint64_t seed = (uint64_t)flip[6];
        keep = seed == 0 ? !d.ref_in
                         : (mix64(seed ^ mix64(((uint64_t)y << 40) ^ ((uint64_t)x << 20) ^
                                               (uint64_t)i)) & 1) != 0;
      }
    } else if (f32) {
      float thr = Dt > 0.0 ? (float)Dt + (float)eps : INFINITY;
      keep = support_f32((float)r[R_MX], (float)r[R_MY], (float)r[R_CA], (float)r[R_CB],
                         (float)r[R_CC], (float)r[R_QMAX], x, y) &&
             (float)r[R_D] < thr;
    } else {
      keep = d.ref_in;
    }
    if (keep) out.push_back({i, d.alpha, d.G, d.dx, d.dy});
  }
  sort_front_to_back(out, rec, f32);
  return out;
}

// Per-pixel adjoint of the blend.  `its`: the Gaussians counted at the pixel,
// front to back; Ctp, Dtp: C_t, D_t there; g, gD: dL/dC* (3) and dL/dD*.
// out[k] (G_N entries, overwritten) receives item k's contribution to its
// Gaussian's 2D gradient.  Returns the number of items the blend uses (all in
// mode 0; mode 1 stops before the first that would take T below 1e-4).
//   mode 0 (Eq. 4), N = 1 + W_G:  dC*/dc_i = a_i / N,  dC*/da_i = (c_i - C*) / N;
//   mode 1: dC*/dc_i = a_i T_i,
//           dC*/da_i = c_i T_i - (sum_{j>i} c_j a_j T_j + T_end C_t) / (1 - a_i);
// likewise for depth (d_i in place of c_i).  Then through alpha = sigma G,
// G = exp(-q/2): dL/dsigma = dL/da G, dL/dq = -dL/da alpha / 2, dq/dconic and
// dq/dmean from q = a dx^2 + 2 b dx dy + c dy^2, dx = x - m_x.  An alpha
// clamped at 0.99 has zero derivative.
size_t pixel_adjoint(const std::vector<Item>& its, const double* rec, const double* Ctp, double Dtp,
                     const double* g, double gD, int mode,
                     std::vector<std::array<double, G_N>>& out) {
  const size_t n = its.size();
  out.assign(n, std::array<double, G_N>{});
  if (n == 0) return 0;
  std::vector<double> a(n), T(n), dLda(n), dLdd(n);
  std::vector<bool> clamped(n, false);
  std::vector<std::array<double, 3>> dLdc(n);
  size_t used = n;
  if (mode == 0) {
    double Cg[3] = {0, 0, 0}, Wg = 0, Z = 0;
    for (size_t k = 0; k < n; ++k) {
      const double* r = rec + (size_t)its[k].id * R_N;
      a[k] = its[k].alpha;
      for (int ch = 0; ch < 3; ++ch) Cg[ch] += r[R_R + ch] * a[k];
      Wg += a[k];
      Z += r[R_D] * a[k];
    }
    double N = 1.0 + Wg, Cs[3], Ds = (Dtp + Z) / N;
    for (int ch = 0; ch < 3; ++ch) Cs[ch] = (Ctp[ch] + Cg[ch]) / N;
    for (size_t k = 0; k < n; ++k) {
      const double* r = rec + (size_t)its[k].id * R_N;
      double v = 0;
      for (int ch = 0; ch < 3; ++ch) {
        dLdc[k][ch] = g[ch] * a[k] / N;
        v += g[ch] * (r[R_R + ch] - Cs[ch]) / N;
      }
      v += gD * (r[R_D] - Ds) / N;
      dLda[k] = v;
      dLdd[k] = gD * a[k] / N;
    }
  } else {
    double Tc = 1.0;
    used = 0;
    for (size_t k = 0; k < n; ++k) {
      double al = its[k].alpha;
      clamped[k] = al > 0.99;
      al = std::min(al, 0.99);
      if (Tc * (1.0 - al) < 1e-4) break;
      a[k] = al;
      T[k] = Tc;
      Tc *= (1.0 - al);
      ++used;
    }
    const double Tend = Tc;
    double S[3] = {Tend * Ctp[0], Tend * Ctp[1], Tend * Ctp[2]}, SD = Tend * Dtp;
    for (size_t kk = used; kk-- > 0;) {
      const double* r = rec + (size_t)its[kk].id * R_N;
      double v = 0;
      for (int ch = 0; ch < 3; ++ch) {
        dLdc[kk][ch] = g[ch] * a[kk] * T[kk];
        v += g[ch] * (r[R_R + ch] * T[kk] - S[ch] / (1.0 - a[kk]));
      }
      v += gD * (r[R_D] * T[kk] - SD / (1.0 - a[kk]));
      dLda[kk] = v;
      dLdd[kk] = gD * a[kk] * T[kk];
      for (int ch = 0; ch < 3; ++ch) S[ch] += r[R_R + ch] * a[kk] * T[kk];
      SD += r[R_D] * a[kk] * T[kk];
    }
  }
  for (size_t k = 0; k < used; ++k) {
    const double* r = rec + (size_t)its[k].id * R_N;
    std::array<double, G_N>& o = out[k];
    for (int ch = 0; ch < 3; ++ch) o[G_R + ch] = dLdc[k][ch];
    o[G_D] = dLdd[k];
    if (clamped[k]) continue;
    const double G = its[k].G, al = its[k].alpha, dx = its[k].dx, dy = its[k].dy;
    o[G_SIG] = dLda[k] * G;
    double dq = dLda[k] * (-0.5 * al);
    o[G_CA] = dq * dx * dx;
    o[G_CB] = dq * 2.0 * dx * dy;
    o[G_CC] = dq * dy * dy;
    // dq/dmean = -2 (conic . delta)
    o[G_MX] = dq * -2.0 * (r[R_CA] * dx + r[R_CB] * dy);
    o[G_MY] = dq * -2.0 * (r[R_CB] * dx + r[R_CC] * dy);
  }
  return used;
}

// Adjoint of one Gaussian's projection: its 2D gradient g (G_N entries) ->
// dm (mean, 3), dl (log-scales, 3), dq (quaternion, 4, through the
// normalisation), *dlogit and drgb (3).  P must be visible.  The Jacobian
// clamp is differentiated exactly (a clamped t_x' = +-lim t_z).  T = double
// is the adjoint; T = Mag evaluates its magnitudes (mag.h).
template <class T>
void proj_adjoint_t(const Cam& c, const Proj& P, const T* g, T* dm, T* dl, T* dq, T* dlogit,
                    T* drgb) {
  const double* R = c.R;
  for (int k = 0; k < 3; ++k) drgb[k] = g[G_R + k];
  *dlogit = g[G_SIG] * P.sig * (1.0 - P.sig);
  // conic = inverse(Sigma_2D): dL/dSigma_2D = -C Gs C with Gs the symmetric
  // gradient of the conic matrix (off-diagonals carry half of dL/db).
  const double Cm[4] = {P.conic[0], P.conic[1], P.conic[1], P.conic[2]};
  const T Gs[4] = {g[G_CA], 0.5 * g[G_CB], 0.5 * g[G_CB], g[G_CC]};
  T tmp[4], dS2[4];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      tmp[a * 2 + b] = 0.0;
      for (int k = 0; k < 2; ++k) tmp[a * 2 + b] += Cm[a * 2 + k] * Gs[k * 2 + b];
    }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      dS2[a * 2 + b] = 0.0;
      for (int k = 0; k < 2; ++k) dS2[a * 2 + b] -= tmp[a * 2 + k] * Cm[k * 2 + b];
    }
  // Sigma_2D = T Sigma T^T (+0.3 I): dT = 2 dS2 T Sigma, dSigma = T^T dS2 T
  T dT[6], dSig[9];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j) {
      T s = 0.0;
      for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 3; ++k) s += dS2[a * 2 + b] * P.T[b * 3 + k] * P.Sig[k * 3 + j];
      dT[a * 3 + j] = 2.0 * s;
    }
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      T s = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) s += P.T[a * 3 + k] * dS2[a * 2 + b] * P.T[b * 3 + l];
      dSig[k * 3 + l] = s;
    }
  // T = J W with W[k][j] = R[j][k]  =>  dJ[a][k] = sum_j dT[a][j] R[j][k]
  T dJ[6];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) {
      T s = 0.0;
      for (int j = 0; j < 3; ++j) s += dT[a * 3 + j] * R[j * 3 + k];
      dJ[a * 3 + k] = s;
    }
  const double tz = P.tc[2], tz2 = tz * tz, tz3 = tz2 * tz;
  T dtc[3] = {0.0, 0.0, 0.0};
  dtc[2] += dJ[0] * (-c.fx / tz2) + dJ[4] * (-c.fy / tz2) + dJ[2] * (2.0 * c.fx * P.txp / tz3) +
            dJ[5] * (2.0 * c.fy * P.typ / tz3);
  const T dtxp = dJ[2] * (-c.fx / tz2), dtyp = dJ[5] * (-c.fy / tz2);
  if (P.clx)
    dtc[2] += dtxp * (P.txp / tz);  // t_x' = +-lim t_z
  else
    dtc[0] += dtxp;
  if (P.cly)
    dtc[2] += dtyp * (P.typ / tz);
  else
    dtc[1] += dtyp;
  // mean2D = (fx tx / tz + cx, fy ty / tz + cy); depth = tz
  dtc[0] += g[G_MX] * c.fx / tz;
  dtc[1] += g[G_MY] * c.fy / tz;
  dtc[2] += -g[G_MX] * c.fx * P.tc[0] / tz2 - g[G_MY] * c.fy * P.tc[1] / tz2 + g[G_D];
  // tc = R^T (p - c)  =>  dp = R dtc
  for (int r = 0; r < 3; ++r) dm[r] = R[r * 3 + 0] * dtc[0] + R[r * 3 + 1] * dtc[1] + R[r * 3 + 2] * dtc[2];
  // Sigma = Mg Mg^T, Mg = Rg diag(s): dMg = 2 dSigma Mg
  double Mg[9];
  T dMg[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Mg[a * 3 + b] = P.Rg[a * 3 + b] * P.s[b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      T s = 0.0;
      for (int k = 0; k < 3; ++k) s += dSig[a * 3 + k] * Mg[k * 3 + b];
      dMg[a * 3 + b] = 2.0 * s;
    }
  T dRg[9];
  for (int b = 0; b < 3; ++b) {
    T ds = 0.0;
    for (int a = 0; a < 3; ++a) {
      dRg[a * 3 + b] = dMg[a * 3 + b] * P.s[b];
      ds += dMg[a * 3 + b] * P.Rg[a * 3 + b];
    }
    dl[b] = ds * P.s[b];
  }
  // rotation matrix entries as polynomials of the unit quaternion (w, x, y, z)
  const double w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
  T dqn[4];
  dqn[0] = dRg[1] * (-2 * z) + dRg[2] * (2 * y) + dRg[3] * (2 * z) + dRg[5] * (-2 * x) +
           dRg[6] * (-2 * y) + dRg[7] * (2 * x);
  dqn[1] = dRg[1] * (2 * y) + dRg[2] * (2 * z) + dRg[3] * (2 * y) + dRg[4] * (-4 * x) +
           dRg[5] * (-2 * w) + dRg[6] * (2 * z) + dRg[7] * (2 * w) + dRg[8] * (-4 * x);
  dqn[2] = dRg[0] * (-4 * y) + dRg[1] * (2 * x) + dRg[2] * (2 * w) + dRg[3] * (2 * x) +
           dRg[5] * (2 * z) + dRg[6] * (-2 * w) + dRg[7] * (2 * z) + dRg[8] * (-4 * y);
  dqn[3] = dRg[0] * (-4 * z) + dRg[1] * (-2 * w) + dRg[2] * (2 * x) + dRg[3] * (2 * w) +
           dRg[4] * (-4 * z) + dRg[5] * (2 * y) + dRg[6] * (2 * x) + dRg[7] * (2 * y);
  // qn = q / |q|: dq = (dqn - qn (qn . dqn)) / |q|
  T dot = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
  for (int k = 0; k < 4; ++k) dq[k] = (dqn[k] - P.qn[k] * dot) / P.qnorm;
}

void proj_adjoint(const Cam& c, const Proj& P, const double* g, double* dm, double* dl,
                  double* dq, double* dlogit, double* drgb) {
  proj_adjoint_t<double>(c, P, g, dm, dl, dq, dlogit, drgb);
}

struct EnvView {
  int M, W, H, mode, P, kmax, f32;
  const double *rec, *Ct, *Dt, *Ctgt, *Dtgt, *band, *JT;
  double eps, sc, sd, lambda;
  long n_valid;
  const double *dC, *dD;
};

struct EnvPixel {  // per-pixel results
  int n_amb = 0, unbounded = 0;
  double aC = 0, aD = 0, aW = 0, aL = 0;
};

// One pixel of orc_envelope.  With P > 0, the reference terms are added to
// g2ref / s2 / s2q and the parameter ranges to allow3 (callers run pixels of
// one view in sequence then); with P == 0 only the image and loss envelope.
EnvPixel envelope_pixel(const EnvView& v, const Lists& L, long pix, double* allow3,
                        double* g2ref, double* s2, double* s2q) {
  EnvPixel res;
  const long npx = (long)v.W * v.H;
  const int x = (int)(pix % v.W), y = (int)(pix / v.W);
  const double* rec = v.rec;
  const double Ctp[3] = {v.Ct[pix], v.Ct[npx + pix], v.Ct[2 * npx + pix]};
  const bool valid = v.Dtgt[pix] > 0.0 && v.Dt[pix] > 0.0 && v.n_valid > 0;
  auto sgn = [](double s) { return s > 0 ? 1.0 : (s < 0 ? -1.0 : 0.0); };
  // classify the candidates: fixed (decided as here whatever the rounding)
  // or ambiguous (within a band of a threshold)
  std::vector<Item> fixed, amb;
  std::vector<double> qb_fixed, qb_amb;
  std::vector<int> amb_ref;  // the FP64 decision of each ambiguous pair
  for (int i : L.cand[pix]) {
    const Decision d = classify(rec + (size_t)i * R_N, x, y, v.Dt[pix], v.eps, v.band, v.f32);
    if (d.ambiguous) {
      amb_ref.push_back(d.ref_in ? 1 : 0);
      amb.push_back({i, d.alpha, d.G, d.dx, d.dy});
      qb_amb.push_back(d.qband);
    } else if (d.ref_in) {
      fixed.push_back({i, d.alpha, d.G, d.dx, d.dy});
      qb_fixed.push_back(d.qband);
    }
  }
  const int k = (int)amb.size();
  // front-to-back blend: the order of two touched Gaussians whose depths lie
  // within the order band of each other, |d_a - d_b| < band (|d_a| + |d_b|),
  // is a decision of its own (either order follows from depths within their
  // rounding), one more bit per such pair: set, the two trade places in the
  // depth-sorted list
  std::vector<std::pair<int, int>> swaps;
  if (v.mode != 0 && v.band[6] > 0.0) {
    std::vector<std::pair<double, int>> byd;
    for (const Item& it : fixed) byd.push_back({rec[(size_t)it.id * R_N + R_D], it.id});
    for (const Item& it : amb) byd.push_back({rec[(size_t)it.id * R_N + R_D], it.id});
    std::sort(byd.begin(), byd.end());
    for (size_t a = 0; a < byd.size(); ++a)
      for (size_t b = a + 1; b < byd.size(); ++b) {
        if (byd[b].first - byd[a].first >= v.band[6] * (std::fabs(byd[a].first) + std::fabs(byd[b].first)))
          break;
        swaps.push_back({byd[a].second, byd[b].second});
      }
  }
  const int kd = k + (int)swaps.size();  // decision bits: k thresholds, then the pairs
  res.n_amb = kd;
  const bool too_many = kd > v.kmax;
  if (too_many) res.unbounded = 1;
  int ref_mask = 0;  // the pairs' reference bit is 0: the FP64 order
  if (!too_many)
    for (int j = 0; j < k; ++j) ref_mask |= amb_ref[j] << j;
  const size_t nf = fixed.size(), nu = nf + (size_t)k;  // the touched Gaussians
  const int P = v.P;
  std::vector<double> vmax(nu * P, -INFINITY), vmin(nu * P, INFINITY);
  std::vector<double> Cm, Dm, Wm, Lm;  // per combination
  std::vector<std::array<double, G_N>> terms, tch;
  bool any_free = false;
  // with too many ambiguous decisions only the FP64 combination is evaluated
  const int nmask = too_many ? 1 : (1 << kd);
  for (int mask = 0; mask < nmask; ++mask) {
    const int m = too_many ? ref_mask : mask;
    const bool is_ref = m == ref_mask;
    auto chosen = [&](int j) { return too_many ? amb_ref[j] != 0 : ((m >> j) & 1) != 0; };
    // the counted items, each with its slot in the union and its band
    std::vector<Item> its = fixed;
    std::vector<size_t> slot(nf);
    std::vector<double> qbs = qb_fixed;
    for (size_t t = 0; t < nf; ++t) slot[t] = t;
    for (int j = 0; j < k; ++j)
      if (chosen(j)) {
        its.push_back(amb[j]);
        slot.push_back(nf + (size_t)j);
        qbs.push_back(qb_amb[j]);
      }
    std::vector<size_t> ord(its.size());
    for (size_t t = 0; t < ord.size(); ++t) ord[t] = t;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) {
      double da = rec[(size_t)its[a].id * R_N + R_D], db = rec[(size_t)its[b].id * R_N + R_D];
      if (v.f32) {
        const float fa = (float)da, fb = (float)db;
        if (fa != fb) return fa < fb;
      } else if (da != db) {
        return da < db;
      }
      return its[a].id < its[b].id;
    });
    std::vector<Item> it2(its.size());
    std::vector<size_t> sl2(its.size());
    std::vector<double> qb2(its.size());
    for (size_t t = 0; t < ord.size(); ++t) {
      it2[t] = its[ord[t]];
      sl2[t] = slot[ord[t]];
      qb2[t] = qbs[ord[t]];
    }
    // the pair decisions of this combination: swapped pairs trade places
    if (!too_many)
      for (size_t j = 0; j < swaps.size(); ++j) {
        if (!((m >> (k + (int)j)) & 1)) continue;
        size_t pa = it2.size(), pb = it2.size();
        for (size_t t = 0; t < it2.size(); ++t) {
          if (it2[t].id == swaps[j].first) pa = t;
          if (it2[t].id == swaps[j].second) pb = t;
        }
        if (pa == it2.size() || pb == it2.size()) continue;
        std::swap(it2[pa], it2[pb]);
        std::swap(sl2[pa], sl2[pb]);
        std::swap(qb2[pa], qb2[pb]);
      }
    // C*, D* (Eq. 4, or the front-to-back variant)
    double Cs[3], Ds, Ws;
    if (v.mode == 0) {
      double Cg[3] = {0, 0, 0}, Wg = 0, Z = 0;
      for (const Item& it : it2) {
        const double* r = rec + (size_t)it.id * R_N;
        for (int ch = 0; ch < 3; ++ch) Cg[ch] += r[R_R + ch] * it.alpha;
        Wg += it.alpha;
        Z += r[R_D] * it.alpha;
      }
      for (int ch = 0; ch < 3; ++ch) Cs[ch] = (Ctp[ch] + Cg[ch]) / (1.0 + Wg);
      Ds = (v.Dt[pix] + Z) / (1.0 + Wg);
      Ws = Wg;
    } else {
      double Cg[3] = {0, 0, 0}, Z = 0, T = 1.0;
      for (const Item& it : it2) {
        const double* r = rec + (size_t)it.id * R_N;
        if (std::fabs(it.alpha - 0.99) < 1e-5) res.unbounded = 1;
        const double al = std::min(it.alpha, 0.99);
        const double test = T * (1.0 - al);
        if (std::fabs(test - 1e-4) < 1e-9) res.unbounded = 1;
        if (test < 1e-4) break;
        for (int ch = 0; ch < 3; ++ch) Cg[ch] += r[R_R + ch] * al * T;
        Z += r[R_D] * al * T;
        T = test;
      }
      for (int ch = 0; ch < 3; ++ch) Cs[ch] = Cg[ch] + T * Ctp[ch];
      Ds = Z + T * v.Dt[pix];
      Ws = 1.0 - T;
    }
    // upstream gradient: the L1 signs, and the channels whose sign is free
    double g[4] = {0, 0, 0, 0};
    bool freec[4] = {false, false, false, false};
    double Lx = 0.0;
    if (v.dC) {
      for (int ch = 0; ch < 3; ++ch) g[ch] = v.dC[ch * npx + pix];
      g[3] = v.dD[pix];
    } else if (valid) {
      for (int ch = 0; ch < 3; ++ch) {
        const double rr = Cs[ch] - v.Ctgt[ch * npx + pix];
        Lx += std::fabs(rr) * v.sc;
        g[ch] = sgn(rr) * v.sc;
        freec[ch] = std::fabs(rr) < v.band[4];
      }
      if (v.lambda != 0.0) {
        const double rd = Ds - v.Dtgt[pix];
        Lx += std::fabs(rd) * v.sd;
        g[3] = sgn(rd) * v.sd;
        freec[3] = std::fabs(rd) < v.band[5] * v.Dtgt[pix];
      }
    }
    Cm.insert(Cm.end(), Cs, Cs + 3);
    Dm.push_back(Ds);
    Wm.push_back(Ws);
    Lm.push_back(Lx);
    for (int ch = 0; ch < 4; ++ch) any_free = any_free || freec[ch];
    if (P == 0) continue;
    if (is_ref) {
      // the FP64 decisions: reference gradient and the rounding sums
      const size_t used = pixel_adjoint(it2, rec, Ctp, v.Dt[pix], g, g[3], v.mode, terms);
      for (size_t t = 0; t < used; ++t) {
        const size_t id = (size_t)it2[t].id;
        for (int c = 0; c < G_N; ++c) {
          g2ref[id * G_N + c] += terms[t][c];
          s2[id * G_N + c] += std::fabs(terms[t][c]);
          s2q[id * G_N + c] += std::fabs(terms[t][c]) * 0.5 * qb2[t];
        }
      }
    }
    if (res.unbounded || (kd == 0 && !any_free)) continue;
    // each touched Gaussian's term over this combination: base (free channels
    // at 0) +- the sum over free channels of |J^T t_ch|
    double gb[4];
    for (int ch = 0; ch < 4; ++ch) gb[ch] = freec[ch] ? 0.0 : g[ch];
    const size_t used = pixel_adjoint(it2, rec, Ctp, v.Dt[pix], gb, gb[3], v.mode, terms);
    std::vector<double> vb(nu * P, 0.0), vf(nu * P, 0.0);
    std::vector<char> present(nu, 0);
    auto project_term = [&](size_t t, const std::array<double, G_N>& tt, bool absval,
                            std::vector<double>& dst) {
      const size_t id = (size_t)it2[t].id, uu = sl2[t];
      present[uu] = 1;
      const double* J = v.JT + id * (size_t)P * G_N;
      for (int p = 0; p < P; ++p) {
        double a = 0.0;
        for (int c = 0; c < G_N; ++c) a += J[p * G_N + c] * tt[c];
        dst[uu * P + p] += absval ? std::fabs(a) : a;
      }
    };
    for (size_t t = 0; t < used; ++t) project_term(t, terms[t], false, vb);
    for (int ch = 0; ch < 4; ++ch) {
      if (!freec[ch]) continue;
      double gu[4] = {0, 0, 0, 0};
      gu[ch] = ch < 3 ? v.sc : v.sd;
      const size_t used2 = pixel_adjoint(it2, rec, Ctp, v.Dt[pix], gu, gu[3], v.mode, tch);
      for (size_t t = 0; t < used2; ++t) project_term(t, tch[t], true, vf);
    }
    for (size_t uu = 0; uu < nu; ++uu)
      for (int p = 0; p < P; ++p) {
        const double hi = present[uu] ? vb[uu * P + p] + vf[uu * P + p] : 0.0;
        const double lo = present[uu] ? vb[uu * P + p] - vf[uu * P + p] : 0.0;
        vmax[uu * P + p] = std::max(vmax[uu * P + p], hi);
        vmin[uu * P + p] = std::min(vmin[uu * P + p], lo);
      }
  }
  if (res.unbounded) {
    res.aC = res.aD = res.aW = INFINITY;
    return res;
  }
  if (kd == 0 && !any_free) return res;  // one combination, fixed signs: no range
  const size_t r0 = (size_t)ref_mask;
  for (size_t mm = 0; mm < Dm.size(); ++mm) {
    for (int ch = 0; ch < 3; ++ch)
      res.aC = std::max(res.aC, std::fabs(Cm[3 * mm + ch] - Cm[3 * r0 + ch]));
    res.aD = std::max(res.aD, std::fabs(Dm[mm] - Dm[r0]));
    res.aW = std::max(res.aW, std::fabs(Wm[mm] - Wm[r0]));
    res.aL = std::max(res.aL, std::fabs(Lm[mm] - Lm[r0]));
  }
  if (P > 0)
    for (size_t uu = 0; uu < nu; ++uu) {
      const size_t id = (size_t)(uu < nf ? fixed[uu].id : amb[uu - nf].id);
      for (int p = 0; p < P; ++p) allow3[id * P + p] += vmax[uu * P + p] - vmin[uu * P + p];
    }
  return res;
}

}  // namespace

extern "C" {

// Projection of M Gaussians into one view.  rec: M x R_N doubles (layout in the
// enum above).  amb[i] != 0 when a decision of the projection sits within a
// relative 1e-6 of its threshold: bit 0 the visibility (near plane, sigma >=
// 1/255), bit 1 the Jacobian clamp (continuous in the forward; only its
// derivative jumps), bit 2 the extent's test against the image border (within
// 1e-3 px).  Returns the number of visible Gaussians.
int orc_project(int M, const double* means, const double* log_scales, const double* quats,
                const double* logits, const double* rgb, int W, int H, const double* K,
                const double* R, const double* t, double near_, double* rec, int* amb) {
  Cam c{K[0], K[1], K[2], K[3], W, H, R, t};
  int nvis = 0;
  for (int i = 0; i < M; ++i) {
    Proj P = project_one(c, means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i], near_);
    double* r = rec + (size_t)i * R_N;
    std::memset(r, 0, sizeof(double) * R_N);
    r[R_MX] = P.mx; r[R_MY] = P.my; r[R_D] = P.tc[2]; r[R_SIG] = P.sig;
    r[R_CA] = P.conic[0]; r[R_CB] = P.conic[1]; r[R_CC] = P.conic[2]; r[R_QMAX] = P.qmax;
    r[R_R] = rgb[3 * i]; r[R_G] = rgb[3 * i + 1]; r[R_B] = rgb[3 * i + 2];
    r[R_EX] = P.ex; r[R_EY] = P.ey; r[R_VIS] = P.vis ? 1.0 : 0.0;
    r[R_S2XX] = P.S2[0]; r[R_S2YY] = P.S2[3];
    nvis += P.vis;
    if (amb) {
      const double limx = 1.3 * (W / (2.0 * K[0])), limy = 1.3 * (H / (2.0 * K[1]));
      double tz = P.tc[2];
      int a = (std::fabs(tz - near_) < 1e-6 * near_ ||
               std::fabs(P.sig - 1.0 / 255.0) < 1e-6 / 255.0) ? 1 : 0;
      if (tz > near_) {
        if (std::fabs(std::fabs(P.tc[0] / tz) - limx) < 1e-6 * limx ||
            std::fabs(std::fabs(P.tc[1] / tz) - limy) < 1e-6 * limy)
          a |= 2;
        if (P.det > 0 && P.sig >= 1.0 / 255.0 &&
            (std::fabs(P.mx + P.ex) < 1e-3 || std::fabs(P.mx - P.ex - (W - 1)) < 1e-3 ||
             std::fabs(P.my + P.ey) < 1e-3 || std::fabs(P.my - P.ey - (H - 1)) < 1e-3))
          a |= 4;
      }
      amb[i] = a;
    }
  }
  return nvis;
}

// Second rendering pass and blend for one view (Eq. 1-4, and the Table 7
// "with sort" variant when mode == 1).
//   mode 0 (order independent): C_G = sum c_i a_i, W_G = sum a_i, Z_G = sum d_i a_i
//          over counted Gaussians; C* = (C_t + C_G) / (1 + W_G) (W_t = 1, Eq. 4);
//          D* = (D_t + Z_G) / (1 + W_G) (the same blend applied to depth).
//   mode 1 (front to back): a_i <- min(a_i, 0.99); stop before the first i with
//          T (1 - a_i) < 1e-4; C* = sum c_i a_i T_i + T_end C_t (likewise D*),
//          W_G = 1 - T_end.
// Outputs: C* [3][H][W], D*, W_G, T_end, n_counted (all [H][W]); amb[pix] = 1 when
// a FP32 implementation could take a different clamp / termination decision.
// Window [x0, x1] x [y0, y1] restricts the work (pixels outside are left 0).
// flip: the diagnostic decisions of `counted`.
void orc_composite(int M, const double* rec, int W, int H, const double* Ct, const double* Dt,
                   double eps, int mode, int f32, int brute, int x0, int x1, int y0, int y1,
                   double* out_C, double* out_D, double* out_W, double* out_T, int* out_n,
                   int* amb, const double* flip) {
  Lists L = build_lists(M, rec, W, H, brute, x0, x1, y0, y1);
  const long npx = (long)W * H;
#pragma omp parallel for schedule(dynamic, 16)
  for (long pix = 0; pix < npx; ++pix) {
    int x = (int)(pix % W), y = (int)(pix / W);
    if (x < x0 || x > x1 || y < y0 || y > y1) continue;
    std::vector<Item> its = counted(L.cand[pix], rec, x, y, Dt[pix], eps, f32, flip);
    double C[3] = {0, 0, 0}, Z = 0, Wg = 0, T = 1.0;
    int n = 0;
    bool a = false;

    for (const Item& it : its) {
      const double* r = rec + (size_t)it.id * R_N;
      double al = it.alpha;
      if (mode == 0) {
        for (int ch = 0; ch < 3; ++ch) C[ch] += r[R_R + ch] * al;
        Wg += al;
        Z += r[R_D] * al;
        ++n;
      } else {
        if (std::fabs(al - 0.99) < 1e-5) a = true;
        al = std::min(al, 0.99);
        double test = T * (1.0 - al);
        if (std::fabs(test - 1e-4) < 1e-9) a = true;
        if (test < 1e-4) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += r[R_R + ch] * al * T;
        Z += r[R_D] * al * T;
        T = test;
        ++n;
      }
    }
    double Ctp[3] = {Ct[pix], Ct[npx + pix], Ct[2 * npx + pix]};
    if (mode == 0) {
      for (int ch = 0; ch < 3; ++ch) out_C[ch * npx + pix] = (Ctp[ch] + C[ch]) / (1.0 + Wg);
      out_D[pix] = (Dt[pix] + Z) / (1.0 + Wg);
      out_W[pix] = Wg;
      out_T[pix] = 1.0;
    } else {
      for (int ch = 0; ch < 3; ++ch) out_C[ch * npx + pix] = C[ch] + T * Ctp[ch];
      out_D[pix] = Z + T * Dt[pix];
      out_W[pix] = 1.0 - T;
      out_T[pix] = T;
    }
    out_n[pix] = n;
    if (amb) amb[pix] = a ? 1 : 0;
  }
}

// L1 loss (Sec. 3.2.2, Eq. 6) over valid pixels (target depth > 0 and ray-cast
// hit D_t > 0), averaged over the N_v valid pixels and the 3 channels, plus
// lambda_depth times the mean absolute depth error.  Writes dL/dC*, dL/dD*
// (sign(0) = 0) and returns L; *n_valid = N_v.  amb[pix] = 1 when a residual is
// within 1e-6 of zero (its sign is then not stable across precisions).
double orc_loss(int W, int H, const double* C, const double* D, const double* Ctgt,
                const double* Dtgt, const double* Dt, double lambda_depth, double* dC,
                double* dD, long* n_valid, int* amb) {
  const long npx = (long)W * H;
  long nv = 0;
  for (long p = 0; p < npx; ++p) nv += (Dtgt[p] > 0.0 && Dt[p] > 0.0);
  *n_valid = nv;
  double L = 0.0;
  auto sgn = [](double v) { return v > 0 ? 1.0 : (v < 0 ? -1.0 : 0.0); };
  for (long p = 0; p < npx; ++p) {
    bool valid = Dtgt[p] > 0.0 && Dt[p] > 0.0 && nv > 0;
    bool a = false;
    for (int ch = 0; ch < 3; ++ch) {
      double r = C[ch * npx + p] - Ctgt[ch * npx + p];
      if (valid) {
        L += std::fabs(r) / (3.0 * nv);
        dC[ch * npx + p] = sgn(r) / (3.0 * nv);
        if (std::fabs(r) < 1e-6) a = true;
      } else {
        dC[ch * npx + p] = 0.0;
      }
    }
    double rd = D[p] - Dtgt[p];
    if (valid && lambda_depth != 0.0) {
      L += lambda_depth * std::fabs(rd) / nv;
      dD[p] = lambda_depth * sgn(rd) / nv;
      if (std::fabs(rd) < 1e-6) a = true;
    } else {
      dD[p] = 0.0;
    }
    if (amb) amb[p] = a ? 1 : 0;
  }
  return L;
}

// Adjoint of orc_composite with respect to the per-Gaussian 2D quantities,
// accumulated into g2 (M x G_N, zeroed here): d/d mean(2), d/d conic (a, b, c
// with q = a dx^2 + 2 b dx dy + c dy^2), d/d sigma, d/d rgb(3), d/d depth.
// The counting decisions are constants; the per-pixel terms are those of
// pixel_adjoint, summed over the pixels in row-major order.
void orc_composite_backward(int M, const double* rec, int W, int H, const double* Ct,
                            const double* Dt, double eps, int mode, int f32, const double* dC,
                            const double* dD, double* g2, const double* flip) {
  Lists L = build_lists(M, rec, W, H, 0, 0, W - 1, 0, H - 1);
  std::memset(g2, 0, sizeof(double) * (size_t)M * G_N);
  const long npx = (long)W * H;
  std::vector<std::array<double, G_N>> terms;
  for (long pix = 0; pix < npx; ++pix) {
    int x = (int)(pix % W), y = (int)(pix / W);
    const double g[3] = {dC[pix], dC[npx + pix], dC[2 * npx + pix]};
    const double gD = dD[pix];
    if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0 && gD == 0.0) continue;  // contributes nothing
    std::vector<Item> its = counted(L.cand[pix], rec, x, y, Dt[pix], eps, f32, flip);
    if (its.empty()) continue;
    const double Ctp[3] = {Ct[pix], Ct[npx + pix], Ct[2 * npx + pix]};
    const size_t used = pixel_adjoint(its, rec, Ctp, Dt[pix], g, gD, mode, terms);
    for (size_t k = 0; k < used; ++k) {
      double* o = g2 + (size_t)its[k].id * G_N;
      for (int c = 0; c < G_N; ++c) o[c] += terms[k][c];
    }
  }
}

// Adjoint of orc_project: per-Gaussian 2D gradients (M x G_N) -> gradients of
// means, log-scales, quaternions (through the normalisation), opacity logits
// and rgb (proj_adjoint per Gaussian).  Outputs are overwritten.  Invisible
// Gaussians get zeros.
void orc_project_backward(int M, const double* means, const double* log_scales,
                          const double* quats, const double* logits, int W, int H,
                          const double* K, const double* R, const double* t, double near_,
                          const double* g2, double* d_means, double* d_ls, double* d_quats,
                          double* d_logits, double* d_rgb) {
  Cam c{K[0], K[1], K[2], K[3], W, H, R, t};
  for (int i = 0; i < M; ++i) {
    Proj P = project_one(c, means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i], near_);
    double* dm = d_means + 3 * i;
    double* dl = d_ls + 3 * i;
    double* dq = d_quats + 4 * i;
    for (int k = 0; k < 3; ++k) dm[k] = dl[k] = d_rgb[3 * i + k] = 0;
    for (int k = 0; k < 4; ++k) dq[k] = 0;
    d_logits[i] = 0;
    if (!P.vis) continue;
    proj_adjoint(c, P, g2 + (size_t)i * G_N, dm, dl, dq, d_logits + i, d_rgb + 3 * i);
  }
}

// Decision envelope of one view (test infrastructure for comparing a
// single-precision evaluation with this FP64 one).
//
// Gradient and image are sums over pixels of per-pixel terms (Eq. 4 and the
// Eq. 6 loss are per pixel; N_v does not depend on the Gaussians), and each
// pixel's terms depend only on that pixel's discrete decisions: which
// Gaussians count (alpha >= 1/255 and d < D_t + eps, Eq. 1-3) and the sign
// of each L1 residual.  A decision whose quantity lies within the error band
// of its threshold may be taken either way by an FP32 evaluation:
//   support:  |qmax - q| < qband = band[0] cn r^2 + 2 band[1] cn r + band[2] qmax,
//             cn = |a| + 2|b| + |c|, r = |(dx, dy)|: the change of q when the
//             conic moves by band[0] cn, the mean by band[1] px and qmax by
//             band[2] of itself (the FP32 rounding of q's own products is
//             below u cn r^2 and taken into band[0]);
//   depth:    |d - (D_t + eps)| < band[3] (D_t + eps);
//   colour residual |C* - C| < band[4], depth residual |D* - D| < band[5] D;
//   mode 1 (front to back) only, the order of two touched Gaussians:
//             |d_a - d_b| < band[6] (|d_a| + |d_b|) (a pair bit; set, the two
//             trade places in the sorted list; the FP64 order has it clear).
// Every other decision is taken as here.  Per pixel the envelope enumerates
// every combination of its k ambiguous counting decisions (k <= kmax, else
// the pixel is flagged in `unbounded`) and, per combination, lets each
// ambiguous residual sign range over +-1 (the terms are linear in the
// upstream gradient, so the extremes lie at the signs).  For every
// Gaussian touched and every parameter p it takes the range (max - min over
// the combinations, a Gaussian absent from a combination contributing 0) of
// the pixel's term J^T t, J^T = JT[i] (P x G_N, the projection adjoint of
// Gaussian i), and adds it to allow3[i][p].  So a single-precision gradient
// that decides everything outside the bands as here lies within allow3 of
// the FP64 gradient, up to its own rounding.  Likewise allow_img[0][pix]
// (max over channels), allow_img[1][pix] and allow_img[2][pix] bound
// |C* - C*_ref|, |D* - D*_ref| and |W_G - W_G,ref|, and *allow_loss the loss.
// Also returned: n_amb[pix] (ambiguous decisions, order pairs included), g2ref (the 2D
// gradient of the FP64 decisions, the sum of pixel_adjoint terms in row-major
// pixel order, as orc_composite_backward), s2[i][c] = sum over pixels of
// |term| and s2q[i][c] = sum over pixels of |term| * qband / 2 (alpha's
// relative error bound from q's band), both per 2D component.
// In mode 1 a pixel whose clamp or termination decision lies within 1e-5
// (1e-9 on T) of its threshold is flagged in `unbounded` too.
// f32 != 0: the counting decisions in FP32 as `counted` takes them (records
// holding FP32 values), nothing ambiguous: only g2ref, s2 and s2q are of use.
// dC, dD (nullable): explicit upstream gradients dL/dC*, dL/dD* in place of
// the L1 loss's (then no sign is free and the loss envelope is 0).
// Returns the number of unbounded pixels.
int orc_envelope(int M, const double* rec, int W, int H, const double* Ct, const double* Dt,
                 double eps, int mode, const double* Ctgt, const double* Dtgt, double lambda,
                 long n_valid, const double* band, int P, const double* JT, int kmax, int f32,
                 const double* dC, const double* dD, double* allow_img, double* allow_loss, int* n_amb, int* unbounded,
                 double* allow3, double* g2ref, double* s2, double* s2q) {
  Lists L = build_lists(M, rec, W, H, 0, 0, W - 1, 0, H - 1);
  const long npx = (long)W * H;
  const double no_band[7] = {0, 0, 0, 0, 0, 0, 0};
  if (f32) band = no_band;
  EnvView v{M, W, H, mode, P, kmax, f32, rec, Ct, Dt, Ctgt, Dtgt, band, JT, eps,
            n_valid > 0 ? 1.0 / (3.0 * (double)n_valid) : 0.0,
            n_valid > 0 ? lambda / (double)n_valid : 0.0, lambda, n_valid, dC, dD};
  if (P > 0) {
    std::memset(allow3, 0, sizeof(double) * (size_t)M * P);
    std::memset(g2ref, 0, sizeof(double) * (size_t)M * G_N);
    std::memset(s2, 0, sizeof(double) * (size_t)M * G_N);
    std::memset(s2q, 0, sizeof(double) * (size_t)M * G_N);
  }
  std::vector<EnvPixel> res((size_t)npx);
  if (P > 0) {
    // per-Gaussian sums in row-major pixel order (g2ref equals
    // orc_composite_backward's sum bit for bit)
    for (long pix = 0; pix < npx; ++pix)
      res[pix] = envelope_pixel(v, L, pix, allow3, g2ref, s2, s2q);
  } else {
#pragma omp parallel for schedule(dynamic, 64)
    for (long pix = 0; pix < npx; ++pix)
      res[pix] = envelope_pixel(v, L, pix, nullptr, nullptr, nullptr, nullptr);
  }
  int n_unb = 0;
  double aL = 0.0;
  for (long pix = 0; pix < npx; ++pix) {
    n_amb[pix] = res[pix].n_amb;
    unbounded[pix] = res[pix].unbounded;
    allow_img[pix] = res[pix].aC;
    allow_img[npx + pix] = res[pix].aD;
    allow_img[2 * npx + pix] = res[pix].aW;
    aL += res[pix].aL;
    n_unb += res[pix].unbounded;
  }
  *allow_loss = aL;
  return n_unb;
}

// Magnitudes of orc_project_backward's results (same arguments; outputs
// overwritten): the adjoint evaluated in magnitude arithmetic (mag.h) from
// |g2|, so that a single-precision adjoint's rounding error is bounded by a
// small multiple of u times these, per element.
void orc_project_backward_mag(int M, const double* means, const double* log_scales,
                              const double* quats, const double* logits, int W, int H,
                              const double* K, const double* R, const double* t, double near_,
                              const double* g2, double* d_means, double* d_ls, double* d_quats,
                              double* d_logits, double* d_rgb) {
  Cam c{K[0], K[1], K[2], K[3], W, H, R, t};
  for (int i = 0; i < M; ++i) {
    Proj P = project_one(c, means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i], near_);
    Mag g[G_N], dm[3], dl[3], dq[4], dlg, drgb[3];
    for (int k = 0; k < G_N; ++k) g[k] = Mag(g2[(size_t)i * G_N + k]);
    if (P.vis) proj_adjoint_t<Mag>(c, P, g, dm, dl, dq, &dlg, drgb);
    for (int k = 0; k < 3; ++k) {
      d_means[3 * i + k] = dm[k].v;
      d_ls[3 * i + k] = dl[k].v;
      d_rgb[3 * i + k] = drgb[k].v;
    }
    for (int k = 0; k < 4; ++k) d_quats[4 * i + k] = dq[k].v;
    d_logits[i] = dlg.v;
  }
}

// OpenMP threads of the oracle's parallel loops (for timing it single-threaded
// and on all cores); returns the previous maximum.
int orc_set_threads(int n) {
  const int prev = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return prev;
}

// Tile binning from FP32 projected records (the kernels' record layout, 16
// floats per Gaussian: mx, my, d, sigma, a, b, c, qmax, r, g, b, ext_x, ext_y, ...).
// Pixel rectangle, in float: [ceil(mx - ext_x), floor(mx + ext_x)] clipped to
// [0, W-1] (likewise y); a Gaussian with ext_x < 0 or an empty rectangle has no
// pairs.  Tiles: [x0 / TW, x1 / TW] x [y0 / TH, y1 / TH].  Key = tile << 32 |
// bits(d); value = Gaussian index; pairs sorted by (key, index) with
// std::stable_sort.  ranges[2 t], ranges[2 t + 1] = [start, end) of tile t.
// Returns the number of pairs (or -1 if it exceeds cap).
long orc_bin(int M, const float* rec32, int W, int H, int TW, int TH, long cap,
             uint64_t* keys, uint32_t* vals, uint32_t* ranges) {
  const int ntx = (W + TW - 1) / TW, nty = (H + TH - 1) / TH;
  std::vector<std::pair<uint64_t, uint32_t>> pairs;
  for (int i = 0; i < M; ++i) {
    const float* r = rec32 + (size_t)i * 16;
    float ex = r[11], ey = r[12];
    if (!(ex >= 0.0f) || !(ey >= 0.0f)) continue;
    float lx = r[0] - ex, hx = r[0] + ex, ly = r[1] - ey, hy = r[1] + ey;
    if (!(hx >= 0.0f) || !(lx <= (float)(W - 1)) || !(hy >= 0.0f) || !(ly <= (float)(H - 1)))
      continue;
    int x0 = std::max(0, (int)std::ceil(std::max(lx, -1.0f)));
    int x1 = std::min(W - 1, (int)std::floor(std::min(hx, (float)W)));
    int y0 = std::max(0, (int)std::ceil(std::max(ly, -1.0f)));
    int y1 = std::min(H - 1, (int)std::floor(std::min(hy, (float)H)));
    if (x0 > x1 || y0 > y1) continue;
    uint32_t dbits;
    std::memcpy(&dbits, &r[2], 4);
    for (int ty = y0 / TH; ty <= y1 / TH; ++ty)
      for (int tx = x0 / TW; tx <= x1 / TW; ++tx) {
        uint64_t tile = (uint64_t)(ty * ntx + tx);
        pairs.push_back({(tile << 32) | dbits, (uint32_t)i});
      }
  }
  std::stable_sort(pairs.begin(), pairs.end(),
                   [](const std::pair<uint64_t, uint32_t>& a,
                      const std::pair<uint64_t, uint32_t>& b) { return a.first < b.first; });
  const long P = (long)pairs.size();
  for (int tIdx = 0; tIdx < ntx * nty; ++tIdx) ranges[2 * tIdx] = ranges[2 * tIdx + 1] = 0;
  if (P > cap) return -1;
  for (long k = 0; k < P; ++k) {
    keys[k] = pairs[k].first;
    vals[k] = pairs[k].second;
    uint32_t tile = (uint32_t)(pairs[k].first >> 32);
    if (k == 0 || (uint32_t)(pairs[k - 1].first >> 32) != tile) ranges[2 * tile] = (uint32_t)k;
    ranges[2 * tile + 1] = (uint32_t)(k + 1);
  }
  return P;
}

// Adam (App. C learning rates; torch.optim.Adam semantics, in place, FP64):
//   m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
//   p <- p - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)
void orc_adam(long n, double* p, const double* g, double* m, double* v, double lr, double b1,
              double b2, double eps, int step) {
  const double bc1 = 1.0 - std::pow(b1, step), bc2 = 1.0 - std::pow(b2, step);
  for (long k = 0; k < n; ++k) {
    m[k] = b1 * m[k] + (1.0 - b1) * g[k];
    v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
    double denom = std::sqrt(v[k]) / std::sqrt(bc2) + eps;
    p[k] -= (lr / bc1) * m[k] / denom;
  }
}

}  // extern "C"
