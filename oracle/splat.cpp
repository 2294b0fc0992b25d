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

// The Gaussians counted at pixel (x, y), sorted front to back by (d, index).
// f32 != 0: decisions in FP32 from the record's float values (see support_f32);
// otherwise alpha >= 1/255 and d < D_t + eps in FP64.
// flip (diagnostic only, nullable): decisions lying within the error band of
// their threshold (flip[0]: conic, flip[1]: depth; see the allowance in
// orc_composite) are taken the other way, giving the result a single-precision
// evaluation reaches when it decides each of them differently.
std::vector<Item> counted(const std::vector<int>& cand, const double* rec, int x, int y,
                          double Dt, double eps, int f32, const double* flip = nullptr) {
  std::vector<Item> out;
  for (int i : cand) {
    const double* r = rec + (size_t)i * R_N;
    double dx = x - r[R_MX], dy = y - r[R_MY];
    double q = r[R_CA] * dx * dx + 2.0 * r[R_CB] * dx * dy + r[R_CC] * dy * dy;
    double G = std::exp(-0.5 * q);
    double alpha = r[R_SIG] * G;
    bool keep;
    if (flip) {
      const double thr = Dt > 0.0 ? Dt + eps : INFINITY;
      const double cn = std::fabs(r[R_CA]) + 2.0 * std::fabs(r[R_CB]) + std::fabs(r[R_CC]);
      const double qband = flip[0] * (std::fabs(q) + cn * (dx * dx + dy * dy));
      const bool in_s = q <= r[R_QMAX], near_s = std::fabs(r[R_QMAX] - q) < qband;
      const bool in_d = r[R_D] < thr, near_d = std::isfinite(thr) && std::fabs(r[R_D] - thr) < flip[1] * thr;
      keep = (in_s != near_s) && (in_d != near_d);
      if (keep) out.push_back({i, alpha, G, dx, dy});
      continue;
    }
    if (f32) {
      float thr = Dt > 0.0 ? (float)Dt + (float)eps : INFINITY;
      keep = support_f32((float)r[R_MX], (float)r[R_MY], (float)r[R_CA], (float)r[R_CB],
                         (float)r[R_CC], (float)r[R_QMAX], x, y) &&
             (float)r[R_D] < thr;
    } else {
      double thr = Dt > 0.0 ? Dt + eps : INFINITY;
      keep = alpha >= 1.0 / 255.0 && r[R_D] < thr;
    }
    if (keep) out.push_back({i, alpha, G, dx, dy});
  }
  std::stable_sort(out.begin(), out.end(), [&](const Item& a, const Item& b) {
    double da = rec[(size_t)a.id * R_N + R_D], db = rec[(size_t)b.id * R_N + R_D];
    if (f32) {
      float fa = (float)da, fb = (float)db;
      if (fa != fb) return fa < fb;
    } else if (da != db) {
      return da < db;
    }
    return a.id < b.id;
  });
  return out;
}

}  // namespace

extern "C" {

// Projection of M Gaussians into one view.  rec: M x R_N doubles (layout in the
// enum above).  amb[i] = 1 when a visibility or clamp decision sits within a
// relative 1e-6 of its threshold.  Returns the number of visible Gaussians.
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
      bool a = std::fabs(tz - near_) < 1e-6 * near_ ||
               std::fabs(P.sig - 1.0 / 255.0) < 1e-6 / 255.0;
      if (tz > near_) {
        a = a || std::fabs(std::fabs(P.tc[0] / tz) - limx) < 1e-6 * limx ||
            std::fabs(std::fabs(P.tc[1] / tz) - limy) < 1e-6 * limy;
        if (P.det > 0 && P.sig >= 1.0 / 255.0) {
          a = a || std::fabs(P.mx + P.ex) < 1e-3 || std::fabs(P.mx - P.ex - (W - 1)) < 1e-3 ||
              std::fabs(P.my + P.ey) < 1e-3 || std::fabs(P.my - P.ey - (H - 1)) < 1e-3;
        }
      }
      amb[i] = a ? 1 : 0;
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
void orc_composite(int M, const double* rec, int W, int H, const double* Ct, const double* Dt,
                   double eps, int mode, int f32, int brute, int x0, int x1, int y0, int y1,
                   double* out_C, double* out_D, double* out_W, double* out_T, int* out_n,
                   int* amb, const double* band, double* allow, double* g_amb, double* g_mass,
                   const double* flip) {
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
    if (allow) {
      // Bound on how much C* (allow[0]) and D* (allow[1]) can move
      // if every counting decision lying within the error band of its
      // threshold were taken the other way, as a single-precision evaluation
      // may.  Support: |qmax - q| < band[0] (|q| + (|a| + 2|b| + |c|)(dx^2 + dy^2)),
      // the rounding error of q from a conic known to a relative band[0];
      // depth: |d - (D_t + eps)| < band[1] (D_t + eps).  g_amb / g_mass collect,
      // per Gaussian, the alpha of such decisions and its total counted alpha.
      const double thr = Dt[pix] > 0.0 ? Dt[pix] + eps : INFINITY;
      const double N = 1.0 + Wg;
      const double Cs[3] = {out_C[pix], out_C[npx + pix], out_C[2 * npx + pix]};
      double aC = 0.0, aD = 0.0;
      for (int i : L.cand[pix]) {
        const double* r = rec + (size_t)i * R_N;
        double dx = x - r[R_MX], dy = y - r[R_MY];
        double q = r[R_CA] * dx * dx + 2.0 * r[R_CB] * dx * dy + r[R_CC] * dy * dy;
        double al = r[R_SIG] * std::exp(-0.5 * q);
        const double cn = std::fabs(r[R_CA]) + 2.0 * std::fabs(r[R_CB]) + std::fabs(r[R_CC]);
        const double qband = band[0] * (std::fabs(q) + cn * (dx * dx + dy * dy));
        bool near_s = std::fabs(r[R_QMAX] - q) < qband;
        bool near_d = std::isfinite(thr) && std::fabs(r[R_D] - thr) < band[1] * thr;
        bool in_s = q <= r[R_QMAX] + qband;
        bool cnt = al >= 1.0 / 255.0 && r[R_D] < thr;
        if (cnt) {
#pragma omp atomic
          g_mass[i] += al;
        }
        if (!(near_s || (near_d && in_s))) continue;
        double dc = 0.0;
        for (int ch = 0; ch < 3; ++ch) dc = std::max(dc, std::fabs(r[R_R + ch] - Cs[ch]));
        if (mode == 0) {
          // exact change of (C_t + C_G) / N when alpha leaves (N - alpha) or joins (N + alpha)
          const double Nm = std::max(N - al, 1.0);
          aC += al * dc / Nm;
          aD += al * std::fabs(r[R_D] - out_D[pix]) / Nm;
        } else {
          aC += al * (1.0 + 1.0 / (1.0 - std::min(al, 0.99)));
          aD += al * (r[R_D] + out_D[pix] / (1.0 - std::min(al, 0.99)));
        }
#pragma omp atomic
        g_amb[i] += al;
      }
      allow[pix] = a ? INFINITY : aC;
      allow[npx + pix] = a ? INFINITY : aD;
    }
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
// The counting decisions are constants; alpha clamped at 0.99 has zero
// derivative.  Mode 0 (Eq. 4): with N = 1 + W_G,
//   dC*/dc_i = a_i / N,  dC*/da_i = (c_i - C*) / N,  and likewise for depth.
// Mode 1: dC*/dc_i = a_i T_i,  dC*/da_i = c_i T_i - (sum_{j>i} c_j a_j T_j + T_end C_t) / (1 - a_i).
void orc_composite_backward(int M, const double* rec, int W, int H, const double* Ct,
                            const double* Dt, double eps, int mode, int f32, const double* dC,
                            const double* dD, double* g2, const double* flip) {
  Lists L = build_lists(M, rec, W, H, 0, 0, W - 1, 0, H - 1);
  std::memset(g2, 0, sizeof(double) * (size_t)M * G_N);
  const long npx = (long)W * H;
  for (long pix = 0; pix < npx; ++pix) {
    int x = (int)(pix % W), y = (int)(pix / W);
    const double g[3] = {dC[pix], dC[npx + pix], dC[2 * npx + pix]};
    const double gD = dD[pix];
    if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0 && gD == 0.0) continue;  // contributes nothing
    std::vector<Item> its = counted(L.cand[pix], rec, x, y, Dt[pix], eps, f32, flip);
    if (its.empty()) continue;
    const double Ctp[3] = {Ct[pix], Ct[npx + pix], Ct[2 * npx + pix]};
    const size_t n = its.size();
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
      double N = 1.0 + Wg, Cs[3], Ds = (Dt[pix] + Z) / N;
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
      double S[3] = {Tend * Ctp[0], Tend * Ctp[1], Tend * Ctp[2]}, SD = Tend * Dt[pix];
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
      double* o = g2 + (size_t)its[k].id * G_N;
      for (int ch = 0; ch < 3; ++ch) o[G_R + ch] += dLdc[k][ch];
      o[G_D] += dLdd[k];
      if (clamped[k]) continue;
      // alpha = sigma G, G = exp(-q/2)
      const double G = its[k].G, al = its[k].alpha, dx = its[k].dx, dy = its[k].dy;
      o[G_SIG] += dLda[k] * G;
      double dq = dLda[k] * (-0.5 * al);
      o[G_CA] += dq * dx * dx;
      o[G_CB] += dq * 2.0 * dx * dy;
      o[G_CC] += dq * dy * dy;
      // dq/dmean = -2 (conic . delta)
      o[G_MX] += dq * -2.0 * (r[R_CA] * dx + r[R_CB] * dy);
      o[G_MY] += dq * -2.0 * (r[R_CB] * dx + r[R_CC] * dy);
    }
  }
}

// Adjoint of orc_project: per-Gaussian 2D gradients (M x G_N) -> gradients of
// means, log-scales, quaternions (through the normalisation), opacity logits
// and rgb.  Outputs are overwritten.  Invisible Gaussians get zeros.  The
// Jacobian clamp is differentiated exactly (a clamped t_x' = +-lim t_z).
void orc_project_backward(int M, const double* means, const double* log_scales,
                          const double* quats, const double* logits, int W, int H,
                          const double* K, const double* R, const double* t, double near_,
                          const double* g2, double* d_means, double* d_ls, double* d_quats,
                          double* d_logits, double* d_rgb) {
  Cam c{K[0], K[1], K[2], K[3], W, H, R, t};
  for (int i = 0; i < M; ++i) {
    Proj P = project_one(c, means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i], near_);
    const double* g = g2 + (size_t)i * G_N;
    double* dm = d_means + 3 * i;
    double* dl = d_ls + 3 * i;
    double* dq = d_quats + 4 * i;
    for (int k = 0; k < 3; ++k) dm[k] = dl[k] = d_rgb[3 * i + k] = 0;
    for (int k = 0; k < 4; ++k) dq[k] = 0;
    d_logits[i] = 0;
    if (!P.vis) continue;
    for (int k = 0; k < 3; ++k) d_rgb[3 * i + k] = g[G_R + k];
    d_logits[i] = g[G_SIG] * P.sig * (1.0 - P.sig);
    // conic = inverse(Sigma_2D): dL/dSigma_2D = -C Gs C with Gs the symmetric
    // gradient of the conic matrix (off-diagonals carry half of dL/db).
    const double Cm[4] = {P.conic[0], P.conic[1], P.conic[1], P.conic[2]};
    const double Gs[4] = {g[G_CA], 0.5 * g[G_CB], 0.5 * g[G_CB], g[G_CC]};
    double tmp[4], dS2[4];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        tmp[a * 2 + b] = 0;
        for (int k = 0; k < 2; ++k) tmp[a * 2 + b] += Cm[a * 2 + k] * Gs[k * 2 + b];
      }
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        dS2[a * 2 + b] = 0;
        for (int k = 0; k < 2; ++k) dS2[a * 2 + b] -= tmp[a * 2 + k] * Cm[k * 2 + b];
      }
    // Sigma_2D = T Sigma T^T (+0.3 I): dT = 2 dS2 T Sigma, dSigma = T^T dS2 T
    double dT[6], dSig[9];
    for (int a = 0; a < 2; ++a)
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int b = 0; b < 2; ++b)
          for (int k = 0; k < 3; ++k) s += dS2[a * 2 + b] * P.T[b * 3 + k] * P.Sig[k * 3 + j];
        dT[a * 3 + j] = 2.0 * s;
      }
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        double s = 0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) s += P.T[a * 3 + k] * dS2[a * 2 + b] * P.T[b * 3 + l];
        dSig[k * 3 + l] = s;
      }
    // T = J W with W[k][j] = R[j][k]  =>  dJ[a][k] = sum_j dT[a][j] R[j][k]
    double dJ[6];
    for (int a = 0; a < 2; ++a)
      for (int k = 0; k < 3; ++k) {
        double s = 0;
        for (int j = 0; j < 3; ++j) s += dT[a * 3 + j] * R[j * 3 + k];
        dJ[a * 3 + k] = s;
      }
    const double tz = P.tc[2], tz2 = tz * tz, tz3 = tz2 * tz;
    double dtc[3] = {0, 0, 0};
    dtc[2] += dJ[0] * (-c.fx / tz2) + dJ[4] * (-c.fy / tz2) + dJ[2] * (2.0 * c.fx * P.txp / tz3) +
              dJ[5] * (2.0 * c.fy * P.typ / tz3);
    const double dtxp = dJ[2] * (-c.fx / tz2), dtyp = dJ[5] * (-c.fy / tz2);
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
    double Mg[9], dMg[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Mg[a * 3 + b] = P.Rg[a * 3 + b] * P.s[b];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += dSig[a * 3 + k] * Mg[k * 3 + b];
        dMg[a * 3 + b] = 2.0 * s;
      }
    double dRg[9];
    for (int b = 0; b < 3; ++b) {
      double ds = 0;
      for (int a = 0; a < 3; ++a) {
        dRg[a * 3 + b] = dMg[a * 3 + b] * P.s[b];
        ds += dMg[a * 3 + b] * P.Rg[a * 3 + b];
      }
      dl[b] = ds * P.s[b];
    }
    // rotation matrix entries as polynomials of the unit quaternion (w, x, y, z)
    const double w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
    double dqn[4];
    dqn[0] = dRg[1] * (-2 * z) + dRg[2] * (2 * y) + dRg[3] * (2 * z) + dRg[5] * (-2 * x) +
             dRg[6] * (-2 * y) + dRg[7] * (2 * x);
    dqn[1] = dRg[1] * (2 * y) + dRg[2] * (2 * z) + dRg[3] * (2 * y) + dRg[4] * (-4 * x) +
             dRg[5] * (-2 * w) + dRg[6] * (2 * z) + dRg[7] * (2 * w) + dRg[8] * (-4 * x);
    dqn[2] = dRg[0] * (-4 * y) + dRg[1] * (2 * x) + dRg[2] * (2 * w) + dRg[3] * (2 * x) +
             dRg[5] * (2 * z) + dRg[6] * (-2 * w) + dRg[7] * (2 * z) + dRg[8] * (-4 * y);
    dqn[3] = dRg[0] * (-4 * z) + dRg[1] * (-2 * w) + dRg[2] * (2 * x) + dRg[3] * (2 * w) +
             dRg[4] * (-4 * z) + dRg[5] * (2 * y) + dRg[6] * (2 * x) + dRg[7] * (2 * y);
    // qn = q / |q|: dq = (dqn - qn (qn . dqn)) / |q|
    double dot = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
    for (int k = 0; k < 4; ++k) dq[k] = (dqn[k] - P.qn[k] * dot) / P.qnorm;
  }
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
