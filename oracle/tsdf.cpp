// Oracle (test infrastructure only): colourised TSDF fusion and SDF ray-cast in FP64.
//
// Plain, slow, obviously-correct restatement of the supporting steps of the
// Gaussian-plus-SDF renderer:
//   * fusion  - Sec. 3.2.1 "SDF fusion": each voxel keeps a truncated signed
//               distance d(p) and a colour c(p) (Sec. 3.1), updated by the
//               standard weighted running average (KinectFusion / InfiniTAM);
//   * ray-cast - Sec. 3.1 first rendering pass: march every pixel's ray to the
//               zero crossing V^g(u), C_t(u) = trilinear colour of the eight
//               neighbouring voxels, D_t(u) = depth of V^g(u) in the camera.
// Readings where the paper is silent (step rule, secant refinement, colour
// weight, rounding of the projected pixel) are stated at each function.
//
// Storage here is linear, x fastest: idx = x + nx * (y + ny * z).  Only tests,
// the package smoke check and the benchmark's CPU-baseline leg may call this.
#include <cmath>
#include <cstdint>
#include <algorithm>

namespace {

struct Vol {
  int nx, ny, nz;
  double voxel, ox, oy, oz, trunc, wmax;
  long idx(int x, int y, int z) const { return x + (long)nx * (y + (long)ny * z); }
};

Vol make_vol(const int* dims, const double* geo) {
  Vol v;
  v.nx = dims[0]; v.ny = dims[1]; v.nz = dims[2];
  v.voxel = geo[0]; v.ox = geo[1]; v.oy = geo[2]; v.oz = geo[3];
  v.trunc = geo[4]; v.wmax = geo[5];
  return v;
}

// world -> camera: X_c = R^T (X_w - t), R camera->world row-major.
inline void world_to_cam(const double* R, const double* t, const double* xw, double* xc) {
  double d0 = xw[0] - t[0], d1 = xw[1] - t[1], d2 = xw[2] - t[2];
  for (int i = 0; i < 3; ++i) xc[i] = R[0 * 3 + i] * d0 + R[1 * 3 + i] * d1 + R[2 * 3 + i] * d2;
}

// Trilinear interpolation of a per-voxel field at continuous voxel coordinate g
// (voxel centres at integer g).  The 8-voxel stencil is clamped to the grid.
double trilinear(const Vol& v, const double* f, int stride, int comp, const double* g) {
  int i0[3];
  double fr[3];
  const int n[3] = {v.nx, v.ny, v.nz};
  for (int k = 0; k < 3; ++k) {
    double gk = g[k];
    int i = (int)std::floor(gk);
    if (i < 0) i = 0;
    if (i > n[k] - 2) i = n[k] - 2;
    i0[k] = i;
    fr[k] = gk - i;
  }
  double acc = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? fr[0] : 1.0 - fr[0]) * (dy ? fr[1] : 1.0 - fr[1]) *
                   (dz ? fr[2] : 1.0 - fr[2]);
        acc += w * f[v.idx(i0[0] + dx, i0[1] + dy, i0[2] + dz) * stride + comp];
      }
  return acc;
}

// Width of the band around a truncation threshold inside which a
// single-precision evaluation of eta = D - z_c may fall on the other side:
// z_c comes from a float transform of metre-scale coordinates (rounding about
// 1e-7 m), so the band is 1e-6 of the magnitudes involved, in metres.
inline double eta_band(double D, double zc) { return 1e-6 * (1.0 + std::fabs(D) + std::fabs(zc)); }

}  // namespace

extern "C" {

// Colourised TSDF fusion of one RGB-D frame (Sec. 3.2.1, "standard SDF fusion").
// For each voxel centre x_v = origin + (idx + 0.5) * voxel:
//   x_c = R^T (x_v - t); skip unless z_c > 0;
//   (u, v) = (fx x/z + cx, fy y/z + cy), nearest pixel = floor(u + 0.5), floor(v + 0.5);
//   skip unless the pixel is inside the image and its depth D > 0;
//   eta = D - z_c; skip if eta < -trunc;
//   f = min(1, eta / trunc); sdf <- (w sdf + f) / (w + 1); w <- min(w + 1, wmax);
//   if |eta| < trunc: rgb <- (cw rgb + C) / (cw + 1); cw <- min(cw + 1, wmax)
// (the colour keeps its own weight cw, as InfiniTAM's coloured voxels do).
// amb[v] |= 1 when a discrete decision of this update sits within rounding
// reach of its threshold (pixel rounding within a relative 1e-6; truncation
// tests within eta_band), so a single-precision implementation may
// legitimately take the other branch.
//
// Voxel hashing (Sec. 3.2.1: the SDF lives in a hash table of voxel blocks,
// as in InfiniTAM), when `alloc` (one byte per 8^3 brick, brick index
// bx + nbx (by + nby bz)) is given: before the update, every brick holding a
// voxel with |eta| < trunc for this frame (the same projection and pixel as
// above) is allocated (alloc = 1, for good); then only voxels of allocated
// bricks are updated.  Unallocated bricks keep sdf 1, weight 0, colour 0.
// amb[v] |= 2 marks a voxel whose band decision sits within eta_band of
// trunc, or whose pixel rounding is within a relative 1e-6.
void orc_fuse(const int* dims, const double* geo, double* sdf, double* w, double* rgb,
              double* cw, int* amb, const double* depth, const double* img, int W, int H,
              const double* K, const double* R, const double* t, unsigned char* alloc) {
  const Vol v = make_vol(dims, geo);
  const double fx = K[0], fy = K[1], cx = K[2], cy = K[3];
  const long n = (long)v.nx * v.ny * v.nz;
  const int nbx = v.nx / 8, nby = v.ny / 8;
  auto brick = [&](long id) {
    int x = (int)(id % v.nx), y = (int)((id / v.nx) % v.ny), z = (int)(id / ((long)v.nx * v.ny));
    return (long)(x / 8) + nbx * ((long)(y / 8) + (long)nby * (z / 8));
  };
  if (alloc) {
#pragma omp parallel for schedule(static)
    for (long id = 0; id < n; ++id) {
      int x = (int)(id % v.nx), y = (int)((id / v.nx) % v.ny), z = (int)(id / ((long)v.nx * v.ny));
      double xw[3] = {v.ox + (x + 0.5) * v.voxel, v.oy + (y + 0.5) * v.voxel,
                      v.oz + (z + 0.5) * v.voxel};
      double xc[3];
      world_to_cam(R, t, xw, xc);
      if (!(xc[2] > 0.0)) continue;
      double u = fx * xc[0] / xc[2] + cx, vv = fy * xc[1] / xc[2] + cy;
      double fu = u + 0.5 - std::floor(u + 0.5), fv = vv + 0.5 - std::floor(vv + 0.5);
      bool near_round = std::min(fu, 1.0 - fu) < 1e-6 * std::max(1.0, std::fabs(u)) ||
                        std::min(fv, 1.0 - fv) < 1e-6 * std::max(1.0, std::fabs(vv));
      double pu = std::floor(u + 0.5), pv = std::floor(vv + 0.5);
      if (pu < 0 || pv < 0 || pu > W - 1 || pv > H - 1) continue;
      double D = depth[(long)pv * W + (long)pu];
      if (!(D > 0.0)) continue;
      double eta = D - xc[2];
      if (amb && (near_round || std::fabs(std::fabs(eta) - v.trunc) < eta_band(D, xc[2])))
        amb[id] |= 2;
      if (std::fabs(eta) < v.trunc) {
#pragma omp atomic write
        alloc[brick(id)] = 1;
      }
    }
  }
#pragma omp parallel for schedule(static)
  for (long id = 0; id < n; ++id) {
    if (alloc && !alloc[brick(id)]) continue;
    int x = (int)(id % v.nx), y = (int)((id / v.nx) % v.ny), z = (int)(id / ((long)v.nx * v.ny));
    double xw[3] = {v.ox + (x + 0.5) * v.voxel, v.oy + (y + 0.5) * v.voxel,
                    v.oz + (z + 0.5) * v.voxel};
    double xc[3];
    world_to_cam(R, t, xw, xc);
    if (!(xc[2] > 0.0)) continue;
    double u = fx * xc[0] / xc[2] + cx, vv = fy * xc[1] / xc[2] + cy;
    double fu = u + 0.5 - std::floor(u + 0.5), fv = vv + 0.5 - std::floor(vv + 0.5);
    bool near_round = std::min(fu, 1.0 - fu) < 1e-6 * std::max(1.0, std::fabs(u)) ||
                      std::min(fv, 1.0 - fv) < 1e-6 * std::max(1.0, std::fabs(vv));
    double pu = std::floor(u + 0.5), pv = std::floor(vv + 0.5);
    if (pu < 0 || pv < 0 || pu > W - 1 || pv > H - 1) {
      if (amb && near_round) amb[id] |= 1;
      continue;
    }
    long pix = (long)pv * W + (long)pu;
    double D = depth[pix];
    if (!(D > 0.0)) {
      if (amb && near_round) amb[id] |= 1;
      continue;
    }
    double eta = D - xc[2];
    if (amb && (near_round || std::fabs(eta + v.trunc) < eta_band(D, xc[2]) ||
                std::fabs(std::fabs(eta) - v.trunc) < eta_band(D, xc[2])))
      amb[id] |= 1;
    if (eta < -v.trunc) continue;
    double f = std::min(1.0, eta / v.trunc);
    double w0 = w[id];
    sdf[id] = (w0 * sdf[id] + f) / (w0 + 1.0);
    w[id] = std::min(w0 + 1.0, v.wmax);
    if (std::fabs(eta) < v.trunc) {
      double c0 = cw[id];
      for (int ch = 0; ch < 3; ++ch)
        rgb[id * 3 + ch] = (c0 * rgb[id * 3 + ch] + img[(long)ch * W * H + pix]) / (c0 + 1.0);
      cw[id] = std::min(c0 + 1.0, v.wmax);
    }
  }
}

// SDF ray-cast (Sec. 3.1 first pass; marching "as in InfiniTAM").
// Ray of pixel (i, j): origin t, direction dir = normalize(R ((i-cx)/fx, (j-cy)/fy, 1)).
// The march is confined to the box spanned by the voxel centres, starting at
// max(near, box entry) and ending at min(far, box exit) (far <= 0: box exit).
// f(s) = trilinear sdf at o + s dir.  Step = max(min(f, 1) * trunc, 0.5 voxel)
// (a full truncation band while f == 1).  The first sample pair with
// f_a > 0 >= f_b is a hit; secant refinement s* = s_a + (s_b - s_a) f_a / (f_a - f_b).
// V^g = o + s* dir; D_t = camera z of V^g; C_t = trilinear of the 8 voxel colours.
// No hit: D_t = 0, C_t = 0, vertex = 0.
// amb[pix] = 1 when a single-precision march may decide differently: each
// sample's position is tracked with a running bound ds on how far an FP32
// march's sample can be from this one (the entry point's and every addition's
// rounding, a few u s, plus trunc times the FP32 error of the f that set the
// step, where the step follows f), and f's bound df = |df/ds| ds + |grad f|
// dp + 8 u (the local slope along the ray; dp, the rounding of the FP32 grid
// coordinates of the sample, off the ray; the trilinear's own rounding); a
// sample whose |f| < df, or whose position lies within ds of the march end,
// flags the pixel.  In noisy stretches of a fused volume the slope amplifies
// ds from sample to sample, as it does the FP32 march's drift.
// out_depth_err (nullable): per pixel, a bound on how far an FP32 march's
// hit depth can be from this one's: the secant root re-solved with the
// bracket ends moved by their bounds (0 where nothing was hit).
// sdf_err (nullable, per voxel, >= 0): how far the other march's volume may
// differ from this one (an FP32 fusion of the same frames); its trilinear
// interpolation adds to every sample's df.
void orc_raycast(const int* dims, const double* geo, const double* sdf, const double* rgb,
                 int W, int H, const double* K, const double* R, const double* t,
                 double near_, double far_, double* out_rgb, double* out_depth,
                 double* out_vertex, int* amb, double* out_depth_err, const double* sdf_err) {
  const Vol v = make_vol(dims, geo);
  const double fx = K[0], fy = K[1], cx = K[2], cy = K[3];
  const double lo[3] = {v.ox + 0.5 * v.voxel, v.oy + 0.5 * v.voxel, v.oz + 0.5 * v.voxel};
  const double hi[3] = {v.ox + (v.nx - 0.5) * v.voxel, v.oy + (v.ny - 0.5) * v.voxel,
                        v.oz + (v.nz - 0.5) * v.voxel};
  const long npx = (long)W * H;
#pragma omp parallel for schedule(dynamic, 64)
  for (long pix = 0; pix < npx; ++pix) {
    const int i = (int)(pix % W), j = (int)(pix / W);
    double dc[3] = {(i - cx) / fx, (j - cy) / fy, 1.0};
    double dw[3];
    for (int r = 0; r < 3; ++r) dw[r] = R[r * 3 + 0] * dc[0] + R[r * 3 + 1] * dc[1] + R[r * 3 + 2] * dc[2];
    double nrm = std::sqrt(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
    for (int r = 0; r < 3; ++r) dw[r] /= nrm;
    double s_in = -INFINITY, s_out = INFINITY;
    for (int k = 0; k < 3; ++k) {
      if (dw[k] != 0.0) {
        double a = (lo[k] - t[k]) / dw[k], b = (hi[k] - t[k]) / dw[k];
        s_in = std::max(s_in, std::min(a, b));
        s_out = std::min(s_out, std::max(a, b));
      } else if (t[k] < lo[k] || t[k] > hi[k]) {
        s_in = INFINITY;
      }
    }
    double s0 = std::max(near_, s_in);
    double s1 = far_ > 0.0 ? std::min(far_, s_out) : s_out;
    out_rgb[pix] = out_rgb[npx + pix] = out_rgb[2 * npx + pix] = 0.0;
    out_depth[pix] = 0.0;
    if (out_vertex) out_vertex[pix * 3] = out_vertex[pix * 3 + 1] = out_vertex[pix * 3 + 2] = 0.0;
    if (amb) amb[pix] = 0;
    if (out_depth_err) out_depth_err[pix] = 0.0;
    if (!(s0 < s1)) continue;
    auto sample = [&](double s) {
      double g[3];
      const double o3[3] = {v.ox, v.oy, v.oz};
      for (int k = 0; k < 3; ++k) g[k] = (t[k] + s * dw[k] - o3[k]) / v.voxel - 0.5;
      return trilinear(v, sdf, 1, 0, g);
    };
    // |df/ds| near s: the larger one-sided difference over h (the trilinear
    // field is piecewise smooth; h spans the position uncertainty)
    auto slope = [&](double s, double f, double h) {
      return std::max(std::fabs(sample(s + h) - f), std::fabs(f - sample(s - h))) / h;
    };
    // |grad f| at the sample at s: central differences along the axes
    auto grad_norm = [&](double s) {
      const double h = 0.01 * v.voxel, o3[3] = {v.ox, v.oy, v.oz};
      double gsq = 0.0;
      for (int a = 0; a < 3; ++a) {
        double gp[3], gm[3];
        for (int k = 0; k < 3; ++k) {
          const double p = t[k] + s * dw[k] + (k == a ? h : 0.0);
          const double m = t[k] + s * dw[k] - (k == a ? h : 0.0);
          gp[k] = (p - o3[k]) / v.voxel - 0.5;
          gm[k] = (m - o3[k]) / v.voxel - 0.5;
        }
        const double d = (trilinear(v, sdf, 1, 0, gp) - trilinear(v, sdf, 1, 0, gm)) / (2.0 * h);
        gsq += d * d;
      }
      return std::sqrt(gsq);
    };
    constexpr double u = 5.9604644775390625e-8;  // 2^-24
    // an FP32 sample at s also sits off the ray by the rounding of the grid
    // coordinates go + s gd (go from |t - origin|, gd from the direction)
    const double t_off = std::sqrt((t[0] - v.ox) * (t[0] - v.ox) + (t[1] - v.oy) * (t[1] - v.oy) +
                                   (t[2] - v.oz) * (t[2] - v.oz));
    auto f_err = [&](double s, double f, double ds) {
      const double dp = u * (2.0 * t_off + 5.0 * std::fabs(s) + v.voxel);
      double e = slope(s, f, std::max(ds, 1e-7)) * ds + grad_norm(s) * dp + 8.0 * u;
      if (sdf_err) {
        double g[3];
        const double o3[3] = {v.ox, v.oy, v.oz};
        for (int k = 0; k < 3; ++k) g[k] = (t[k] + s * dw[k] - o3[k]) / v.voxel - 0.5;
        e += trilinear(v, sdf_err, 1, 0, g);
      }
      return e;
    };
    const double s1_err = 4.0 * u * s1;
    double sa = s0, fa = sample(sa);
    double dsa = 4.0 * u * std::fabs(s0);
    double dfa = f_err(sa, fa, dsa);
    bool hit = false, ambig = std::fabs(fa) < dfa;
    double sb = 0.0, fb = 0.0, dsb = 0.0;
    while (true) {
      const double fs = std::min(fa, 1.0) * v.trunc;
      double step = std::max(fs, 0.5 * v.voxel);
      sb = sa + step;
      // the step follows f only where min(f, 1) trunc sets it
      dsb = dsa + (fs > 0.5 * v.voxel && fa < 1.0 ? v.trunc * dfa : 0.0) +
            u * (std::fabs(sb) + step);
      if (std::fabs(sb - s1) < dsb + s1_err) ambig = true;
      if (sb > s1) break;
      fb = sample(sb);
      const double dfb = f_err(sb, fb, dsb);
      if (std::fabs(fb) < dfb) ambig = true;
      if (fa > 0.0 && fb <= 0.0) {
        hit = true;
        break;
      }
      sa = sb;
      fa = fb;
      dsa = dsb;
      dfa = dfb;
    }
    if (amb) amb[pix] = ambig ? 1 : 0;
    if (!hit) continue;
    double ss = sa + (sb - sa) * fa / (fa - fb);
    double V[3] = {t[0] + ss * dw[0], t[1] + ss * dw[1], t[2] + ss * dw[2]};
    double xc[3];
    world_to_cam(R, t, V, xc);
    out_depth[pix] = xc[2];
    if (out_depth_err) {
      // the secant solved again with each bracket end moved by its position
      // bound (f sampled there) and f off by its rounding; the largest move
      // of the root, plus the secant's and the camera transform's roundings,
      // scaled by the ray's camera z per unit length
      double droot = 0.0;
      const double ra = f_err(sa, fa, 0.0), rb = f_err(sb, fb, 0.0);
      for (int c = 0; c < 16; ++c) {
        const double sa2 = sa + ((c & 1) ? dsa : -dsa), sb2 = sb + ((c & 2) ? dsb : -dsb);
        const double fa2 = sample(sa2) + ((c & 4) ? ra : -ra);
        const double fb2 = sample(sb2) + ((c & 8) ? rb : -rb);
        if (!(fa2 > fb2)) {
          droot = INFINITY;
          break;
        }
        droot = std::max(droot, std::fabs(sa2 + (sb2 - sa2) * fa2 / (fa2 - fb2) - ss));
      }
      const double dz = std::fabs(xc[2] / ss);  // camera z per unit of ray length
      out_depth_err[pix] = (droot + 8.0 * u * ss) * dz + 8.0 * u * std::fabs(xc[2]);
    }
    double g[3] = {(V[0] - v.ox) / v.voxel - 0.5, (V[1] - v.oy) / v.voxel - 0.5,
                   (V[2] - v.oz) / v.voxel - 0.5};
    for (int ch = 0; ch < 3; ++ch) out_rgb[ch * npx + pix] = trilinear(v, rgb, 3, ch, g);
    if (out_vertex)
      for (int k = 0; k < 3; ++k) out_vertex[pix * 3 + k] = V[k];
  }
}

}  // extern "C"
