"""FP64 CPU oracle of the Gaussian-plus-SDF hot path - TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  It shares no code with the CUDA path
(`paper_2509_11574_b300`), which never imports it.

The arithmetic lives in `tsdf.cpp` (fusion, ray-cast), `splat.cpp`
(projection, compositing Eq. 1-4 and the Table 7 "with sort" variant, L1 loss
Eq. 6, adjoints, tile binning, Adam) and `sh.cpp` (view-dependent colour from
spherical harmonics of degree 1-3 and its adjoint).  This module builds `liboracle.so` with
g++ (FP64, `-ffp-contract=off`, OpenMP over independent pixels / voxels) and
wraps it with ctypes on float64 numpy arrays.

Parity status per function (what pins it, see tests/test_oracle_*.py):
  fuse              - fronto-parallel plane closed form, weight / re-fusion invariants
  fuse (hashed)     - the bricks a plane allocates, by hand; dense arithmetic
                      inside allocated bricks; closed-form values of a brick
                      allocated in a later frame (tests/test_oracle_hash.py)
  raycast           - analytic plane / box (exact) and sphere (0.1 voxel) hits
  project           - on-axis isotropic closed form, off-axis hand value, invariances
  composite (OIT)   - 1- and 2-Gaussian hand blends, M = 0, eps limits, brute force,
                      permutation invariance
  composite (ALPHA) - 1-Gaussian blend, opaque limit, termination count by hand;
                      the paper never writes this variant, so its formula is a reading
  loss              - torch.nn.functional.l1_loss (FP64)
  backward          - central finite differences (FP64) end to end, rotation
                      invariance, single-Gaussian closed form
  bin               - brute-force enumeration of tiles + Python sorted()
  adam              - torch.optim.Adam (FP64)
  quantise          - torch's float16 / bfloat16 casts, tie-to-even hand values
  sh (sh.cpp)       - basis = sqrt2 Re / Im of scipy's complex harmonics (Condon-
                      Shortley phase), orthonormal under exact quadrature; closed-
                      form colours and parity under d -> -d; colour and whole-loss
                      gradients (SH coefficients, means via the view direction)
                      against central differences
  edit.py (insertion / removal, Sec. 3.2 and App. A, plain numpy):
    splitmix64      - the generator's published outputs from seed 0
    sampling        - fraction and uniformity over 10^6 pixels, seed independence
    mask, removal   - threshold cases by hand
    insert          - planes: means, colours, opacity, disc radius from pixel
                      spacing, short axis on the analytic normal (scipy Rotation)
  icp.py (camera tracking, Sec. 3.2, Eq. 5, point-to-plane ICP, plain numpy):
    se3_exp         - scipy.linalg.expm of the twist matrix
    residual / J    - central differences of the residual under exp(xi) T
    pyramid, normals- 2x2 means and coarse intrinsics by hand; a tilted plane's
                      analytic normal
    track           - a rendered frame's known pose recovered from a 2 cm /
                      1.5 degree start (3 seeds); a single plane leaves the
                      pose unchanged (singular system)
  schedule.py (keyframes and optimisation views, Sec. 3.2, Fig. 5, App. C):
    is_keyframe     - rotations (scipy) and translations just under / over the
                      thresholds, relative to a rotated last keyframe
    local frames    - spacing by hand
    global draw     - a hand value from SplitMix64's published first output;
                      history bounds, no repeats; marginal, first-draw and pair
                      frequencies of a uniform draw without replacement
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRCS = [os.path.join(_HERE, f) for f in ("tsdf.cpp", "splat.cpp", "sh.cpp")]
_HDRS = [os.path.join(_HERE, "mag.h")]

# projected record layout (FP64), mirrors the enum in splat.cpp
R_MX, R_MY, R_D, R_SIG, R_CA, R_CB, R_CC, R_QMAX, R_R, R_G, R_B, R_EX, R_EY, R_VIS, \
    R_S2XX, R_S2YY = range(16)
R_N = 16
# per-Gaussian 2D gradient layout
G_MX, G_MY, G_CA, G_CB, G_CC, G_SIG, G_R, G_G, G_B, G_D = range(10)
G_N = 10

OIT, ALPHA = 0, 1
# storage types of the colour images (the values of the C-ABI's GPS_PREC_*)
FP32, FP16, BF16 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the sources (g++, FP64, OpenMP)."""
    newest = max(os.path.getmtime(s) for s in _SRCS + _HDRS)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _SO] + _SRCS
        subprocess.check_call(cmd)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        _lib.orc_project.restype = ctypes.c_int
        _lib.orc_loss.restype = ctypes.c_double
        _lib.orc_bin.restype = ctypes.c_long
        _lib.orc_set_threads.restype = ctypes.c_int
    return _lib


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's parallel loops; returns the previous count."""
    return int(lib().orc_set_threads(ctypes.c_int(n)))


def _p(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "arrays passed to the oracle must be contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _cam(cam):
    K = _f64([cam.fx, cam.fy, cam.cx, cam.cy])
    return K, _f64(cam.R).reshape(9), _f64(cam.t).reshape(3)


def _vol(spec):
    dims = np.ascontiguousarray([spec.nx, spec.ny, spec.nz], dtype=np.int32)
    geo = _f64([spec.voxel, *spec.origin, spec.trunc, spec.max_weight])
    return dims, geo


class Volume:
    """FP64 TSDF in linear storage (x fastest): sdf, w, cw [nz][ny][nx], rgb [...][3].
    Unobserved voxels: sdf = 1, w = 0, rgb = 0, cw = 0.  hashed=True gives the
    voxel-hashing semantics: `alloc` [nz/8][ny/8][nx/8] marks the allocated
    bricks, and only their voxels are ever updated (see orc_fuse)."""

    def __init__(self, spec, hashed: bool = False):
        self.spec = spec
        shape = (spec.nz, spec.ny, spec.nx)
        self.sdf = np.ones(shape)
        self.w = np.zeros(shape)
        self.rgb = np.zeros(shape + (3,))
        self.cw = np.zeros(shape)
        self.amb = np.zeros(shape, dtype=np.int32)
        self.alloc = (np.zeros((spec.nz // 8, spec.ny // 8, spec.nx // 8), np.uint8)
                      if hashed else None)


def fuse(vol: Volume, depth, rgb, cam) -> None:
    """Sec. 3.2.1 SDF fusion of one frame into `vol` (in place)."""
    dims, geo = _vol(vol.spec)
    K, R, t = _cam(cam)
    d = _f64(depth)
    c = _f64(rgb)
    lib().orc_fuse(_p(dims), _p(geo), _p(vol.sdf), _p(vol.w), _p(vol.rgb), _p(vol.cw),
                   _p(vol.amb), _p(d), _p(c), ctypes.c_int(cam.width), ctypes.c_int(cam.height),
                   _p(K), _p(R), _p(t), _p(vol.alloc))


def raycast(spec, sdf, rgb, cam, near=0.2, far=0.0, depth_err=False, sdf_err=None):
    """Sec. 3.1 first pass.  Returns (C_t [3][H][W], D_t [H][W], vertex [H][W][3], amb),
    plus, with depth_err, a per-pixel bound on an FP32 march's hit depth error.
    sdf_err (per voxel, like sdf): how far an FP32 march's volume may differ."""
    dims, geo = _vol(spec)
    K, R, t = _cam(cam)
    H, W = cam.height, cam.width
    out_rgb = np.zeros((3, H, W))
    out_d = np.zeros((H, W))
    out_v = np.zeros((H, W, 3))
    amb = np.zeros((H, W), dtype=np.int32)
    err = np.zeros((H, W)) if depth_err else None
    lib().orc_raycast(_p(dims), _p(geo), _p(_f64(sdf)), _p(_f64(rgb)), ctypes.c_int(W),
                      ctypes.c_int(H), _p(K), _p(R), _p(t), ctypes.c_double(near),
                      ctypes.c_double(far), _p(out_rgb), _p(out_d), _p(out_v), _p(amb), _p(err),
                      _p(_f64(sdf_err)) if sdf_err is not None else None)
    return (out_rgb, out_d, out_v, amb, err) if depth_err else (out_rgb, out_d, out_v, amb)


def _sh_degree(g) -> int:
    return int(getattr(g, "sh_degree", 0) or 0)


def sh_basis(dirs, degree: int) -> np.ndarray:
    """Real orthonormal SH Y_lm (l = 1..degree, m = -l..l) at unit directions
    dirs [n][3] -> [n][(degree + 1)^2 - 1]."""
    d = _f64(dirs).reshape(-1, 3)
    K = (degree + 1) ** 2 - 1
    Y = np.zeros((d.shape[0], K))
    lib().orc_sh_basis(ctypes.c_int(d.shape[0]), ctypes.c_int(degree), _p(d), _p(Y))
    return Y


def sh_colour(g, cam) -> np.ndarray:
    """View-dependent colour [M][3] of a GaussianSet seen from cam's centre
    (rgb itself when the set has no SH coefficients)."""
    rgb = _f64(g.rgb)
    D = _sh_degree(g)
    if D == 0:
        return rgb
    out = np.zeros_like(rgb)
    lib().orc_sh_colour(ctypes.c_int(g.M), ctypes.c_int(D), _p(_f64(g.means)), _p(rgb),
                        _p(_f64(g.sh_rest)), _p(_f64(cam.t).reshape(3)), _p(out))
    return out


def project(g, cam, near=0.2):
    """Projection of a GaussianSet into one view -> (rec [M][16] f64, amb [M])."""
    M = g.M
    arrs = [_f64(a) for a in g.arrays()]
    arrs[4] = sh_colour(g, cam)
    K, R, t = _cam(cam)
    rec = np.zeros((M, R_N))
    amb = np.zeros(M, dtype=np.int32)
    lib().orc_project(ctypes.c_int(M), *[_p(a) for a in arrs[:4]], _p(arrs[4]),
                      ctypes.c_int(cam.width), ctypes.c_int(cam.height), _p(K), _p(R), _p(t),
                      ctypes.c_double(near), _p(rec), _p(amb))
    return rec, amb


def composite(rec, Ct, Dt, eps, mode=OIT, f32=False, brute=False, window=None, flip=None):
    """Eq. 1-4 (mode OIT) or the Table 7 variant (mode ALPHA) for one view.
    Returns dict C [3][H][W], D, W (= W_G), T (T_end), n (counted) and amb
    (ALPHA clamp / termination decisions near their thresholds).
    flip (diagnostic, see `flip_spec`): the decisions inside the error bands
    taken the other way, or by a seeded coin."""
    Ct = _f64(Ct)
    Dt = _f64(Dt)
    H, W = Dt.shape
    x0, x1, y0, y1 = window if window is not None else (0, W - 1, 0, H - 1)
    rec = _f64(rec)
    M = rec.shape[0]
    out = dict(C=np.zeros((3, H, W)), D=np.zeros((H, W)), W=np.zeros((H, W)),
               T=np.zeros((H, W)), n=np.zeros((H, W), np.int32), amb=np.zeros((H, W), np.int32))
    lib().orc_composite(ctypes.c_int(M), _p(rec), ctypes.c_int(W), ctypes.c_int(H),
                        _p(Ct), _p(Dt), ctypes.c_double(eps), ctypes.c_int(mode),
                        ctypes.c_int(int(f32)), ctypes.c_int(int(brute)), ctypes.c_int(x0),
                        ctypes.c_int(x1), ctypes.c_int(y0), ctypes.c_int(y1), _p(out["C"]),
                        _p(out["D"]), _p(out["W"]), _p(out["T"]), _p(out["n"]), _p(out["amb"]),
                        _p(_f64(flip)) if flip is not None else None)
    return out


def flip_spec(bands: dict, seed=0) -> np.ndarray:
    """The `flip` argument of composite / composite_backward / render_loss_grads:
    the decisions `envelope` calls ambiguous under `bands` (see `bands_for`)
    are inverted (seed 0) or decided by a coin drawn from the seed
    (diagnostic only)."""
    b = bands
    return _f64([b["conic"], b["mean"], b["qmax"], b["depth"], 0.0, 0.0, float(seed)])


def loss(C, D, Ctgt, Dtgt, Dt, lambda_depth=0.0):
    """Eq. 6 L1 loss -> (L, dL/dC* [3][H][W], dL/dD* [H][W], N_v, amb)."""
    C, D, Ctgt, Dtgt, Dt = (_f64(a) for a in (C, D, Ctgt, Dtgt, Dt))
    H, W = D.shape
    dC = np.zeros((3, H, W))
    dD = np.zeros((H, W))
    nv = ctypes.c_long(0)
    amb = np.zeros((H, W), np.int32)
    L = lib().orc_loss(ctypes.c_int(W), ctypes.c_int(H), _p(C), _p(D), _p(Ctgt), _p(Dtgt),
                       _p(Dt), ctypes.c_double(lambda_depth), _p(dC), _p(dD), ctypes.byref(nv),
                       _p(amb))
    return float(L), dC, dD, int(nv.value), amb


def composite_backward(rec, Ct, Dt, eps, dC, dD, mode=OIT, f32=False, flip=None):
    """Adjoint of `composite` -> per-Gaussian 2D gradients [M][10]."""
    rec = _f64(rec)
    Ct, Dt, dC, dD = (_f64(a) for a in (Ct, Dt, dC, dD))
    H, W = Dt.shape
    g2 = np.zeros((rec.shape[0], G_N))
    lib().orc_composite_backward(ctypes.c_int(rec.shape[0]), _p(rec), ctypes.c_int(W),
                                 ctypes.c_int(H), _p(Ct), _p(Dt), ctypes.c_double(eps),
                                 ctypes.c_int(mode), ctypes.c_int(int(f32)), _p(dC), _p(dD),
                                 _p(g2), _p(_f64(flip)) if flip is not None else None)
    return g2


def project_backward(g, cam, g2, near=0.2):
    """Adjoint of `project` -> dict of gradients (means, log_scales, quats,
    opacity_logits, rgb, and sh_rest when the set has SH coefficients),
    float64."""
    M = g.M
    arrs = [_f64(a) for a in g.arrays()]
    K, R, t = _cam(cam)
    out = dict(means=np.zeros((M, 3)), log_scales=np.zeros((M, 3)), quats=np.zeros((M, 4)),
               opacity_logits=np.zeros(M), rgb=np.zeros((M, 3)))
    lib().orc_project_backward(ctypes.c_int(M), *[_p(a) for a in arrs[:4]],
                               ctypes.c_int(cam.width), ctypes.c_int(cam.height), _p(K), _p(R),
                               _p(t), ctypes.c_double(near), _p(_f64(g2)), _p(out["means"]),
                               _p(out["log_scales"]), _p(out["quats"]),
                               _p(out["opacity_logits"]), _p(out["rgb"]))
    D = _sh_degree(g)
    if D > 0:
        # the colour gradient reaches rgb unchanged, the SH coefficients through
        # Y_lm(d) and the mean through the viewing direction d
        out["sh_rest"] = np.zeros(g.sh_rest.shape)
        lib().orc_sh_backward(ctypes.c_int(M), ctypes.c_int(D), _p(arrs[0]),
                              _p(_f64(g.sh_rest)), _p(t), _p(np.ascontiguousarray(out["rgb"])),
                              _p(out["means"]), _p(out["sh_rest"]))
    return out


PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "rgb", "sh_rest")


def project_backward_magnitude(g, cam, g2, near=0.2):
    """Magnitudes of `project_backward`'s results: the same adjoint evaluated
    in magnitude arithmetic (mag.h: |operands|, subtractions as additions)
    from |g2|.  An FP32 adjoint's rounding error is a small multiple of u
    times these, per element (running error analysis)."""
    M = g.M
    arrs = [_f64(a) for a in g.arrays()]
    K, R, t = _cam(cam)
    out = dict(means=np.zeros((M, 3)), log_scales=np.zeros((M, 3)), quats=np.zeros((M, 4)),
               opacity_logits=np.zeros(M), rgb=np.zeros((M, 3)))
    lib().orc_project_backward_mag(ctypes.c_int(M), *[_p(a) for a in arrs[:4]],
                                   ctypes.c_int(cam.width), ctypes.c_int(cam.height), _p(K),
                                   _p(R), _p(t), ctypes.c_double(near), _p(_f64(g2)),
                                   _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]),
                                   _p(out["opacity_logits"]), _p(out["rgb"]))
    D = _sh_degree(g)
    if D > 0:
        out["sh_rest"] = np.zeros(g.sh_rest.shape)
        lib().orc_sh_backward_mag(ctypes.c_int(M), ctypes.c_int(D), _p(arrs[0]),
                                  _p(_f64(g.sh_rest)), _p(t), _p(np.ascontiguousarray(out["rgb"])),
                                  _p(out["means"]), _p(out["sh_rest"]))
    return out


def projection_adjoint_matrix(g, cam, near=0.2) -> np.ndarray:
    """J^T of every Gaussian's projection, [M][P][G_N]: the parameter gradient
    of a per-Gaussian 2D gradient g2 [M][G_N] is JT[i] @ g2[i], parameters in
    PARAM_KEYS order flattened (P = 14, plus 3 K SH coefficients).  Built
    column by column from `project_backward` (linear in g2)."""
    M = g.M
    cols = []
    for c in range(G_N):
        e = np.zeros((M, G_N))
        e[:, c] = 1.0
        gr = project_backward(g, cam, e, near)
        cols.append(np.concatenate([gr[k].reshape(M, -1) for k in PARAM_KEYS if k in gr], axis=1))
    return np.ascontiguousarray(np.stack(cols, axis=2))


def split_params(v: np.ndarray, like: dict) -> dict:
    """[M][P] per-parameter array -> dict shaped like a project_backward result."""
    out, o = {}, 0
    for k in PARAM_KEYS:
        if k not in like:
            continue
        n = int(np.prod(like[k].shape[1:])) if like[k].ndim > 1 else 1
        out[k] = v[:, o:o + n].reshape(like[k].shape)
        o += n
    return out


U32 = 2.0 ** -24  # unit roundoff of binary32


def bands_for(W: int, H: int, **over) -> dict:
    """Error bands of a single-precision (FP32) evaluation of a W x H view, the
    `bands` of `envelope` and `flip_spec`:
      conic 2.5e-6: the conic entries within 2e-6 of cn = |a| + 2|b| + |c|,
        plus the rounding of q's own products (8 u cn r^2);
      mean 4 u (W + H) px: m = f t_x / t_z + c carries a few roundings of
        numbers below W + H;
      qmax 2e-7 and depth 3.5e-7 (relative): a few roundings each, the depth
        threshold D_t + eps rounded once more (2 u);
      res_colour 1e-4 and res_depth 1e-4 (relative): the image tolerance;
      order 2.3e-7 (relative): the front-to-back blend's order of two
        Gaussians whose depths, each within 2.3e-7 of itself, lie within
        order (|d_a| + |d_b|) of each other can go either way.
    The record bounds these assume are asserted on the kernels' records by the
    end-to-end tests."""
    b = dict(conic=2.5e-6, mean=4.0 * U32 * (W + H), qmax=2e-7, depth=3.5e-7,
             res_colour=1e-4, res_depth=1e-4, order=2.3e-7)
    b.update(over)
    return b


def envelope(rec, Ct, Dt, eps, mode, Ctgt, Dtgt, lambda_depth, n_valid, JT=None, bands=None,
             kmax=12, f32=False, dC=None, dD=None):
    """Decision envelope of one view (orc_envelope in splat.cpp): how far a
    single-precision evaluation that takes every decision outside the error
    bands as the FP64 definition does can be from it, per pixel, for the loss
    and per parameter.  Bands (dict, default `bands_for(W, H)`): the counting decision
    q <= qmax is ambiguous where |qmax - q| < conic cn r^2 + 2 mean cn r +
    qmax |qmax| (cn = |a| + 2|b| + |c|, r the pixel's distance from the mean:
    a conic known within `conic` of cn, a mean within `mean` px, qmax within
    `qmax` of itself), the depth test where |d - (D_t + eps)| < depth
    (D_t + eps); residual signs where |C* - C| < res_colour or
    |D* - D| < res_depth D; in the front-to-back (ALPHA) blend the order of
    two touched Gaussians where |d_a - d_b| < order (|d_a| + |d_b|) (both
    orders evaluated).  JT = None: the image and loss envelope only.
    f32=True: FP32 decisions on records holding FP32 values (as `composite`
    with f32), nothing ambiguous - for the reference terms' sums s2, s2q.
    dC, dD: explicit upstream gradients in place of the L1 loss's.
    Returns allow_C, allow_D, allow_W [H][W] (C*, D*, W_G; inf where
    unbounded), allow_L, n_amb,
    unbounded [H][W], allow3 [M][P] (per parameter, PARAM_KEYS order), g2ref
    [M][G_N] (the FP64 2D gradient), s2, s2q [M][G_N] (sums over pixels of
    |term| and |term| qband / 2)."""
    rec = _f64(rec)
    Ct, Dt, Ctgt, Dtgt = (_f64(a) for a in (Ct, Dt, Ctgt, Dtgt))
    H, W = Dt.shape
    b = bands if bands is not None else bands_for(W, H)
    M = rec.shape[0]
    if JT is None:
        JT = np.zeros((M, 0, G_N))
    JT = np.ascontiguousarray(JT, dtype=np.float64)
    P = JT.shape[1]
    assert JT.shape == (M, P, G_N)
    band = _f64([b["conic"], b["mean"], b["qmax"], b["depth"], b["res_colour"], b["res_depth"],
                 b.get("order", 0.0)])
    allow_img = np.zeros((3, H, W))
    allow_L = ctypes.c_double(0.0)
    n_amb = np.zeros((H, W), np.int32)
    unb = np.zeros((H, W), np.int32)
    allow3 = np.zeros((M, max(P, 1)))
    g2ref, s2, s2q = np.zeros((M, G_N)), np.zeros((M, G_N)), np.zeros((M, G_N))
    lib().orc_envelope(ctypes.c_int(M), _p(rec), ctypes.c_int(W), ctypes.c_int(H), _p(Ct),
                       _p(Dt), ctypes.c_double(eps), ctypes.c_int(mode), _p(Ctgt), _p(Dtgt),
                       ctypes.c_double(lambda_depth), ctypes.c_long(n_valid), _p(band),
                       ctypes.c_int(P), _p(JT), ctypes.c_int(kmax), ctypes.c_int(int(f32)),
                       _p(_f64(dC)) if dC is not None else None,
                       _p(_f64(dD)) if dD is not None else None, _p(allow_img),
                       ctypes.byref(allow_L), _p(n_amb), _p(unb), _p(allow3), _p(g2ref), _p(s2),
                       _p(s2q))
    return dict(allow_C=allow_img[0], allow_D=allow_img[1], allow_W=allow_img[2],
                allow_L=allow_L.value, n_amb=n_amb,
                unbounded=unb, allow3=allow3, g2ref=g2ref, s2=s2, s2q=s2q)


def bin_records(rec32: np.ndarray, W: int, H: int, TW: int, TH: int, cap: int = 1 << 26):
    """Tile binning of FP32 records [M][16] -> (keys u64 [P], vals u32 [P],
    ranges u32 [tiles][2])."""
    rec32 = np.ascontiguousarray(rec32, dtype=np.float32)
    M = rec32.shape[0]
    ntiles = ((W + TW - 1) // TW) * ((H + TH - 1) // TH)
    cap = int(min(cap, max(1, _count_pairs(rec32, W, H, TW, TH))))
    keys = np.zeros(cap, np.uint64)
    vals = np.zeros(cap, np.uint32)
    ranges = np.zeros((ntiles, 2), np.uint32)
    P = lib().orc_bin(ctypes.c_int(M), _p(rec32), ctypes.c_int(W), ctypes.c_int(H),
                      ctypes.c_int(TW), ctypes.c_int(TH), ctypes.c_long(cap), _p(keys), _p(vals),
                      _p(ranges))
    if P < 0:
        raise RuntimeError("pair capacity exceeded")
    return keys[:P].copy(), vals[:P].copy(), ranges


def _count_pairs(rec32, W, H, TW, TH) -> int:
    """Upper bound on the number of (tile, Gaussian) pairs (buffer sizing only)."""
    ex, ey = rec32[:, 11].astype(np.float64), rec32[:, 12].astype(np.float64)
    ok = (ex >= 0) & (ey >= 0)
    mx, my = rec32[:, 0].astype(np.float64), rec32[:, 1].astype(np.float64)
    x0 = np.clip(np.floor(mx - ex), 0, W - 1)
    x1 = np.clip(np.ceil(mx + ex), 0, W - 1)
    y0 = np.clip(np.floor(my - ey), 0, H - 1)
    y1 = np.clip(np.ceil(my + ey), 0, H - 1)
    n = (x1 // TW - x0 // TW + 1) * (y1 // TH - y0 // TH + 1)
    return int(np.where(ok & np.isfinite(n), n, 0).sum())


def adam(p, g, m, v, lr, b1=0.9, b2=0.999, eps=1e-15, step=1) -> None:
    """In-place FP64 Adam step on flat contiguous float64 arrays."""
    n = p.size
    lib().orc_adam(ctypes.c_long(n), _p(p), _p(g), _p(m), _p(v), ctypes.c_double(lr),
                   ctypes.c_double(b1), ctypes.c_double(b2), ctypes.c_double(eps),
                   ctypes.c_int(step))


# --------------------------------------------------------------------------
# conversions and whole-view helpers
# --------------------------------------------------------------------------
EXT_REL = np.float32(1.0 + 2.0 ** -7)
EXT_ABS = np.float32(2.0 ** -4)


def records_f32(rec: np.ndarray) -> np.ndarray:
    """FP32 records in the kernels' 16-float layout from FP64 oracle records:
    (mx, my, d, sigma, a, b, c, qmax, r, g, b, ext_x, ext_y, 0, 0, 0) rounded to
    float, with the conservative extent ext = sqrt(qmax * S2xx) * (1 + 2^-7) + 2^-4
    evaluated in float, and ext = -1 for invisible Gaussians."""
    M = rec.shape[0]
    out = np.zeros((M, 16), np.float32)
    for k_out, k_in in enumerate((R_MX, R_MY, R_D, R_SIG, R_CA, R_CB, R_CC, R_QMAX, R_R, R_G,
                                  R_B)):
        out[:, k_out] = rec[:, k_in].astype(np.float32)
    q = out[:, 7]
    with np.errstate(invalid="ignore"):
        ex = np.sqrt(q * rec[:, R_S2XX].astype(np.float32)) * EXT_REL + EXT_ABS
        ey = np.sqrt(q * rec[:, R_S2YY].astype(np.float32)) * EXT_REL + EXT_ABS
    vis = rec[:, R_VIS] != 0
    out[:, 11] = np.where(vis, ex, np.float32(-1))
    out[:, 12] = np.where(vis, ey, np.float32(-1))
    return out


def rounded(rec: np.ndarray) -> np.ndarray:
    """FP64 record array holding the FP32-rounded values (for f32 decisions)."""
    r = rec.astype(np.float32).astype(np.float64)
    r[:, R_VIS] = rec[:, R_VIS]
    return r


def render_loss_grads(g, cam, Ct, Dt, Ctgt, Dtgt, eps=0.01, lambda_depth=0.0, mode=OIT,
                      f32=False, near=0.2, flip=None):
    """One view end to end: project -> composite -> loss -> adjoints.
    f32=True takes the counting decisions in FP32 on FP32-rounded records;
    flip (diagnostic) inverts the decisions inside that error band."""
    rec, pamb = project(g, cam, near)
    rr = rounded(rec) if f32 else rec
    out = composite(rr, Ct, Dt, eps, mode, f32, flip=flip)
    L, dC, dD, nv, lamb = loss(out["C"], out["D"], Ctgt, Dtgt, Dt, lambda_depth)
    g2 = composite_backward(rr, Ct, Dt, eps, dC, dD, mode, f32, flip=flip)
    grads = project_backward(g, cam, g2, near)
    return dict(L=L, rec=rec, proj_amb=pamb, out=out, dC=dC, dD=dD, n_valid=nv, loss_amb=lamb,
                g2=g2, grads=grads)


def quantise(x, precision: int) -> np.ndarray:
    """Colour values as stored in the given type, returned as float64: binary32
    rounding first (the images are float), then IEEE binary16 (numpy's cast
    rounds to nearest, ties to even) or bfloat16 (the upper half of the
    binary32 pattern after rounding the lower 16 bits to nearest, ties to
    even: add 0x7FFF plus the lowest kept bit, then truncate)."""
    a = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    if precision == FP32:
        return a.astype(np.float64)
    if precision == FP16:
        return a.astype(np.float16).astype(np.float64)
    if precision == BF16:
        bits = a.view(np.uint32).astype(np.uint64)
        keep = (bits >> np.uint64(16)) & np.uint64(1)
        r = ((bits + np.uint64(0x7FFF) + keep) >> np.uint64(16)) << np.uint64(16)
        return r.astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(f"unknown precision {precision}")
