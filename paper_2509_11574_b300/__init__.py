"""Python binding of libgps.so (the Gaussian-plus-SDF hot path on sm_103a).

Argument marshalling only: every step runs in the CUDA kernels behind the C ABI
declared in include/gps.h.  PyTorch supplies device memory and streams.  There
is no CPU fallback: importing works anywhere, but every call needs the built
library and a CUDA device and raises otherwise.

Layers:
  * ctypes mirrors of the C structs and `lib()` (the loaded library);
  * thin wrappers with the C names (`fuse_frame`, `raycast_sdf`,
    `render_forward`, `render_backward`, `adam_step`, `gps_workspace_size`, ...);
  * convenience holders: `Tsdf`, `Gaussians`, `Renderer`, `Adam`, and the
    autograd functions `RenderImages` / `RenderLoss`.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import List, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgps.so")

GPS_OK = 0
GPS_ERR_INVALID_ARG = -1
GPS_ERR_WORKSPACE_TOO_SMALL = -2
GPS_ERR_CAPACITY = -3
GPS_ERR_CUDA = -4
GPS_ERR_TIMEOUT = -5
BLEND_OIT, BLEND_ALPHA = 0, 1
PREC_FP32, PREC_FP16, PREC_BF16 = 0, 1, 2
SCHEDULE_TILES, SCHEDULE_PER_GAUSSIAN = 0, 1
PREC_DTYPE = {PREC_FP32: torch.float32, PREC_FP16: torch.float16, PREC_BF16: torch.bfloat16}
STAGE_PROJECT, STAGE_BIN, STAGE_COMPOSITE, STAGE_COMPOSITE_BWD, STAGE_PROJECT_BWD = 1, 2, 4, 8, 16

# learning rates of App. C; the RGB colour plays the role of the degree-0 SH
# coefficient, whose value is scaled by the SH basis constant 0.28209479
LR_APP_C = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3 * 0.28209479177387814)
LR_SH_REST = 5e-4  # App. C: SH coefficients of degree >= 1
SH_DEGREE_OF = {3: 1, 8: 2, 15: 3}  # coefficients per colour channel -> degree

c_float, c_int32, c_int64, c_size_t, c_void_p = (ctypes.c_float, ctypes.c_int32, ctypes.c_int64,
                                                 ctypes.c_size_t, ctypes.c_void_p)
P_float = ctypes.POINTER(ctypes.c_float)


class GpsIntrinsics(ctypes.Structure):
    _fields_ = [("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("width", c_int32), ("height", c_int32)]


class GpsPose(ctypes.Structure):
    _fields_ = [("R", c_float * 9), ("t", c_float * 3)]


class GpsTsdf(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32), ("voxel", c_float),
                ("origin", c_float * 3), ("trunc", c_float), ("max_weight", c_float),
                ("sdf", c_void_p), ("weight", c_void_p), ("rgbw", c_void_p),
                ("brick_flags", c_void_p)]


class GpsHashTsdf(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32), ("voxel", c_float),
                ("origin", c_float * 3), ("trunc", c_float), ("max_weight", c_float),
                ("n_buckets", c_int32), ("capacity", c_int32), ("keys", c_void_p),
                ("slots", c_void_p), ("brick_of_slot", c_void_p), ("state", c_void_p),
                ("sdf", c_void_p), ("weight", c_void_p), ("rgbw", c_void_p),
                ("slot_flags", c_void_p)]


class GpsGaussians(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p),
                ("opacity_logits", c_void_p), ("rgb", c_void_p), ("M", c_int32),
                ("sh_degree", c_int32), ("sh_rest", c_void_p)]


class GpsView(ctypes.Structure):
    _fields_ = [("K", GpsIntrinsics), ("T_wc", GpsPose), ("sdf_rgb", c_void_p),
                ("sdf_depth", c_void_p), ("target_rgb", c_void_p), ("target_depth", c_void_p),
                ("out_rgb", c_void_p), ("out_depth", c_void_p), ("out_weight", c_void_p),
                ("grad_rgb", c_void_p), ("grad_depth", c_void_p)]


class GpsRenderSettings(ctypes.Structure):
    _fields_ = [("eps_depth", c_float), ("lambda_depth", c_float), ("near_plane", c_float),
                ("blend_mode", c_int32), ("precision", c_int32), ("tile_w", c_int32),
                ("tile_h", c_int32), ("deterministic", c_int32), ("stages", c_int32),
                ("instrument", c_int32), ("schedule", c_int32), ("pair_capacity", c_int64)]


class GpsEditSettings(ctypes.Structure):
    _fields_ = [("delta_c", c_float), ("delta_w", c_float), ("sample_fraction", c_float),
                ("radius", c_int32), ("seed", ctypes.c_uint64), ("delta_sigma", c_float),
                ("delta_smax", c_float), ("delta_smin", c_float), ("precision", c_int32)]


def edit_settings(delta_c=0.05, delta_w=4.0, sample_fraction=0.25, radius=3, seed=0,
                  delta_sigma=0.005, delta_smax=0.1, delta_smin=0.003,
                  precision=0) -> "GpsEditSettings":
    """Sec. 3.2 thresholds (the defaults are the paper's)."""
    return GpsEditSettings(delta_c, delta_w, sample_fraction, radius, seed, delta_sigma, delta_smax,
                           delta_smin, precision)


class GpsViewSchedule(ctypes.Structure):
    _fields_ = [("delta_angle_deg", c_float), ("delta_move", c_float), ("interval", c_int32),
                ("n_global", c_int32), ("n_local", c_int32), ("reserved", c_int32),
                ("seed", ctypes.c_uint64)]


def view_schedule(delta_angle_deg=30.0, delta_move=0.3, interval=10, n_global=4, n_local=4,
                  seed=0) -> "GpsViewSchedule":
    """Keyframe thresholds of App. C (30 degrees, 0.3 m) and the optimisation
    interval of Sec. 4.1 (every 10 frames); four global and four local views."""
    return GpsViewSchedule(delta_angle_deg, delta_move, interval, n_global, n_local, 0, seed)


class GpsIcpSettings(ctypes.Structure):
    _fields_ = [("levels", c_int32), ("iters", c_int32 * 4), ("eps_d", c_float),
                ("eps_theta_deg", c_float)]


def icp_settings(levels=3, iters=(10, 5, 4), eps_d=0.1, eps_theta_deg=20.0) -> GpsIcpSettings:
    """Point-to-plane ICP over a `levels`-level pyramid; iters finest first
    (KinectFusion's 10, 5, 4 and its 0.1 m / 20 degree rejection)."""
    it = list(iters) + [0] * (4 - len(iters))
    return GpsIcpSettings(levels, (c_int32 * 4)(*it), eps_d, eps_theta_deg)


class GpsAdamHyper(ctypes.Structure):
    _fields_ = [("lr", c_float * 5), ("beta1", c_float), ("beta2", c_float), ("eps", c_float),
                ("lr_sh_rest", c_float)]


class GpsWorkspaceLayout(ctypes.Structure):
    _fields_ = [("total_bytes", c_size_t), ("status", c_size_t), ("records", c_size_t),
                ("super_counts", c_size_t), ("block_base", c_size_t), ("super_ranges", c_size_t),
                ("super_keys", c_size_t), ("super_scratch", c_size_t),
                ("tile_ranges", c_size_t),
                ("pair_keys", c_size_t), ("pix_state", c_size_t), ("tile_partials", c_size_t),
                ("view_scalars", c_size_t), ("grad2d", c_size_t), ("pair_grads", c_size_t),
                ("pix_grad", c_size_t),
                ("tiles_x", c_int32), ("tiles_y", c_int32), ("tile_w", c_int32),
                ("tile_h", c_int32), ("super_x", c_int32), ("super_y", c_int32),
                ("super_px", c_int32), ("tile_bins", c_int32), ("pair_capacity", c_int64),
                ("pair_base", c_size_t), ("tile_order", c_size_t), ("grad_fixed", c_size_t)]


EXPORTED = ("gps_last_error", "gps_version", "gps_workspace_size", "gps_workspace_layout",
            "gps_query_status", "fuse_frame", "raycast_sdf", "render_forward", "render_backward",
            "adam_step", "render_forward_noalloc", "gps_noalloc_query_status",
            "gps_autotune_tiles",
            "gps_edit_scratch_size", "insert_gaussians", "remove_gaussians",
            "tsdf_mark_bricks", "gps_is_keyframe", "gps_select_views",
            "gps_icp_workspace_size", "icp_track", "gps_hash_scratch_size", "fuse_frame_hashed",
            "raycast_sdf_hashed", "tsdf_hash_to_dense", "render_backward_adam")
AUTOTUNE_SHAPES = ((16, 16), (16, 8), (8, 8), (32, 8))  # the order of GPS_AUTOTUNE_SHAPES
NOALLOC_SCRATCH_BYTES = 64 << 20

_lib: Optional[ctypes.CDLL] = None


class GpsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libgps error {code}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded libgps.so.  Raises if the library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2509_11574_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        L.gps_last_error.restype = ctypes.c_char_p
        L.gps_version.restype = ctypes.c_char_p
        for n in EXPORTED[2:]:
            getattr(L, n).restype = c_int32
        L.gps_workspace_size.argtypes = [c_int32, ctypes.POINTER(GpsView), c_int32,
                                         ctypes.POINTER(GpsRenderSettings), ctypes.POINTER(c_size_t)]
        L.gps_workspace_layout.argtypes = [c_int32, ctypes.POINTER(GpsView), c_int32,
                                           ctypes.POINTER(GpsRenderSettings), c_int32,
                                           ctypes.POINTER(GpsWorkspaceLayout)]
        L.gps_query_status.argtypes = [c_void_p, c_size_t, ctypes.POINTER(c_int32), c_void_p]
        L.fuse_frame.argtypes = [ctypes.POINTER(GpsTsdf), c_void_p, c_void_p,
                                 ctypes.POINTER(GpsIntrinsics), ctypes.POINTER(GpsPose), c_void_p]
        L.raycast_sdf.argtypes = [ctypes.POINTER(GpsTsdf), ctypes.POINTER(GpsIntrinsics),
                                  ctypes.POINTER(GpsPose), c_float, c_float, c_void_p, c_int32,
                                  c_void_p, c_void_p, c_void_p]
        L.render_forward.argtypes = [ctypes.POINTER(GpsGaussians), ctypes.POINTER(GpsView), c_int32,
                                     ctypes.POINTER(GpsRenderSettings), c_void_p, c_size_t,
                                     c_void_p, c_void_p]
        L.render_backward.argtypes = [ctypes.POINTER(GpsGaussians), ctypes.POINTER(GpsView),
                                      c_int32, ctypes.POINTER(GpsRenderSettings), c_void_p,
                                      c_size_t, c_void_p, ctypes.POINTER(GpsGaussians), c_void_p]
        L.render_backward_adam.argtypes = [
            ctypes.POINTER(GpsGaussians), ctypes.POINTER(GpsView), c_int32,
            ctypes.POINTER(GpsRenderSettings), c_void_p, c_size_t, c_void_p,
            ctypes.POINTER(GpsGaussians), ctypes.POINTER(GpsGaussians),
            ctypes.POINTER(GpsAdamHyper), c_int32, c_void_p, c_void_p]
        L.gps_autotune_tiles.argtypes = [ctypes.POINTER(GpsGaussians), ctypes.POINTER(GpsView),
                                         c_int32, ctypes.POINTER(GpsRenderSettings), c_void_p,
                                         c_size_t, ctypes.POINTER(GpsGaussians), c_int32,
                                         ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                         ctypes.POINTER(c_float), c_void_p]
        P_G = ctypes.POINTER(GpsGaussians)
        L.tsdf_mark_bricks.argtypes = [ctypes.POINTER(GpsTsdf), c_void_p]
        L.gps_edit_scratch_size.argtypes = [c_int32, c_int32, c_int32, ctypes.POINTER(c_size_t)]
        L.insert_gaussians.argtypes = [P_G, c_int32, P_G, P_G, P_G, ctypes.POINTER(GpsIntrinsics),
                                       ctypes.POINTER(GpsPose), c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, ctypes.POINTER(GpsEditSettings),
                                       c_void_p, c_size_t, c_void_p, c_void_p]
        L.remove_gaussians.argtypes = [P_G, P_G, P_G, P_G, ctypes.POINTER(GpsEditSettings),
                                       c_void_p, c_size_t, c_void_p, c_void_p]
        L.adam_step.argtypes = [ctypes.POINTER(GpsGaussians), ctypes.POINTER(GpsGaussians),
                                ctypes.POINTER(GpsGaussians), ctypes.POINTER(GpsGaussians),
                                ctypes.POINTER(GpsAdamHyper), c_int32, c_void_p, c_void_p]
        L.render_forward_noalloc.argtypes = [ctypes.POINTER(GpsGaussians),
                                             ctypes.POINTER(GpsView), c_int32,
                                             ctypes.POINTER(GpsRenderSettings), c_void_p,
                                             c_void_p]
        L.gps_noalloc_query_status.argtypes = [ctypes.POINTER(c_int32), c_void_p]
        L.gps_is_keyframe.argtypes = [ctypes.POINTER(GpsPose), ctypes.POINTER(GpsPose),
                                      ctypes.POINTER(GpsViewSchedule), ctypes.POINTER(c_int32)]
        L.gps_select_views.argtypes = [ctypes.POINTER(c_int32), c_int32, c_int32, c_int32,
                                       ctypes.POINTER(GpsViewSchedule), ctypes.POINTER(c_int32),
                                       c_int32, ctypes.POINTER(c_int32)]
        L.gps_icp_workspace_size.argtypes = [c_int32, c_int32, ctypes.POINTER(GpsIcpSettings),
                                             ctypes.POINTER(c_size_t)]
        L.icp_track.argtypes = [ctypes.POINTER(GpsIntrinsics), c_void_p, c_void_p, c_void_p,
                                ctypes.POINTER(GpsPose), ctypes.POINTER(GpsIcpSettings), c_void_p,
                                c_void_p, c_size_t, c_void_p, c_void_p]
        P_H = ctypes.POINTER(GpsHashTsdf)
        L.gps_hash_scratch_size.argtypes = [c_int32, ctypes.POINTER(c_size_t)]
        L.fuse_frame_hashed.argtypes = [P_H, c_void_p, c_void_p, ctypes.POINTER(GpsIntrinsics),
                                        ctypes.POINTER(GpsPose), c_void_p, c_size_t, c_int32,
                                        c_void_p]
        L.raycast_sdf_hashed.argtypes = [P_H, ctypes.POINTER(GpsIntrinsics),
                                         ctypes.POINTER(GpsPose), c_float, c_float, c_void_p,
                                         c_int32, c_void_p, c_void_p, c_void_p]
        L.tsdf_hash_to_dense.argtypes = [P_H, ctypes.POINTER(GpsTsdf), c_void_p]
        _lib = L
    return _lib


def _check(code: int) -> None:
    if code != GPS_OK:
        raise GpsError(code, lib().gps_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libgps takes CUDA tensors only")
    if not t.is_contiguous():
        raise ValueError("libgps takes contiguous tensors only")
    return c_void_p(t.data_ptr())


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- structs
def intrinsics(cam) -> GpsIntrinsics:
    return GpsIntrinsics(float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy),
                         int(cam.width), int(cam.height))


def pose(cam) -> GpsPose:
    R = [float(x) for x in torch.as_tensor(cam.R, dtype=torch.float64).reshape(9)]
    t = [float(x) for x in torch.as_tensor(cam.t, dtype=torch.float64).reshape(3)]
    return GpsPose((c_float * 9)(*R), (c_float * 3)(*t))


@dataclasses.dataclass
class Gaussians:
    """Gaussian parameters (or same-shaped gradients / moments) on the device;
    sh_rest [M][K][3] (K = 3, 8 or 15) adds view-dependent colour of degree
    1, 2 or 3."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    rgb: torch.Tensor
    sh_rest: Optional[torch.Tensor] = None

    @property
    def M(self) -> int:
        return int(self.means.shape[0])

    @property
    def sh_degree(self) -> int:
        return 0 if self.sh_rest is None else SH_DEGREE_OF[int(self.sh_rest.shape[1])]

    def tensors(self) -> List[torch.Tensor]:
        t = [self.means, self.log_scales, self.quats, self.opacity_logits, self.rgb]
        return t + ([self.sh_rest] if self.sh_rest is not None else [])

    def c(self) -> GpsGaussians:
        return GpsGaussians(*[_ptr(t) for t in self.tensors()[:5]], self.M, self.sh_degree,
                            _ptr(self.sh_rest))

    @staticmethod
    def from_numpy(gs, device="cuda") -> "Gaussians":
        arrs = list(gs.arrays())
        if getattr(gs, "sh_rest", None) is not None:
            arrs.append(gs.sh_rest)
        return Gaussians(*[torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
                           for a in arrs])

    def zeros_like(self) -> "Gaussians":
        return Gaussians(*[torch.zeros_like(t) for t in self.tensors()])

    def flat(self) -> torch.Tensor:
        return torch.cat([t.reshape(-1) for t in self.tensors()])


def brick_to_linear(a: torch.Tensor, nx: int, ny: int, nz: int) -> torch.Tensor:
    """Reorder a brick-major voxel array (see GpsTsdf) to [nz][ny][nx](...) (x fastest)."""
    tail = a.shape[1:]
    b = a.reshape(nz // 8, ny // 8, nx // 8, 8, 8, 8, *tail)
    perm = (0, 3, 1, 4, 2, 5) + tuple(range(6, 6 + len(tail)))
    return b.permute(*perm).reshape(nz, ny, nx, *tail)


def linear_to_brick(a: torch.Tensor) -> torch.Tensor:
    """Inverse of brick_to_linear: [nz][ny][nx](...) -> brick-major [n](...)."""
    nz, ny, nx = a.shape[:3]
    tail = a.shape[3:]
    b = a.reshape(nz // 8, 8, ny // 8, 8, nx // 8, 8, *tail)
    perm = (0, 2, 4, 1, 3, 5) + tuple(range(6, 6 + len(tail)))
    return b.permute(*perm).reshape(nz * ny * nx, *tail).contiguous()


class Tsdf:
    """Dense colourised TSDF on the device (brick-major, see include/gps.h)."""

    def __init__(self, spec, device="cuda"):
        self.spec = spec
        n = spec.nx * spec.ny * spec.nz
        self.sdf = torch.ones(n, dtype=torch.float32, device=device)
        self.weight = torch.zeros(n, dtype=torch.float32, device=device)
        self.rgbw = torch.zeros(n, 4, dtype=torch.float32, device=device)
        self.brick_flags = torch.zeros(n // 512, dtype=torch.uint8, device=device)

    def reset(self):
        self.sdf.fill_(1.0)
        self.weight.zero_()
        self.rgbw.zero_()
        self.brick_flags.zero_()

    def mark_bricks(self, stream=None):
        """Recompute the brick flags after writing sdf directly."""
        t = self.c()
        _check(lib().tsdf_mark_bricks(ctypes.byref(t), _stream(stream)))

    def c(self) -> GpsTsdf:
        s = self.spec
        return GpsTsdf(s.nx, s.ny, s.nz, float(s.voxel), (c_float * 3)(*map(float, s.origin)),
                       float(s.trunc), float(s.max_weight), _ptr(self.sdf), _ptr(self.weight),
                       _ptr(self.rgbw), _ptr(self.brick_flags))

    def linear(self):
        s = self.spec
        return (brick_to_linear(self.sdf, s.nx, s.ny, s.nz),
                brick_to_linear(self.weight, s.nx, s.ny, s.nz),
                brick_to_linear(self.rgbw, s.nx, s.ny, s.nz))


class HashTsdf:
    """Voxel-hashed TSDF on the device (see GpsHashTsdf): a pool of `capacity`
    8^3 bricks, a table of n_buckets buckets (default: the power of two at
    least 4 x capacity), the same index space and fusion parameters as the
    dense `spec`, and the per-frame candidate scratch."""

    def __init__(self, spec, capacity: int, n_buckets: Optional[int] = None,
                 max_candidates: int = 1 << 17, device="cuda"):
        self.spec = spec
        self.capacity = capacity
        nb = 2
        while nb < (n_buckets or 4 * capacity):
            nb <<= 1
        self.n_buckets = nb
        self.max_candidates = max_candidates
        dev = torch.device(device)
        self.keys = torch.zeros(nb, dtype=torch.int64, device=dev)
        self.slots = torch.zeros(nb, dtype=torch.int32, device=dev)
        self.brick_of_slot = torch.zeros(capacity, dtype=torch.int64, device=dev)
        self.state = torch.zeros(4, dtype=torch.int32, device=dev)
        self.sdf = torch.ones(capacity * 512, device=dev)
        self.weight = torch.zeros(capacity * 512, device=dev)
        self.rgbw = torch.zeros(capacity * 512, 4, device=dev)
        self.slot_flags = torch.zeros(capacity, dtype=torch.uint8, device=dev)
        self.scratch = torch.zeros(gps_hash_scratch_size(max_candidates), dtype=torch.uint8,
                                   device=dev)

    def reset(self):
        self.keys.zero_()
        self.state.zero_()

    def c(self) -> GpsHashTsdf:
        s = self.spec
        return GpsHashTsdf(s.nx, s.ny, s.nz, float(s.voxel), (c_float * 3)(*map(float, s.origin)),
                           float(s.trunc), float(s.max_weight), self.n_buckets, self.capacity,
                           _ptr(self.keys), _ptr(self.slots), _ptr(self.brick_of_slot),
                           _ptr(self.state), _ptr(self.sdf), _ptr(self.weight), _ptr(self.rgbw),
                           _ptr(self.slot_flags))

    def allocated(self) -> int:
        """Bricks in use (reads the device counter: synchronises)."""
        return min(int(self.state[0].item()), self.capacity)

    def error(self) -> int:
        return int(self.state[1].item())

    def bricks(self) -> torch.Tensor:
        """Brick indices of the allocated bricks, in pool order."""
        return self.brick_of_slot[:self.allocated()]

    def to_dense(self, dense: "Tsdf", stream=None) -> None:
        h, d = self.c(), dense.c()
        _check(lib().tsdf_hash_to_dense(ctypes.byref(h), ctypes.byref(d), _stream(stream)))


def gps_hash_scratch_size(max_candidates: int) -> int:
    n = c_size_t(0)
    _check(lib().gps_hash_scratch_size(max_candidates, ctypes.byref(n)))
    return int(n.value)


def fuse_frame_hashed(vol: HashTsdf, depth: torch.Tensor, rgb: torch.Tensor, cam,
                      stream=None) -> None:
    K, P = intrinsics(cam), pose(cam)
    h = vol.c()
    _check(lib().fuse_frame_hashed(ctypes.byref(h), _ptr(depth), _ptr(rgb), ctypes.byref(K),
                                   ctypes.byref(P), _ptr(vol.scratch), vol.scratch.numel(),
                                   vol.max_candidates, _stream(stream)))


def raycast_sdf_hashed(vol: HashTsdf, cam, near=0.2, far=0.0, out_rgb=None, out_depth=None,
                       out_vertex=None, stream=None, precision=PREC_FP32):
    """raycast_sdf on a hashed volume."""
    H, W = cam.height, cam.width
    dev = vol.sdf.device
    if out_rgb is None:
        out_rgb = torch.empty(3, H, W, device=dev, dtype=PREC_DTYPE[precision])
    prec = _precision_of(out_rgb)
    out_depth = out_depth if out_depth is not None else torch.empty(H, W, device=dev)
    K, P = intrinsics(cam), pose(cam)
    h = vol.c()
    _check(lib().raycast_sdf_hashed(ctypes.byref(h), ctypes.byref(K), ctypes.byref(P), near, far,
                                    _ptr(out_rgb), prec, _ptr(out_depth), _ptr(out_vertex),
                                    _stream(stream)))
    return out_rgb, out_depth


def settings(eps_depth=0.01, lambda_depth=0.0, near=0.2, blend_mode=BLEND_OIT,
             precision=PREC_FP32, tile=(16, 16), deterministic=False, stages=0,
             pair_capacity=0, instrument=False, schedule=0) -> GpsRenderSettings:
    return GpsRenderSettings(eps_depth, lambda_depth, near, blend_mode, precision, tile[0], tile[1],
                             int(deterministic), stages, int(instrument), schedule, pair_capacity)


@dataclasses.dataclass
class View:
    """One view of the second rendering pass (device images)."""
    cam: object
    sdf_rgb: torch.Tensor
    sdf_depth: torch.Tensor
    target_rgb: Optional[torch.Tensor] = None
    target_depth: Optional[torch.Tensor] = None
    out_rgb: Optional[torch.Tensor] = None
    out_depth: Optional[torch.Tensor] = None
    out_weight: Optional[torch.Tensor] = None
    grad_rgb: Optional[torch.Tensor] = None
    grad_depth: Optional[torch.Tensor] = None

    def c(self) -> GpsView:
        return GpsView(intrinsics(self.cam), pose(self.cam), _ptr(self.sdf_rgb),
                       _ptr(self.sdf_depth), _ptr(self.target_rgb), _ptr(self.target_depth),
                       _ptr(self.out_rgb), _ptr(self.out_depth), _ptr(self.out_weight),
                       _ptr(self.grad_rgb), _ptr(self.grad_depth))


def _views(views: Sequence[View], s: Optional[GpsRenderSettings] = None):
    if s is not None:
        want = PREC_DTYPE[s.precision]
        for k, v in enumerate(views):
            for name in ("sdf_rgb", "target_rgb", "out_rgb"):
                t = getattr(v, name)
                if t is not None and t.dtype != want:
                    raise ValueError(f"view {k}: {name} is {t.dtype}, settings.precision "
                                     f"stores colour as {want}")
    arr = (GpsView * len(views))(*[v.c() for v in views])
    return arr


def _precision_of(t: torch.Tensor) -> int:
    for p, dt in PREC_DTYPE.items():
        if t.dtype == dt:
            return p
    raise ValueError(f"colour images are float32, float16 or bfloat16, not {t.dtype}")


def _size_views(cams) -> ctypes.Array:
    return (GpsView * len(cams))(*[GpsView(intrinsics(c), pose(c)) for c in cams])


# ---------------------------------------------------------------- C names
def gps_version() -> str:
    return lib().gps_version().decode()


def gps_workspace_size(M: int, cams, s: GpsRenderSettings) -> int:
    n = c_size_t(0)
    v = _size_views(cams)
    _check(lib().gps_workspace_size(M, v, len(cams), ctypes.byref(s), ctypes.byref(n)))
    return int(n.value)


def gps_workspace_layout(M: int, cams, s: GpsRenderSettings, view: int) -> GpsWorkspaceLayout:
    out = GpsWorkspaceLayout()
    v = _size_views(cams)
    _check(lib().gps_workspace_layout(M, v, len(cams), ctypes.byref(s), view, ctypes.byref(out)))
    return out


def gps_query_status(ws: torch.Tensor, stream=None) -> int:
    st = c_int32(0)
    _check(lib().gps_query_status(_ptr(ws), ws.numel(), ctypes.byref(st), _stream(stream)))
    return int(st.value)


def fuse_frame(vol: Tsdf, depth: torch.Tensor, rgb: torch.Tensor, cam, stream=None) -> None:
    K, P = intrinsics(cam), pose(cam)
    t = vol.c()
    _check(lib().fuse_frame(ctypes.byref(t), _ptr(depth), _ptr(rgb), ctypes.byref(K),
                            ctypes.byref(P), _stream(stream)))


def raycast_sdf(vol: Tsdf, cam, near=0.2, far=0.0, out_rgb=None, out_depth=None,
                out_vertex=None, stream=None, precision=PREC_FP32):
    """C_t, D_t (and the world vertex map) of `cam`.  C_t's element type is
    that of out_rgb when given, else the one `precision` names."""
    H, W = cam.height, cam.width
    dev = vol.sdf.device
    if out_rgb is None:
        out_rgb = torch.empty(3, H, W, device=dev, dtype=PREC_DTYPE[precision])
    prec = _precision_of(out_rgb)
    out_depth = out_depth if out_depth is not None else torch.empty(H, W, device=dev)
    K, P = intrinsics(cam), pose(cam)
    t = vol.c()
    _check(lib().raycast_sdf(ctypes.byref(t), ctypes.byref(K), ctypes.byref(P), near, far,
                             _ptr(out_rgb), prec, _ptr(out_depth), _ptr(out_vertex),
                             _stream(stream)))
    return out_rgb, out_depth


def render_forward(g: Gaussians, views: Sequence[View], s: GpsRenderSettings, ws: torch.Tensor,
                   loss: Optional[torch.Tensor] = None, stream=None) -> None:
    gc = g.c()
    va = _views(views, s)
    _check(lib().render_forward(ctypes.byref(gc), va, len(views), ctypes.byref(s), _ptr(ws),
                                ws.numel(), _ptr(loss), _stream(stream)))


def render_forward_noalloc(g: Gaussians, views: Sequence[View], s: GpsRenderSettings,
                           loss: Optional[torch.Tensor] = None, stream=None) -> None:
    """render_forward on the library's static device scratch (no workspace)."""
    gc = g.c()
    va = _views(views, s)
    _check(lib().render_forward_noalloc(ctypes.byref(gc), va, len(views), ctypes.byref(s),
                                        _ptr(loss), _stream(stream)))


def noalloc_status(stream=None) -> int:
    """Status word of the static scratch behind render_forward_noalloc
    (gps_noalloc_query_status; synchronises the stream)."""
    st = c_int32(0)
    _check(lib().gps_noalloc_query_status(ctypes.byref(st), _stream(stream)))
    return st.value


def render_backward(g: Gaussians, views: Sequence[View], s: GpsRenderSettings, ws: torch.Tensor,
                    grads: Gaussians, dloss: Optional[torch.Tensor] = None, stream=None) -> None:
    gc, gr = g.c(), grads.c()
    va = _views(views, s)
    _check(lib().render_backward(ctypes.byref(gc), va, len(views), ctypes.byref(s), _ptr(ws),
                                 ws.numel(), _ptr(dloss), ctypes.byref(gr), _stream(stream)))


def render_backward_adam(g: Gaussians, views: Sequence[View], s: GpsRenderSettings,
                         ws: torch.Tensor, m: Gaussians, v: Gaussians, lr=None, beta1=0.9,
                         beta2=0.999, eps=1e-15, step: int = 1,
                         device_step: Optional[torch.Tensor] = None,
                         dloss: Optional[torch.Tensor] = None, stream=None,
                         lr_sh_rest: float = None) -> None:
    """render_backward + adam_step in one call (at most 8 views); g is updated
    in place."""
    lr = LR_APP_C if lr is None else lr
    h = GpsAdamHyper((c_float * 5)(*lr), beta1, beta2, eps,
                     LR_SH_REST if lr_sh_rest is None else lr_sh_rest)
    gc, mc, vc = g.c(), m.c(), v.c()
    va = _views(views, s)
    _check(lib().render_backward_adam(ctypes.byref(gc), va, len(views), ctypes.byref(s), _ptr(ws),
                                      ws.numel(), _ptr(dloss), ctypes.byref(mc), ctypes.byref(vc),
                                      ctypes.byref(h), step, _ptr(device_step), _stream(stream)))


def gps_autotune_tiles(g: Gaussians, views: Sequence[View], s: GpsRenderSettings,
                       ws: torch.Tensor, scratch_grads: Gaussians, repeats: int = 3,
                       stream=None):
    """Fastest tile shape for these Gaussians and views: ((tile_w, tile_h),
    {shape: ms per forward + backward, or None where skipped})."""
    gc, sg = g.c(), scratch_grads.c()
    va = _views(views, s)
    tw, th = c_int32(0), c_int32(0)
    times = (c_float * len(AUTOTUNE_SHAPES))()
    _check(lib().gps_autotune_tiles(ctypes.byref(gc), va, len(views), ctypes.byref(s), _ptr(ws),
                                    ws.numel(), ctypes.byref(sg), repeats, ctypes.byref(tw),
                                    ctypes.byref(th), times, _stream(stream)))
    return (tw.value, th.value), {shp: (t if t >= 0 else None)
                                  for shp, t in zip(AUTOTUNE_SHAPES, times)}


def gps_edit_scratch_size(capacity: int, width: int, height: int) -> int:
    n = c_size_t(0)
    _check(lib().gps_edit_scratch_size(capacity, width, height, ctypes.byref(n)))
    return int(n.value)


def _gs(z: Optional["Gaussians"], M: Optional[int] = None):
    if z is None:
        return None
    c = z.c()
    if M is not None:
        c.M = M
    return ctypes.byref(c)


def insert_gaussians(g: "Gaussians", M: int, m: Optional["Gaussians"], v: Optional["Gaussians"],
                     grads: Optional["Gaussians"], cam, vertex: torch.Tensor, sdf_depth: torch.Tensor,
                     rendered_rgb: torch.Tensor, weight: torch.Tensor, target_rgb: torch.Tensor,
                     s: GpsEditSettings, scratch: torch.Tensor, count: torch.Tensor,
                     stream=None) -> None:
    """Appends new Gaussians after the first M rows of g (its rows are the
    capacity); the new count lands in count[0] (device int32)."""
    K, P = intrinsics(cam), pose(cam)
    gc = g.c()
    gc.M = M
    _check(lib().insert_gaussians(ctypes.byref(gc), g.M, _gs(m, M), _gs(v, M), _gs(grads, M),
                                  ctypes.byref(K), ctypes.byref(P), _ptr(vertex), _ptr(sdf_depth),
                                  _ptr(rendered_rgb), _ptr(weight), _ptr(target_rgb),
                                  ctypes.byref(s), _ptr(scratch), scratch.numel(), _ptr(count),
                                  _stream(stream)))


def remove_gaussians(g: "Gaussians", M: int, m: Optional["Gaussians"], v: Optional["Gaussians"],
                     grads: Optional["Gaussians"], s: GpsEditSettings, scratch: torch.Tensor,
                     count: torch.Tensor, stream=None) -> None:
    """Compacts the first M rows of g (and m, v, grads); kept count -> count[0]."""
    gc = g.c()
    gc.M = M
    _check(lib().remove_gaussians(ctypes.byref(gc), _gs(m, M), _gs(v, M), _gs(grads, M),
                                  ctypes.byref(s), _ptr(scratch), scratch.numel(), _ptr(count),
                                  _stream(stream)))


def gps_is_keyframe(last_cam, cam, sched: Optional[GpsViewSchedule] = None) -> bool:
    """Host-only: does `cam`'s pose start a new keyframe after `last_cam`'s
    (None: the first frame)?"""
    sched = sched if sched is not None else view_schedule()
    out = c_int32(0)
    last = ctypes.byref(pose(last_cam)) if last_cam is not None else None
    _check(lib().gps_is_keyframe(last, ctypes.byref(pose(cam)), ctypes.byref(sched),
                                 ctypes.byref(out)))
    return bool(out.value)


def gps_select_views(keyframes: Sequence[int], frame: int, event: int,
                     sched: Optional[GpsViewSchedule] = None) -> List[int]:
    """Host-only: frame ids of the optimisation `event` taken at `frame`
    (local frames newest first, then the keyframes drawn)."""
    sched = sched if sched is not None else view_schedule()
    kf = (c_int32 * max(1, len(keyframes)))(*[int(k) for k in keyframes])
    cap = max(0, sched.n_local) + max(0, sched.n_global)
    out = (c_int32 * max(1, cap))()
    n = c_int32(0)
    _check(lib().gps_select_views(kf, len(keyframes), frame, event, ctypes.byref(sched), out, cap,
                                  ctypes.byref(n)))
    return [int(out[i]) for i in range(n.value)]


def gps_icp_workspace_size(width: int, height: int, s: GpsIcpSettings) -> int:
    n = c_size_t(0)
    _check(lib().gps_icp_workspace_size(width, height, ctypes.byref(s), ctypes.byref(n)))
    return int(n.value)


def icp_track(cam, depth: torch.Tensor, ref_vertex: torch.Tensor, ref_depth: torch.Tensor,
              ref_cam, pose_dev: torch.Tensor, s: GpsIcpSettings, ws: torch.Tensor,
              stats: Optional[torch.Tensor] = None, stream=None) -> None:
    """Refines pose_dev (device float [12]: R row-major, t; camera->world) in
    place against the reference ray-cast at ref_cam's pose; cam gives the
    intrinsics of both."""
    K, Pr = intrinsics(cam), pose(ref_cam)
    _check(lib().icp_track(ctypes.byref(K), _ptr(depth), _ptr(ref_vertex), _ptr(ref_depth),
                           ctypes.byref(Pr), ctypes.byref(s), _ptr(pose_dev), _ptr(ws),
                           ws.numel(), _ptr(stats), _stream(stream)))


class PoseCam:
    """Intrinsics of `cam` with another camera->world pose (R [3][3], t [3])."""

    def __init__(self, cam, R, t):
        self.fx, self.fy, self.cx, self.cy = cam.fx, cam.fy, cam.cx, cam.cy
        self.width, self.height = cam.width, cam.height
        self.R = torch.as_tensor(R, dtype=torch.float64).reshape(3, 3).cpu()
        self.t = torch.as_tensor(t, dtype=torch.float64).reshape(3).cpu()


class Tracker:
    """Workspace and device pose of icp_track for frames of `cam`'s size."""

    def __init__(self, cam, s: Optional[GpsIcpSettings] = None, device="cuda"):
        self.cam = cam
        self.s = s if s is not None else icp_settings()
        self.ws = torch.zeros(gps_icp_workspace_size(cam.width, cam.height, self.s),
                              dtype=torch.uint8, device=device)
        self.pose = torch.zeros(12, device=device)
        n_it = sum(self.s.iters[l] for l in range(self.s.levels))
        self.stats = torch.zeros(max(1, n_it), 2, device=device)

    def track(self, depth: torch.Tensor, ref_vertex: torch.Tensor, ref_depth: torch.Tensor,
              ref_cam, init_cam=None, stream=None) -> None:
        """Pose of the frame `depth` against the reference ray-cast at
        ref_cam; starts from init_cam's pose (default: ref_cam's).  The
        result stays in self.pose (device); read it with `result()`."""
        c = init_cam if init_cam is not None else ref_cam
        R = torch.as_tensor(c.R, dtype=torch.float32).reshape(9)
        t = torch.as_tensor(c.t, dtype=torch.float32).reshape(3)
        self.pose.copy_(torch.cat([R, t]).to(self.pose.device), non_blocking=True)
        icp_track(self.cam, depth, ref_vertex, ref_depth, ref_cam, self.pose, self.s, self.ws,
                  self.stats, stream)

    def result(self) -> PoseCam:
        p = self.pose.double().cpu()
        return PoseCam(self.cam, p[:9].reshape(3, 3), p[9:])


def adam_step(params: Gaussians, grads: Gaussians, m: Gaussians, v: Gaussians, lr=LR_APP_C,
              beta1=0.9, beta2=0.999, eps=1e-15, step: int = 1,
              device_step: Optional[torch.Tensor] = None, stream=None,
              lr_sh_rest: float = LR_SH_REST) -> None:
    h = GpsAdamHyper((c_float * 5)(*lr), beta1, beta2, eps, lr_sh_rest)
    pc, gc, mc, vc = params.c(), grads.c(), m.c(), v.c()
    _check(lib().adam_step(ctypes.byref(pc), ctypes.byref(gc), ctypes.byref(mc), ctypes.byref(vc),
                           ctypes.byref(h), step, _ptr(device_step), _stream(stream)))


# ---------------------------------------------------------------- holders
class Renderer:
    """Owns the workspace of render_forward / render_backward for fixed sizes."""

    def __init__(self, M: int, cams, s: Optional[GpsRenderSettings] = None, device="cuda"):
        self.s = s if s is not None else settings()
        self.cams = list(cams)
        self.M = M
        nbytes = gps_workspace_size(M, self.cams, self.s)
        self.ws = torch.zeros(nbytes, dtype=torch.uint8, device=device)

    def layout(self, view: int = 0) -> GpsWorkspaceLayout:
        return gps_workspace_layout(self.M, self.cams, self.s, view)

    def region(self, view: int, name: str, dtype, count: int) -> torch.Tensor:
        L = self.layout(view)
        off = getattr(L, name)
        esz = torch.empty((), dtype=dtype).element_size()
        return self.ws[off:off + count * esz].view(dtype)

    def forward(self, g: Gaussians, views: Sequence[View], loss=None, stream=None):
        render_forward(g, views, self.s, self.ws, loss, stream)

    def backward(self, g: Gaussians, views: Sequence[View], grads: Gaussians, dloss=None,
                 stream=None):
        render_backward(g, views, self.s, self.ws, grads, dloss, stream)

    def status(self, stream=None) -> int:
        return gps_query_status(self.ws, stream)

    def autotune(self, g: Gaussians, views: Sequence[View], repeats: int = 3, stream=None):
        """Time every tile shape on these Gaussians and views, switch to the
        fastest and size the workspace for it.  Returns gps_autotune_tiles'
        result.  Synchronises; call before capturing graphs."""
        need = 0
        for tw, th in AUTOTUNE_SHAPES:
            s = GpsRenderSettings.from_buffer_copy(self.s)
            s.tile_w, s.tile_h = tw, th
            need = max(need, gps_workspace_size(self.M, self.cams, s))
        dev = self.ws.device
        self.ws = torch.zeros(need, dtype=torch.uint8, device=dev)
        best, times = gps_autotune_tiles(g, views, self.s, self.ws, g.zeros_like(), repeats, stream)
        self.s.tile_w, self.s.tile_h = best
        self.ws = torch.zeros(gps_workspace_size(self.M, self.cams, self.s), dtype=torch.uint8,
                              device=dev)
        return best, times


class Adam:
    """Adam state (FP32 moments) for a Gaussian set; step() calls adam_step."""

    def __init__(self, params: Gaussians, lr=LR_APP_C, betas=(0.9, 0.999), eps=1e-15,
                 device_step: bool = False, lr_sh_rest: float = LR_SH_REST):
        self.params = params
        self.m = params.zeros_like()
        self.v = params.zeros_like()
        self.lr, self.betas, self.eps, self.lr_sh_rest = lr, betas, eps, lr_sh_rest
        self.t = 0
        self.device_step = (torch.zeros(1, dtype=torch.int32, device=params.means.device)
                            if device_step else None)

    def step(self, grads: Gaussians, stream=None):
        if self.device_step is not None:
            adam_step(self.params, grads, self.m, self.v, self.lr, *self.betas, self.eps, 0,
                      self.device_step, stream, self.lr_sh_rest)
        else:
            self.t += 1
            adam_step(self.params, grads, self.m, self.v, self.lr, *self.betas, self.eps, self.t,
                      None, stream, self.lr_sh_rest)

    def backward_step(self, views: Sequence[View], s: GpsRenderSettings, ws: torch.Tensor,
                      dloss: Optional[torch.Tensor] = None, stream=None):
        """render_backward of the last forward and this optimiser's step in one
        call (render_backward_adam: no gradient array)."""
        if self.device_step is not None:
            step = 0
        else:
            self.t += 1
            step = self.t
        render_backward_adam(self.params, views, s, ws, self.m, self.v, self.lr, *self.betas,
                             self.eps, step, self.device_step, dloss, stream, self.lr_sh_rest)


class RenderImages(torch.autograd.Function):
    """C*, D*, W_G of one view as differentiable outputs of the parameter
    tensors (means, log_scales, quats, logits, rgb[, sh_rest]); the backward
    calls render_backward with dL/dC*, dL/dD*.  The renderer's workspace holds
    this forward's state until the backward: one forward in flight per
    renderer."""

    @staticmethod
    def forward(ctx, renderer: Renderer, view: View, *params):
        g = Gaussians(*[t.detach() for t in params])
        means = params[0]
        H, W = view.cam.height, view.cam.width
        dev = means.device
        cdt = PREC_DTYPE[renderer.s.precision]
        out = dataclasses.replace(view, target_rgb=None, target_depth=None,
                                  out_rgb=torch.empty(3, H, W, device=dev, dtype=cdt),
                                  out_depth=torch.empty(H, W, device=dev),
                                  out_weight=torch.empty(H, W, device=dev))
        renderer.forward(g, [out])
        ctx.renderer, ctx.view, ctx.g = renderer, out, g
        ctx.mark_non_differentiable(out.out_weight)
        return out.out_rgb, out.out_depth, out.out_weight

    @staticmethod
    def backward(ctx, d_rgb, d_depth, d_weight):
        g = ctx.g
        grads = g.zeros_like()
        # upstream gradients are float32 whatever the colour storage type
        v = dataclasses.replace(ctx.view,
                                grad_rgb=(d_rgb.float().contiguous() if d_rgb is not None
                                          else torch.zeros_like(ctx.view.out_depth).expand(3, -1, -1).contiguous()),
                                grad_depth=(d_depth.contiguous() if d_depth is not None
                                            else torch.zeros_like(ctx.view.out_depth)))
        ctx.renderer.backward(g, [v], grads)
        return (None, None, *grads.tensors())


class RenderLoss(torch.autograd.Function):
    """Fused colour (+ depth) L1 loss of Eq. 6 over views with targets, as a
    function of the parameter tensors (means, log_scales, quats, logits,
    rgb[, sh_rest])."""

    @staticmethod
    def forward(ctx, renderer: Renderer, views: Sequence[View], *params):
        g = Gaussians(*[t.detach() for t in params])
        loss = torch.zeros(1, device=params[0].device)
        renderer.forward(g, views, loss)
        ctx.renderer, ctx.views, ctx.g = renderer, views, g
        return loss[0]

    @staticmethod
    def backward(ctx, dloss):
        g = ctx.g
        grads = g.zeros_like()
        ctx.renderer.backward(g, ctx.views, grads, dloss.reshape(1).contiguous().float())
        return (None, None, *grads.tensors())
