"""The online reconstruction loop (Sec. 3.2, Fig. 2) on one device, built on
the C-ABI calls: every frame is tracked (optional), fused into the TSDF and
tested as a keyframe; every `interval` frames a Gaussian reconstruction runs -
insertion on that frame, selection of the optimisation views (Fig. 5), one
ray-cast per view, `iterations` batched forward + backward + Adam steps over
those views, and removal.

The volume is a dense `Tsdf` or a voxel-hashed `HashTsdf`.  With
track=True, frame k > 0 is tracked by point-to-plane ICP against the
ray-cast of the TSDF at frame k-1's estimated pose, starting from that pose,
and is fused and later rendered at its estimate; frame 0 keeps the pose it
is given (it anchors the map).  Without tracking the given poses are used.

Device memory is fixed at construction: the Gaussians, their gradients and
Adam moments have `capacity` rows, the render workspace is sized for
`capacity` Gaussians and `max_views` views, and every frame that a later
optimisation can select (the frames of the current interval and all
keyframes) keeps its colour and depth on the device.  The host reads the
Gaussian count back twice per reconstruction (after insertion and after
removal), because the launch sizes of the next calls depend on it.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import torch

from . import (LR_APP_C, PREC_DTYPE, GpsEditSettings, GpsIcpSettings, GpsRenderSettings,
               GpsViewSchedule, Gaussians, HashTsdf, PoseCam, Tracker, Tsdf, View, adam_step,
               edit_settings, fuse_frame, fuse_frame_hashed, gps_edit_scratch_size,
               gps_is_keyframe, gps_query_status, gps_select_views, gps_workspace_size,
               insert_gaussians, raycast_sdf, raycast_sdf_hashed, remove_gaussians,
               render_backward, render_backward_adam, render_forward,
               settings as render_settings, view_schedule)
from . import GPS_OK, GpsError

MAX_VIEWS_PER_CALL = 8  # views one render_forward / render_backward call takes


def fuse_volume(vol, depth, rgb, cam):
    """fuse_frame or fuse_frame_hashed, by the volume's type."""
    if isinstance(vol, HashTsdf):
        fuse_frame_hashed(vol, depth, rgb, cam)
    else:
        fuse_frame(vol, depth, rgb, cam)


def raycast_volume(vol, cam, near, out_rgb, out_depth, out_vertex=None):
    """raycast_sdf or raycast_sdf_hashed, by the volume's type."""
    if isinstance(vol, HashTsdf):
        return raycast_sdf_hashed(vol, cam, near, 0.0, out_rgb, out_depth, out_vertex)
    return raycast_sdf(vol, cam, near, 0.0, out_rgb, out_depth, out_vertex)


@dataclasses.dataclass
class Reconstruction:
    """What one Gaussian reconstruction did (host values, read after it ran)."""
    frame: int
    views: List[int]
    inserted: int
    removed: int
    count: int            # Gaussians after removal
    loss_first: float     # fused L1 of the first iteration (summed over the views)
    loss_last: float      # and of the last


def _rows(g: Gaussians, n: int) -> Gaussians:
    return Gaussians(*[t[:n] for t in g.tensors()])  # sh_rest too, when present


class Mapper:
    def __init__(self, vol, cam, capacity: int,
                 s: Optional[GpsRenderSettings] = None,
                 edit: Optional[GpsEditSettings] = None,
                 sched: Optional[GpsViewSchedule] = None,
                 iterations: int = 20, lr=LR_APP_C, near: float = 0.2,
                 max_views: Optional[int] = None, sh_degree: int = 0, track: bool = False,
                 icp: Optional[GpsIcpSettings] = None, device="cuda"):
        self.vol, self.cam, self.capacity = vol, cam, capacity
        self.s = GpsRenderSettings.from_buffer_copy(s if s is not None else
                                                    render_settings(tile=(16, 8)))
        if self.s.pair_capacity == 0:
            # fixed for the capacity, so that the layout does not shrink with the count
            self.s.pair_capacity = 16 * capacity
        self.edit = edit if edit is not None else edit_settings(precision=self.s.precision)
        if self.edit.precision != self.s.precision:
            raise ValueError("edit and render settings must store colour in the same precision")
        self.sched = sched if sched is not None else view_schedule()
        self.iterations, self.lr, self.near = iterations, lr, near
        self.dtype = PREC_DTYPE[self.s.precision]
        dev = torch.device(device)
        H, W = cam.height, cam.width

        K = (sh_degree + 1) ** 2 - 1

        def zeros():
            return Gaussians(torch.zeros(capacity, 3, device=dev),
                             torch.zeros(capacity, 3, device=dev),
                             torch.zeros(capacity, 4, device=dev),
                             torch.zeros(capacity, device=dev),
                             torch.zeros(capacity, 3, device=dev),
                             torch.zeros(capacity, K, 3, device=dev) if K else None)
        self.g, self.grads, self.m, self.v = zeros(), zeros(), zeros(), zeros()
        self.M = 0
        self.t = 0          # Adam step counter shared by all reconstructions
        nv = max_views if max_views is not None else \
            max(1, self.sched.n_local) + max(0, self.sched.n_global)
        self.max_views = nv
        per_call = min(nv, MAX_VIEWS_PER_CALL)
        self.ws = torch.zeros(gps_workspace_size(capacity, [cam] * per_call, self.s),
                              dtype=torch.uint8, device=dev)
        self.scratch = torch.zeros(gps_edit_scratch_size(capacity, W, H), dtype=torch.uint8,
                                   device=dev)
        self.count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.loss = torch.zeros(2, device=dev)
        self.loss_parts = torch.zeros((nv + MAX_VIEWS_PER_CALL - 1) // MAX_VIEWS_PER_CALL,
                                      device=dev)
        # per-view buffers of one reconstruction
        self.ct = [torch.zeros(3, H, W, device=dev, dtype=self.dtype) for _ in range(nv)]
        self.dt = [torch.zeros(H, W, device=dev) for _ in range(nv)]
        self.vertex = torch.zeros(H, W, 3, device=dev)
        self.c_star = torch.zeros(3, H, W, device=dev, dtype=self.dtype)
        self.d_star = torch.zeros(H, W, device=dev)
        self.w_g = torch.zeros(H, W, device=dev)
        # frames a later optimisation can select: id -> (cam, rgb, depth)
        self.frames: Dict[int, tuple] = {}
        self.keyframes: List[int] = []
        self.last_keyframe_cam = None
        self.event = 0
        self.history: List[Reconstruction] = []
        # tracking: the reference ray-cast at the previous estimate
        self.tracker = Tracker(cam, icp, device=dev) if track else None
        if track:
            self.ref_rgb = torch.zeros(3, H, W, device=dev)
            self.ref_depth = torch.zeros(H, W, device=dev)
            self.ref_vertex = torch.zeros(H, W, 3, device=dev)
        self.poses: List = []     # estimated (or given) camera of every frame

    def reset(self) -> None:
        """Forget every frame, keyframe and Gaussian (the TSDF is the
        caller's: reset it separately)."""
        for g in (self.grads, self.m, self.v):
            for t in g.tensors():
                t.zero_()
        self.M = self.t = self.event = 0
        self.frames.clear()
        self.keyframes.clear()
        self.poses.clear()
        self.last_keyframe_cam = None
        self.history.clear()

    # ------------------------------------------------------------ per frame
    def process(self, frame: int, cam, rgb: torch.Tensor,
                depth: torch.Tensor) -> Optional[Reconstruction]:
        """Fuse one frame (rgb [3][H][W] float32, depth [H][W] metres) taken
        at `cam`'s pose, then run a reconstruction if `frame` closes an
        interval.  Frames must arrive in order, numbered from 0.  Everything
        is enqueued on torch's current stream."""
        if self.tracker is not None and self.poses:
            prev = self.poses[-1]
            raycast_volume(self.vol, prev, self.near, self.ref_rgb, self.ref_depth, self.ref_vertex)
            self.tracker.track(depth, self.ref_vertex, self.ref_depth, prev)
            cam = self.tracker.result()          # reads the pose back (synchronises)
        self.poses.append(cam)
        fuse_volume(self.vol, depth, rgb, cam)
        if gps_is_keyframe(self.last_keyframe_cam, cam, self.sched):
            self.keyframes.append(frame)
            self.last_keyframe_cam = cam
        self.frames[frame] = (cam, rgb.to(self.dtype, copy=True), depth.clone())
        # keep what a later selection can still pick: the interval and the keyframes
        oldest_local = frame - self.sched.interval + 1
        kf = set(self.keyframes)
        for f in [f for f in self.frames if f < oldest_local and f not in kf]:
            del self.frames[f]
        if (frame + 1) % self.sched.interval == 0:
            return self.reconstruct(frame)
        return None

    # ---------------------------------------------------- Gaussian reconstruction
    def _sync_count(self) -> int:
        return int(self.count.item())   # synchronises the current stream

    def reconstruct(self, frame: int) -> Reconstruction:
        cam, rgb, depth = self.frames[frame]
        # insertion (Sec. 3.2): second-pass render of this frame with the
        # current Gaussians gives C* and W_G
        ct, dt = raycast_volume(self.vol, cam, self.near, self.ct[0], self.dt[0], self.vertex)
        if self.M > 0:
            v = View(cam, ct, dt, out_rgb=self.c_star, out_depth=self.d_star, out_weight=self.w_g)
            render_forward(_rows(self.g, self.M), [v], self.s, self.ws, None)
        else:
            self.c_star.copy_(ct)
            self.w_g.zero_()
        M0 = self.M
        insert_gaussians(self.g, M0, self.m, self.v, self.grads, cam, self.vertex, dt,
                         self.c_star, self.w_g, rgb, self.edit, self.scratch, self.count)
        self.M = self._sync_count()
        inserted = self.M - M0
        # the views of this optimisation (Fig. 5), ray-cast once with the latest SDF
        ids = gps_select_views(self.keyframes, frame, self.event, self.sched)[:self.max_views]
        views = []
        for k, f in enumerate(ids):
            c, col, dep = self.frames[f]
            if not (k == 0 and f == frame):    # view 0 is usually this frame: ray-cast above
                raycast_volume(self.vol, c, self.near, self.ct[k], self.dt[k], None)
            views.append(View(c, self.ct[k], self.dt[k], col, dep))
        g, gr = _rows(self.g, self.M), _rows(self.grads, self.M)
        m, v = _rows(self.m, self.M), _rows(self.v, self.M)
        self.loss.zero_()
        if self.M > 0:
            for it in range(self.iterations):
                if len(views) <= MAX_VIEWS_PER_CALL:
                    # one call per stage for all views; the backward feeds Adam
                    # directly (render_backward_adam)
                    render_forward(g, views, self.s, self.ws, self.loss_parts[:1])
                    self.t += 1
                    render_backward_adam(g, views, self.s, self.ws, m, v, self.lr, 0.9, 0.999,
                                         1e-15, self.t)
                else:
                    for b in range(0, len(views), MAX_VIEWS_PER_CALL):
                        k = b // MAX_VIEWS_PER_CALL
                        part = views[b:b + MAX_VIEWS_PER_CALL]
                        render_forward(g, part, self.s, self.ws, self.loss_parts[k:k + 1])
                        render_backward(g, part, self.s, self.ws, gr, None)
                    self.t += 1
                    adam_step(g, gr, m, v, self.lr, 0.9, 0.999, 1e-15, self.t, None)
                if it == 0 or it == self.iterations - 1:
                    self.loss[min(it, 1)] = self.loss_parts.sum()
        st = gps_query_status(self.ws)
        if st != GPS_OK:
            raise GpsError(st, "device status after the optimisation")
        # removal (Sec. 3.2)
        before = self.M
        if self.M > 0:
            remove_gaussians(self.g, self.M, self.m, self.v, self.grads, self.edit, self.scratch,
                             self.count)
            self.M = self._sync_count()
        losses = self.loss.tolist()
        r = Reconstruction(frame, ids, inserted, before - self.M, self.M, losses[0],
                           losses[1] if self.iterations > 1 else losses[0])
        self.event += 1
        self.history.append(r)
        return r

    def gaussians(self) -> Gaussians:
        """The current Gaussians (row views of the capacity buffers)."""
        return _rows(self.g, self.M)
