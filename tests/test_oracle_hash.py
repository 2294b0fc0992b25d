"""Pins of the oracle's voxel-hashing semantics (oracle/tsdf.cpp, orc_fuse
with a brick allocation mask): which bricks a frame allocates, that the
update arithmetic inside allocated bricks is the dense one, and the
closed-form values of bricks allocated in a later frame."""
import numpy as np

import oracle
from datagen.scenes import TsdfSpec


class _Cam:
    def __init__(self, W=40, H=30, f=50.0):
        self.fx = self.fy = f
        self.cx, self.cy = W / 2, H / 2
        self.width, self.height = W, H
        self.R = np.eye(3)
        self.t = np.zeros(3)


SPEC = TsdfSpec(64, 64, 64, 0.02, (-0.64, -0.64, 0.2), 0.06)


def _plane(Z, cam):
    return np.full((cam.height, cam.width), Z), np.full((3, cam.height, cam.width), 0.5)


def _centres(spec):
    k = np.arange(spec.nx)
    return (spec.origin[0] + (k + 0.5) * spec.voxel, spec.origin[1] + (k + 0.5) * spec.voxel,
            spec.origin[2] + (k + 0.5) * spec.voxel)


def test_fronto_parallel_plane_allocates_the_band_bricks():
    cam = _Cam()
    Z0 = 1.01
    vol = oracle.Volume(SPEC, hashed=True)
    d, c = _plane(Z0, cam)
    oracle.fuse(vol, d, c, cam)
    # by hand: voxel (x, y, z) is in the band when |Z0 - z| < trunc and its
    # centre projects inside the image; its brick is then allocated
    xs, ys, zs = _centres(SPEC)
    want = np.zeros_like(vol.alloc)
    for iz, z in enumerate(zs):
        if abs(Z0 - z) >= SPEC.trunc:
            continue
        u = np.floor(cam.fx * xs / z + cam.cx + 0.5)
        v = np.floor(cam.fy * ys / z + cam.cy + 0.5)
        okx = np.nonzero((u >= 0) & (u <= cam.width - 1))[0]
        oky = np.nonzero((v >= 0) & (v <= cam.height - 1))[0]
        want[iz // 8, oky.min() // 8:oky.max() // 8 + 1, okx.min() // 8:okx.max() // 8 + 1] = 1
    np.testing.assert_array_equal(vol.alloc, want)
    assert 0 < want.sum() < want.size // 4


def test_allocated_bricks_carry_the_dense_update():
    cam = _Cam()
    d, c = _plane(1.01, cam)
    d[10:20, 5:25] = 0.77                      # a step, so the band bends
    dense, hashed = oracle.Volume(SPEC), oracle.Volume(SPEC, hashed=True)
    oracle.fuse(dense, d, c, cam)
    oracle.fuse(hashed, d, c, cam)
    a = np.repeat(np.repeat(np.repeat(hashed.alloc, 8, 0), 8, 1), 8, 2).astype(bool)
    for f in ("sdf", "w", "cw"):
        np.testing.assert_array_equal(getattr(hashed, f)[a], getattr(dense, f)[a])
    np.testing.assert_array_equal(hashed.rgb[a], dense.rgb[a])
    assert np.all(hashed.sdf[~a] == 1) and np.all(hashed.w[~a] == 0) and np.all(hashed.rgb[~a] == 0)
    # every band voxel (colour updated) lies in an allocated brick
    assert np.all(a[dense.cw > 0])
    # the dense volume updated free-space voxels the hashed one never stores
    assert (dense.w[~a] > 0).any()


def test_bricks_allocated_later_start_fresh():
    """Frame 0 sees a plane at 1.31 m, frame 1 one at 1.01 m.  Voxels near 1.01
    were free space in frame 0 (dense: sdf stays 1, weight 1), so the dense
    volume averages frame 1's value with that 1, while a brick allocated in
    frame 1 holds frame 1's value alone: sdf = min(1, (1.01 - z) / mu), w = 1."""
    cam = _Cam()
    dense, hashed = oracle.Volume(SPEC), oracle.Volume(SPEC, hashed=True)
    for Z in (1.31, 1.01):
        d, c = _plane(Z, cam)
        oracle.fuse(dense, d, c, cam)
        oracle.fuse(hashed, d, c, cam)
    _, _, zs = _centres(SPEC)
    iz = int(np.argmin(np.abs(zs - 0.99)))     # z = 0.99 m: in frame 1's band only
    z = zs[iz]
    f = min(1.0, (1.01 - z) / SPEC.trunc)
    y, x = SPEC.ny // 2, SPEC.nx // 2          # on the optical axis
    assert hashed.alloc[iz // 8, y // 8, x // 8] == 1
    np.testing.assert_allclose(hashed.sdf[iz, y, x], f, rtol=1e-12)
    assert hashed.w[iz, y, x] == 1.0
    np.testing.assert_allclose(dense.sdf[iz, y, x], (1.0 + f) / 2.0, rtol=1e-12)
    assert dense.w[iz, y, x] == 2.0
