"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/gps.h declares, the ctypes mirrors match the C struct
layouts, and argument validation rejects bad calls before any launch."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2509_11574_b300 as gps
from paper_2509_11574_b300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gps.h")


@pytest.fixture(scope="module")
def L():
    gbuild.build()
    return gps.lib()


def declared_functions():
    src = open(HEADER).read()
    return re.findall(r"GPS_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)


def test_header_declares_the_five_calls():
    names = declared_functions()
    for n in ("fuse_frame", "raycast_sdf", "render_forward", "render_backward", "adam_step"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    out = subprocess.check_output(["nm", "-D", "--defined-only", gps.LIB_PATH]).decode()
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for n in declared_functions():
        assert n in exported, n
        assert hasattr(L, n)
    assert set(gps.EXPORTED) == set(declared_functions())


def test_struct_layouts_match_header(tmp_path):
    structs = ["GpsIntrinsics", "GpsPose", "GpsTsdf", "GpsGaussians", "GpsView",
               "GpsRenderSettings", "GpsAdamHyper", "GpsWorkspaceLayout", "GpsEditSettings",
               "GpsViewSchedule", "GpsIcpSettings", "GpsHashTsdf"]
    prog = tmp_path / "sz.c"
    body = "".join(f'  printf("{s} %zu\\n", sizeof({s}));\n' for s in structs)
    body += '  printf("off_pair_capacity %zu\\n", offsetof(GpsRenderSettings, pair_capacity));\n'
    body += '  printf("off_grad_depth %zu\\n", offsetof(GpsView, grad_depth));\n'
    body += '  printf("off_schedule %zu\\n", offsetof(GpsRenderSettings, schedule));\n'
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gps.h"\nint main(){\n'
                    + body + "  return 0;\n}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)])
    sizes = dict(ln.split() for ln in subprocess.check_output([str(exe)]).decode().splitlines())
    for s in structs:
        assert int(sizes[s]) == ctypes.sizeof(getattr(gps, s)), s
    assert int(sizes["off_pair_capacity"]) == gps.GpsRenderSettings.pair_capacity.offset
    assert int(sizes["off_schedule"]) == gps.GpsRenderSettings.schedule.offset
    assert int(sizes["off_grad_depth"]) == gps.GpsView.grad_depth.offset


class _Cam:
    def __init__(self, W, H):
        self.fx = self.fy = 100.0
        self.cx, self.cy = W / 2, H / 2
        self.width, self.height = W, H
        self.R = [1, 0, 0, 0, 1, 0, 0, 0, 1]
        self.t = [0, 0, 0]


def test_workspace_size_and_layout_host_only(L):
    # depth-sorted lists (the "with sort" blend): super-tile bins
    s = gps.settings(deterministic=True, blend_mode=gps.BLEND_ALPHA)
    cams = [_Cam(160, 120), _Cam(77, 33)]
    n = gps.gps_workspace_size(2000, cams, s)
    assert n > 0 and n % 256 == 0
    L0 = gps.gps_workspace_layout(2000, cams, s, 0)
    L1 = gps.gps_workspace_layout(2000, cams, s, 1)
    assert L0.tiles_x == 10 and L0.tiles_y == 8 and L1.tiles_x == 5 and L1.tiles_y == 3
    # 16 x 16 tiles are whole 16-px super-tiles: the tile lists are the segments
    assert L0.records < L0.super_keys == L0.pair_keys < L0.grad2d < L1.records
    assert L0.tile_ranges == L0.super_ranges
    for off in (L0.records, L0.block_base, L0.pair_keys, L0.pix_state, L1.grad2d):
        assert off % 256 == 0
    assert L0.pair_capacity == 16 * 2000
    assert (L0.super_px, L0.super_x, L0.super_y, L1.super_x, L1.super_y) == (16, 10, 8, 5, 3)
    assert L0.tile_bins == 0
    L8 = gps.gps_workspace_layout(2000, cams, gps.settings(tile=(16, 8), blend_mode=gps.BLEND_ALPHA), 0)
    assert L8.super_keys < L8.pair_keys and L8.super_ranges < L8.tile_ranges
    assert L8.tiles_y == 15
    # deterministic mode with the OIT blend: fixed-order lists straight into
    # tile bins (no sort) up to 6144 tiles per view, else depth-sorted super-tiles
    D8 = gps.gps_workspace_layout(2000, cams, gps.settings(tile=(16, 8), deterministic=True), 0)
    assert D8.tile_bins == 1 and D8.super_px == 0 and D8.pair_keys == D8.super_keys
    D_big = gps.gps_workspace_layout(10, [_Cam(1280, 720)], gps.settings(tile=(8, 8), deterministic=True), 0)
    assert D_big.tiles_x * D_big.tiles_y == 14400 > 6144
    assert D_big.tile_bins == 0 and D_big.super_px == 16
    L32 = gps.gps_workspace_layout(2000, cams, gps.settings(tile=(32, 8), blend_mode=gps.BLEND_ALPHA), 0)
    assert L32.super_px == 32 and (L32.super_x, L32.super_y) == (5, 4)
    # unsorted lists (the default): the bins are the tiles, the emission writes
    # the lists (room for tiles per super-tile x pair_capacity entries)
    T8 = gps.gps_workspace_layout(2000, cams, gps.settings(tile=(16, 8)), 0)
    assert T8.tile_bins == 1 and T8.super_px == 0
    assert (T8.super_x, T8.super_y) == (T8.tiles_x, T8.tiles_y) == (10, 15)
    assert T8.pair_keys == T8.super_keys == T8.super_scratch and T8.tile_ranges == T8.super_ranges
    assert T8.pix_state - T8.pair_keys >= 2 * 16 * 2000 * 8
    T32 = gps.gps_workspace_layout(2000, cams, gps.settings(tile=(32, 8)), 1)
    assert T32.tile_bins == 1 and (T32.super_x, T32.super_y) == (3, 5)
    # a tile grid too large for the shared-memory histogram: super-tile bins
    big = gps.gps_workspace_layout(10, [_Cam(2048, 1040)], gps.settings(tile=(8, 8)), 0)
    assert big.tile_bins == 0 and big.super_px == 16
    # binning blocks take 256 Gaussians, or up to 8 chunks of 256 so that
    # about 600 blocks remain: one block-base row per block
    Lm = gps.gps_workspace_layout(1_000_000, cams[:1], gps.settings(tile=(16, 8)), 0)
    assert Lm.super_ranges - Lm.block_base == -(-652 * 150 * 4 // 256) * 256  # 6 chunks
    Ls = gps.gps_workspace_layout(100_000, cams[:1], gps.settings(tile=(16, 8)), 0)
    assert Ls.super_ranges - Ls.block_base == -(-391 * 150 * 4 // 256) * 256  # 1 chunk
    n = gps.gps_workspace_size(2000, cams, gps.settings())
    assert gps.gps_workspace_size(2000, cams, s) > n
    with pytest.raises(gps.GpsError) as e:
        gps.gps_workspace_size(2000, cams, gps.settings(tile=(12, 12)))
    assert e.value.code == gps.GPS_ERR_INVALID_ARG
    with pytest.raises(gps.GpsError):
        gps.gps_workspace_size(2000, [_Cam(0, 10)], s)


def test_invalid_arguments_fail_before_launch(L):
    K = gps.GpsIntrinsics(100.0, 100.0, 10.0, 10.0, 20, 20)
    P = gps.GpsPose((ctypes.c_float * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1), (ctypes.c_float * 3)(0, 0, 0))
    vol = gps.GpsTsdf(12, 8, 8, 0.01, (ctypes.c_float * 3)(0, 0, 0), 0.03, 100.0, None, None, None)
    assert L.fuse_frame(ctypes.byref(vol), None, None, ctypes.byref(K), ctypes.byref(P), None) \
        == gps.GPS_ERR_INVALID_ARG
    assert b"NULL" in L.gps_last_error()
    fake = ctypes.c_void_p(4096)
    assert L.fuse_frame(ctypes.byref(vol), fake, fake, ctypes.byref(K), ctypes.byref(P), None) \
        == gps.GPS_ERR_INVALID_ARG  # nx = 12 is not a multiple of 8
    g = gps.GpsGaussians(None, None, None, None, None, 10)
    v = (gps.GpsView * 1)(gps.GpsView(K, P))
    s = gps.settings()
    assert L.render_forward(ctypes.byref(g), v, 1, ctypes.byref(s), fake, 1 << 20, None, None) \
        == gps.GPS_ERR_INVALID_ARG
    gz = gps.GpsGaussians(None, None, None, None, None, 0)
    # sdf images missing
    assert L.render_forward(ctypes.byref(gz), v, 1, ctypes.byref(s), fake, 1 << 20, None, None) \
        == gps.GPS_ERR_INVALID_ARG
    v[0].sdf_rgb = fake
    v[0].sdf_depth = fake
    # workspace too small
    assert L.render_forward(ctypes.byref(gz), v, 1, ctypes.byref(s), fake, 256, None, None) \
        == gps.GPS_ERR_WORKSPACE_TOO_SMALL
    pg_alpha = gps.settings(blend_mode=gps.BLEND_ALPHA, schedule=gps.SCHEDULE_PER_GAUSSIAN)
    assert L.render_forward(ctypes.byref(gz), v, 1, ctypes.byref(pg_alpha), fake, 1 << 30, None,
                            None) == gps.GPS_ERR_INVALID_ARG
    assert b"order-independent" in L.gps_last_error()
    bad = gps.settings(blend_mode=7)
    assert L.render_forward(ctypes.byref(gz), v, 1, ctypes.byref(bad), fake, 1 << 30, None, None) \
        == gps.GPS_ERR_INVALID_ARG
    vol8 = gps.GpsTsdf(8, 8, 8, 0.01, (ctypes.c_float * 3)(0, 0, 0), 0.03, 100.0, fake, fake, fake)
    assert L.raycast_sdf(ctypes.byref(vol8), ctypes.byref(K), ctypes.byref(P), 0.2, 0.0, fake, 9,
                         fake, None, None) == gps.GPS_ERR_INVALID_ARG
    assert b"precision" in L.gps_last_error()
    tw, th = ctypes.c_int32(0), ctypes.c_int32(0)
    assert L.gps_autotune_tiles(ctypes.byref(gz), v, 1, ctypes.byref(s), fake, 1 << 20, None, 3,
                                ctypes.byref(tw), ctypes.byref(th), None, None) \
        == gps.GPS_ERR_INVALID_ARG
    assert L.gps_autotune_tiles(ctypes.byref(gz), v, 1, ctypes.byref(s), fake, 1 << 20,
                                ctypes.byref(gz), 0, ctypes.byref(tw), ctypes.byref(th), None,
                                None) == gps.GPS_ERR_INVALID_ARG
    es = gps.edit_settings()
    cnt = ctypes.c_void_p(512)
    assert L.insert_gaussians(ctypes.byref(gz), 10, None, None, None, ctypes.byref(K),
                              ctypes.byref(P), None, fake, fake, fake, fake, ctypes.byref(es),
                              fake, 1 << 20, cnt, None) == gps.GPS_ERR_INVALID_ARG
    assert L.remove_gaussians(ctypes.byref(gz), None, None, None, ctypes.byref(es), None, 0, cnt,
                              None) == gps.GPS_ERR_INVALID_ARG
    n = ctypes.c_size_t(0)
    assert L.gps_edit_scratch_size(1000, 640, 480, ctypes.byref(n)) == gps.GPS_OK
    assert n.value >= 1000 * 56 + 2 * 640 * 480
    h = gps.GpsAdamHyper((ctypes.c_float * 5)(*gps.LR_APP_C), 0.9, 0.999, 1e-15)
    assert L.adam_step(ctypes.byref(gz), ctypes.byref(gz), ctypes.byref(gz), ctypes.byref(gz),
                       ctypes.byref(h), 0, None, None) == gps.GPS_ERR_INVALID_ARG
    # the fused backward + Adam: one batch of at most 8 views, every stage,
    # targets or upstream gradients, and adam_step's own checks
    v9 = (gps.GpsView * 9)(*[gps.GpsView(K, P, fake, fake, fake, fake) for _ in range(9)])
    assert L.render_backward_adam(ctypes.byref(gz), v9, 9, ctypes.byref(s), fake, 1 << 30, None,
                                  ctypes.byref(gz), ctypes.byref(gz), ctypes.byref(h), 1, None,
                                  None) == gps.GPS_ERR_INVALID_ARG
    assert b"at most 8 views" in L.gps_last_error()
    staged = gps.settings()
    staged.stages = gps.STAGE_COMPOSITE_BWD   # the Adam step needs the projection adjoint
    assert L.render_backward_adam(ctypes.byref(gz), v9, 1, ctypes.byref(staged), fake, 1 << 30,
                                  None, ctypes.byref(gz), ctypes.byref(gz), ctypes.byref(h), 1,
                                  None, None) == gps.GPS_ERR_INVALID_ARG
    assert L.render_backward_adam(ctypes.byref(gz), v, 1, ctypes.byref(s), fake, 1 << 30, None,
                                  ctypes.byref(gz), ctypes.byref(gz), ctypes.byref(h), 1, None,
                                  None) == gps.GPS_ERR_INVALID_ARG  # no targets, no gradients
    assert L.render_backward_adam(ctypes.byref(gz), v9, 1, ctypes.byref(s), fake, 1 << 30, None,
                                  ctypes.byref(gz), ctypes.byref(gz), ctypes.byref(h), 0, None,
                                  None) == gps.GPS_ERR_INVALID_ARG  # step 0 without device_step
    assert b"device_step" in L.gps_last_error()


def test_layout_helpers_roundtrip():
    import torch
    a = torch.arange(16 * 8 * 24 * 3, dtype=torch.float32).reshape(16, 8, 24, 3)  # nz, ny, nx
    b = gps.linear_to_brick(a)
    assert b.shape == (16 * 8 * 24, 3)
    # voxel (x=9, y=3, z=10): brick (1, 0, 1), local (1, 3, 2)
    nbx, nby = 3, 1
    idx = ((1 * nby + 0) * nbx + 1) * 512 + 2 * 64 + 3 * 8 + 1
    assert torch.equal(b[idx], a[10, 3, 9])
    assert torch.equal(gps.brick_to_linear(b, 24, 8, 16), a)


def test_icp_arguments_are_checked_on_the_host(L):
    # sizes and settings are validated before anything touches the device
    with pytest.raises(gps.GpsError):
        gps.gps_icp_workspace_size(8, 8, gps.icp_settings(levels=3))     # level 2 is 2 x 2
    with pytest.raises(gps.GpsError):
        gps.gps_icp_workspace_size(64, 48, gps.icp_settings(levels=5))
    with pytest.raises(gps.GpsError):
        gps.gps_icp_workspace_size(64, 48, gps.icp_settings(eps_d=0.0))
    with pytest.raises(gps.GpsError):
        gps.gps_icp_workspace_size(64, 48, gps.icp_settings(iters=(3, -1, 2)))
    n1 = gps.gps_icp_workspace_size(64, 48, gps.icp_settings(levels=1))
    n3 = gps.gps_icp_workspace_size(64, 48, gps.icp_settings())
    assert 0 < n1 < n3 and n3 % 256 == 0


def test_hashed_volume_arguments_are_checked_on_the_host(L):
    import ctypes as C
    fake = C.c_void_p(256)     # never dereferenced: validation fails before any launch
    h = gps.GpsHashTsdf(64, 64, 64, 0.02, (C.c_float * 3)(0, 0, 0), 0.06, 100.0, 1024, 256,
                        fake, fake, fake, fake, fake, fake, fake)
    K = gps.GpsIntrinsics(100.0, 100.0, 50.0, 40.0, 100, 80)
    P = gps.GpsPose((C.c_float * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1), (C.c_float * 3)(0, 0, 0))
    n = gps.gps_hash_scratch_size(1000)
    for field, bad in (("nx", 60), ("n_buckets", 1000), ("capacity", 0), ("voxel", 0.0)):
        hb = gps.GpsHashTsdf.from_buffer_copy(h)
        setattr(hb, field, bad)
        assert L.fuse_frame_hashed(C.byref(hb), fake, fake, C.byref(K), C.byref(P), fake, n,
                                   1000, None) == gps.GPS_ERR_INVALID_ARG, field
    assert L.fuse_frame_hashed(C.byref(h), fake, fake, C.byref(K), C.byref(P), fake, n - 1,
                               1000, None) == gps.GPS_ERR_WORKSPACE_TOO_SMALL
    with pytest.raises(gps.GpsError):
        gps.gps_hash_scratch_size(0)
