"""Pins of the insertion / removal oracle (oracle/edit.py) against values fixed
by the paper's definitions, published generator outputs and geometry."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import edit


def test_splitmix64_reference_outputs():
    # first three outputs of SplitMix64 seeded with 0 (the seeding generator of
    # the xoshiro family; Steele, Lea and Flood 2014)
    z = edit.splitmix64(0, np.arange(1, 4, dtype=np.uint64))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_sampling_keeps_a_quarter_uniformly():
    mask = np.ones((1000, 1000), bool)
    a = edit.sampled_pixels(mask, seed=7)
    assert abs(len(a) / mask.size - 0.25) < 0.003
    # uniform over the image: each quadrant keeps a quarter of its pixels
    y, x = np.divmod(a, 1000)
    for qy in (0, 1):
        for qx in (0, 1):
            n = np.sum((y // 500 == qy) & (x // 500 == qx))
            assert abs(n / 250000 - 0.25) < 0.005
    b = edit.sampled_pixels(mask, seed=8)
    assert 0.2 < len(np.intersect1d(a, b)) / len(a) < 0.3  # another seed: an independent draw
    half = mask.copy()
    half[:, 500:] = False
    c = edit.sampled_pixels(half, seed=7)
    np.testing.assert_array_equal(c, a[a % 1000 < 500])  # draws do not depend on the mask


def test_mask_thresholds():
    H, W = 2, 4
    C_k = np.zeros((3, H, W), np.float32)
    C_star = np.zeros((3, H, W), np.float32)
    C_star[:, 0, 0] = 0.06          # mean error 0.06 > 0.05
    C_star[:, 0, 1] = 0.04          # 0.04: no
    C_star[0, 0, 2] = 0.2           # mean 0.0667: yes
    C_star[:, 0, 3] = 0.06          # but weight 4: no (strict)
    C_star[:, 1, 0] = 0.06          # but no ray-cast hit
    W_G = np.zeros((H, W), np.float32)
    W_G[0, 3] = 4.0
    D_t = np.ones((H, W), np.float32)
    D_t[1, 0] = 0.0
    m = edit.insertion_mask(C_star, W_G, C_k, D_t)
    assert m.tolist() == [[True, False, True, False], [False, False, False, False]]


def _plane(H, W, f, depth_fn):
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    rx, ry = (xs - W / 2) / f, (ys - H / 2) / f
    z = depth_fn(rx, ry)
    return np.stack([rx * z, ry * z, z], -1), z


def test_insert_on_a_fronto_parallel_plane():
    H, W, f = 20, 30, 100.0
    V, z = _plane(H, W, f, lambda rx, ry: np.full_like(rx, 2.0))
    D_t = z.astype(np.float32)
    C_k = np.random.default_rng(0).uniform(0, 1, (3, H, W)).astype(np.float32)
    C_star = C_k + 0.1
    W_G = np.zeros((H, W), np.float32)
    new, pix, mask = edit.insert(V, D_t, C_star, W_G, C_k, f, np.zeros(3), seed=3, M=0,
                                 capacity=10 ** 6)
    assert mask.all() and len(pix) > 0
    y, x = np.divmod(pix, W)
    np.testing.assert_allclose(new["means"], V[y, x])
    np.testing.assert_allclose(new["rgb"], C_k[:, y, x].T)
    assert np.all(new["opacity_logits"] == 0.0)
    # nearest mask vertices: 4-neighbours, 2 / 100 m apart -> s1 = 0.02; a corner
    # pixel has two, its third nearest is diagonal: sqrt((1 + 1 + 2) / 3) * 0.02
    corner = ((y == 0) | (y == H - 1)) & ((x == 0) | (x == W - 1))
    s1 = np.where(corner, 0.02 * np.sqrt(4.0 / 3.0), 0.02)
    np.testing.assert_allclose(new["log_scales"], np.log(np.stack([s1, s1, 0.1 * s1], 1)),
                               rtol=1e-12)
    # the plane faces the camera: the short axis lies on the z line (either sign
    # is the same disc)
    for q in new["quats"]:
        n = Rotation.from_quat([q[1], q[2], q[3], q[0]]).apply([0.0, 0.0, 1.0])
        np.testing.assert_allclose(np.abs(n), [0.0, 0.0, 1.0], atol=1e-12)


def test_insert_on_a_tilted_plane_orients_the_disc_along_the_normal():
    H, W, f = 24, 24, 120.0
    # plane z = 2 + 0.5 x (world), through the camera rays: z = 2 / (1 - 0.5 rx)
    V, z = _plane(H, W, f, lambda rx, ry: 2.0 / (1.0 - 0.5 * rx))
    n_true = np.array([0.5, 0.0, -1.0]) / np.sqrt(1.25)  # facing the camera at the origin
    D_t = z.astype(np.float32)
    C_k = np.zeros((3, H, W), np.float32)
    C_star = np.full((3, H, W), 0.5, np.float32)
    W_G = np.zeros((H, W), np.float32)
    new, pix, _ = edit.insert(V, D_t, C_star, W_G, C_k, f, np.zeros(3), seed=1, M=0,
                              capacity=10 ** 6)
    for q in new["quats"]:
        n = Rotation.from_quat([q[1], q[2], q[3], q[0]]).apply([0.0, 0.0, 1.0])
        np.testing.assert_allclose(n * np.sign(n @ n_true), n_true, atol=1e-9)
        assert n[2] >= 0  # the sign with non-negative z
    # the short scale is a tenth of the long ones
    np.testing.assert_allclose(new["log_scales"][:, 2] - new["log_scales"][:, 0], np.log(0.1))


def test_insert_respects_capacity_and_appends_in_pixel_order():
    H, W, f = 16, 16, 100.0
    V, z = _plane(H, W, f, lambda rx, ry: np.full_like(rx, 1.0))
    D_t = z.astype(np.float32)
    C_k = np.zeros((3, H, W), np.float32)
    C_star = np.ones((3, H, W), np.float32)
    W_G = np.zeros((H, W), np.float32)
    full, pix, _ = edit.insert(V, D_t, C_star, W_G, C_k, f, np.zeros(3), seed=5, M=0,
                               capacity=10 ** 6)
    part, pix2, _ = edit.insert(V, D_t, C_star, W_G, C_k, f, np.zeros(3), seed=5, M=90,
                                capacity=100)
    assert len(pix2) == 10 and np.array_equal(pix2, pix[:10]) and np.all(np.diff(pix) > 0)
    np.testing.assert_array_equal(part["means"], full["means"][:10])


def test_isolated_pixel_uses_its_footprint_and_the_scale_cap():
    H, W, f = 9, 9, 50.0
    V, z = _plane(H, W, f, lambda rx, ry: np.full_like(rx, 3.0))
    D_t = np.zeros((H, W), np.float32)
    D_t[4, 4] = 3.0                   # one hit only: no neighbour in the mask
    C_k = np.zeros((3, H, W), np.float32)
    C_star = np.ones((3, H, W), np.float32)
    W_G = np.zeros((H, W), np.float32)
    for seed in range(64):            # some seed samples the pixel
        new, pix, _ = edit.insert(V, D_t, C_star, W_G, C_k, f, np.zeros(3), seed=seed, M=0,
                                  capacity=10)
        if len(pix):
            break
    assert list(pix) == [4 * W + 4]
    np.testing.assert_allclose(np.exp(new["log_scales"][0, 0]), min(0.1, 3.0 / 50.0))
    # no neighbour on either axis: the disc's short axis lies along the viewing ray
    q = new["quats"][0]
    n = Rotation.from_quat([q[1], q[2], q[3], q[0]]).apply([0.0, 0.0, 1.0])
    ray = V[4, 4] / np.linalg.norm(V[4, 4])
    np.testing.assert_allclose(n * np.sign(n @ ray), ray, atol=1e-12)


def test_removal_criteria():
    logit = lambda s: np.log(s / (1 - s))
    ls = np.log(np.array([[0.01, 0.01, 0.001],    # keep
                          [0.2, 0.01, 0.01],      # largest scale 0.2 > 0.1: remove
                          [0.002, 0.001, 0.001],  # largest 0.002 < 0.003: remove
                          [0.05, 0.004, 0.004],   # keep
                          [0.01, 0.01, 0.01]]))   # but opacity below 0.005: remove
    lg = np.array([logit(0.5), logit(0.5), logit(0.5), logit(0.006), logit(0.004)])
    assert edit.removal_keep(ls, lg).tolist() == [True, False, False, True, False]
