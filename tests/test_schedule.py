"""The library's keyframe test and view selection (host-only C-ABI calls, no
GPU needed) against the oracle: identical decisions and identical frame ids
on random poses, keyframe lists and optimisation events."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import paper_2509_11574_b300 as gps
from paper_2509_11574_b300 import build as gbuild
from oracle import schedule as osched


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gbuild.build()
    gps.lib()


class _Cam:
    def __init__(self, R, t):
        self.R = np.asarray(R, np.float32).reshape(9)
        self.t = np.asarray(t, np.float32)


def _f32(R, t):
    return np.asarray(R, np.float32).astype(np.float64).reshape(3, 3), \
        np.asarray(t, np.float32).astype(np.float64)


def test_keyframe_decisions_match_the_oracle():
    rng = np.random.default_rng(0)
    n_kf = 0
    for i in range(400):
        base = Rotation.random(random_state=rng)
        t0 = rng.normal(size=3)
        deg = rng.uniform(0, 60)
        step = Rotation.from_rotvec(np.radians(deg) * Rotation.random(random_state=rng).apply([0, 0, 1]))
        t1 = t0 + rng.normal(size=3) * rng.uniform(0, 0.3)
        a, b = _Cam(base.as_matrix(), t0), _Cam((base * step).as_matrix(), t1)
        want = osched.is_keyframe(_f32(a.R, a.t), _f32(b.R, b.t))
        got = gps.gps_is_keyframe(a, b)
        # decisions that sit within 1e-6 of a threshold may legitimately differ
        near = abs(osched.rotation_angle_deg(_f32(a.R, a.t)[0], _f32(b.R, b.t)[0]) - 30) < 1e-6
        assert got == want or near
        n_kf += got
    assert 50 < n_kf < 350            # both outcomes well represented
    assert gps.gps_is_keyframe(None, _Cam(np.eye(3), [0, 0, 0]))
    s = gps.view_schedule(delta_angle_deg=10.0, delta_move=2.0)
    a = _Cam(np.eye(3), [0, 0, 0])
    b = _Cam(Rotation.from_euler("y", 11, degrees=True).as_matrix(), [0.2, 0, 0])
    assert gps.gps_is_keyframe(a, b, s) and not gps.gps_is_keyframe(a, b, gps.view_schedule())


@pytest.mark.parametrize("interval,n_global,n_local,seed", [(10, 4, 4, 0), (10, 4, 4, 12345),
                                                            (5, 3, 2, 7), (1, 8, 1, 99),
                                                            (10, 0, 8, 3), (20, 7, 0, 5)])
def test_select_views_matches_the_oracle(interval, n_global, n_local, seed):
    rng = np.random.default_rng(seed)
    kf = sorted(set(rng.integers(0, 300, size=40).tolist()))
    sched = gps.view_schedule(interval=interval, n_global=n_global, n_local=n_local, seed=seed)
    for event, frame in enumerate(range(interval - 1, 320, interval)):
        have = [k for k in kf if k <= frame]
        got = gps.gps_select_views(have, frame, event, sched)
        want = osched.select_views(have, frame, event, interval, n_global, n_local, seed)
        assert got == want, (frame, event)


def test_select_views_invalid_arguments():
    s = gps.view_schedule()
    for bad in ([3, 3], [5, 2], [-1, 4]):
        with pytest.raises(gps.GpsError) as e:
            gps.gps_select_views(bad, 30, 0, s)
        assert e.value.code == gps.GPS_ERR_INVALID_ARG
    with pytest.raises(gps.GpsError):
        gps.gps_select_views([0], -1, 0, s)
    with pytest.raises(gps.GpsError):
        gps.gps_select_views([0], 10, 0, gps.view_schedule(interval=0))
    with pytest.raises(gps.GpsError):
        gps.gps_select_views([0], 10, 0, gps.view_schedule(n_global=2000))
    assert gps.gps_select_views([], 0, 0, s) == [0]
