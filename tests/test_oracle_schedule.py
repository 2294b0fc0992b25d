"""Pins of the keyframe / view-sampling oracle (oracle/schedule.py) against
hand values, rotations built by scipy and the statistics a uniform draw
without replacement must have."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import schedule


def _pose(rot: Rotation, t):
    return rot.as_matrix(), np.asarray(t, np.float64)


def test_first_frame_is_a_keyframe():
    assert schedule.is_keyframe(None, _pose(Rotation.identity(), [0, 0, 0]))


def test_rotation_threshold_relative_to_the_last_keyframe():
    rng = np.random.default_rng(0)
    for _ in range(20):
        base = Rotation.random(random_state=rng)
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        last = _pose(base, rng.normal(size=3))
        for deg, want in ((29.9, False), (30.1, True), (5.0, False), (170.0, True)):
            # rotate in the camera frame of the last keyframe; same centre
            cur = _pose(base * Rotation.from_rotvec(np.radians(deg) * axis), last[1])
            assert schedule.is_keyframe(last, cur) == want, (deg, axis)
        assert abs(schedule.rotation_angle_deg(
            base.as_matrix(), (base * Rotation.from_rotvec(0.4 * axis)).as_matrix())
            - np.degrees(0.4)) < 1e-9


def test_translation_threshold():
    rng = np.random.default_rng(1)
    for _ in range(20):
        base = Rotation.random(random_state=rng)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        last = _pose(base, rng.normal(size=3))
        for dist, want in ((0.299, False), (0.301, True)):
            assert schedule.is_keyframe(last, _pose(base, last[1] + dist * d)) == want
        # a custom threshold
        assert not schedule.is_keyframe(last, _pose(base, last[1] + 0.5 * d), delta_move=0.6)


def test_local_frames_by_hand():
    # interval 10, four views: 10 frames split at floor(j * 10 / 4) = 0, 2, 5, 7
    assert schedule.local_frames(9, 10, 4) == [9, 7, 4, 2]
    assert schedule.local_frames(29, 10, 4) == [29, 27, 24, 22]
    assert schedule.local_frames(2, 10, 4) == [2, 1, 0]       # only three frames exist
    assert schedule.local_frames(19, 10, 1) == [19]
    assert schedule.local_frames(19, 10, 20) == list(range(19, 9, -1))
    assert schedule.local_frames(15, 5, 2) == [15, 13]


def test_global_draw_hand_value():
    # the first output of SplitMix64(0) is 0xE220A8397B1DCDAF: its high 32 bits
    # 3793791033 * 10 / 2^32 = 8.83, so from ten keyframes the first draw is the
    # ninth (index 8)
    kf = list(range(0, 100, 10))          # ten keyframes, all before the interval
    got = schedule.global_keyframes(kf, frame=200, event=0, interval=10, n_global=1, seed=0)
    assert got == [80]


def test_global_draw_history_and_no_repeats():
    kf = [0, 3, 9, 12, 18, 25, 31]
    # frame 30, interval 10: history = ids <= 20
    for e in range(50):
        g = schedule.global_keyframes(kf, frame=30, event=e, interval=10, n_global=4, seed=7)
        assert len(g) == 4 and len(set(g)) == 4 and set(g) <= {0, 3, 9, 12, 18}
    assert sorted(schedule.global_keyframes(kf, 30, 0, 10, 10, 7)) == [0, 3, 9, 12, 18]
    assert schedule.global_keyframes(kf, 9, 0, 10, 4, 7) == []     # no history yet
    v = schedule.select_views(kf, 30, 3, 10, 4, 4, 7)
    assert v[:4] == [30, 28, 25, 23] and len(v) == 8


def test_global_draw_is_uniform_without_replacement():
    H, n, E = 20, 4, 20000
    kf = list(range(H))
    hits = np.zeros(H)
    first = np.zeros(H)
    pair = 0
    for e in range(E):
        g = schedule.global_keyframes(kf, frame=1000, event=e, interval=10, n_global=n, seed=3)
        hits[g] += 1
        first[g[0]] += 1
        pair += (2 in g) and (11 in g)
    # each keyframe: n / H = 0.2; the first draw: 1 / H; a given pair: n(n-1)/(H(H-1))
    p = hits / E
    assert np.all(np.abs(p - n / H) < 5 * np.sqrt(0.2 * 0.8 / E))
    q = first / E
    assert np.all(np.abs(q - 1 / H) < 5 * np.sqrt(0.05 * 0.95 / E))
    pp = n * (n - 1) / (H * (H - 1))
    assert abs(pair / E - pp) < 5 * np.sqrt(pp * (1 - pp) / E)
