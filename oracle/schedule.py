"""Keyframe selection and optimisation-view sampling (Sec. 3.2 "Gaussian
optimization", Fig. 5, App. C) in plain Python - TEST INFRASTRUCTURE ONLY,
like the rest of `oracle/`.

Keyframes.  Frame k becomes a keyframe when there is no keyframe yet, or when
its pose relative to the last keyframe, T_last^-1 T_k, rotates by more than
delta_angle (30 degrees, App. C) or translates by more than delta_move (0.3 m).

Views of one Gaussian optimisation.  Optimisations run every delta_k frames;
the e-th (e = 0, 1, ...) is taken at frame k.  Its views are
  - local: n_local frames spread evenly over the L = min(delta_k, k + 1)
    frames of the interval (k - delta_k, k], newest first,
    k - floor(j L / n) for j = 0 .. n - 1 with n = min(n_local, L);
  - global: n_global keyframes drawn uniformly without replacement from the
    keyframes before the interval (frame id <= k - delta_k), in draw order.

Readings of points the paper leaves open (listed with the other readings):
- The first frame is a keyframe; both motion tests are strict.
- The rotation angle is that of the relative rotation R_last^T R_k, from its
  trace; the translation is the length of R_last^T (t_k - t_last), i.e. the
  distance between the two camera centres.
- "Evenly select" is the floor spacing above; "keyframe history" excludes the
  keyframes inside the current interval, which are local frames already.
- n_global and n_local are not given; the defaults are 4 and 4, eight views,
  the most one render call takes.
- The draw is a partial Fisher-Yates shuffle of the history (ascending ids):
  step i swaps position i with position i + floor(hi32(r_i) * (H - i) / 2^32),
  r_i the (1024 e + i + 1)-th output of SplitMix64 seeded with `seed` (the
  generator of oracle/edit.py), H the history length.  This maps 32 random
  bits onto a range by multiplication (Lemire 2019), so each position's
  chance is exact to 2^-32 relative.
"""
from __future__ import annotations

import math

import numpy as np

from .edit import splitmix64


def rotation_angle_deg(R_a, R_b) -> float:
    """Angle of the rotation R_a^T R_b, degrees (plain arccos of the trace)."""
    R = np.asarray(R_a, np.float64).reshape(3, 3).T @ np.asarray(R_b, np.float64).reshape(3, 3)
    c = (np.trace(R) - 1.0) / 2.0
    return math.degrees(math.acos(min(1.0, max(-1.0, c))))


def is_keyframe(last, cur, delta_angle_deg=30.0, delta_move=0.3) -> bool:
    """last, cur: (R [3][3] camera -> world, t [3]) or last None."""
    if last is None:
        return True
    R_l, t_l = last
    R_c, t_c = cur
    rel_t = np.asarray(R_l, np.float64).reshape(3, 3).T @ (np.asarray(t_c, np.float64)
                                                          - np.asarray(t_l, np.float64))
    return bool(rotation_angle_deg(R_l, R_c) > delta_angle_deg or
                np.linalg.norm(rel_t) > delta_move)


def local_frames(frame: int, interval: int, n_local: int) -> list:
    L = min(interval, frame + 1)
    n = min(n_local, L)
    return [frame - (j * L) // n for j in range(n)]


def global_keyframes(keyframes, frame: int, event: int, interval: int, n_global: int,
                     seed: int) -> list:
    hist = [int(f) for f in keyframes if f <= frame - interval]
    H = len(hist)
    n = min(n_global, H)
    for i in range(n):
        r = int(splitmix64(seed, np.array([1024 * event + i + 1], np.uint64))[0])
        j = i + (((r >> 32) * (H - i)) >> 32)
        hist[i], hist[j] = hist[j], hist[i]
    return hist[:n]


def select_views(keyframes, frame: int, event: int, interval=10, n_global=4, n_local=4,
                 seed=0) -> list:
    """Local frames (newest first) followed by the global keyframes drawn."""
    return local_frames(frame, interval, n_local) + \
        global_keyframes(keyframes, frame, event, interval, n_global, seed)
