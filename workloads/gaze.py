"""Seeded gaze trajectories in display pixel coordinates (inputs only).

Gaze is modelled as an angular direction (yaw, pitch) in degrees relative to
the view axis and converted to a pixel position with the pinhole projection
of the display (x right, y down, pixel centres at i + 0.5).

* ``saccade_trajectory``: fixations of U[200, 400] ms joined by saccades of
  uniform direction and amplitude U(0, max] degrees; saccade duration follows
  the main-sequence approximation 2.2 ms/deg + 21 ms (Carpenter 1988).
* ``random_walk_trajectory``: Gaussian random walk, sigma deg per frame.
"""

from __future__ import annotations

import math

import numpy as np


def _to_pixels(yaw_deg, pitch_deg, width, height, fov_v_deg):
    f_px = (height / 2.0) / math.tan(math.radians(fov_v_deg) / 2.0)
    x = width / 2.0 + np.tan(np.radians(yaw_deg)) * f_px
    y = height / 2.0 - np.tan(np.radians(pitch_deg)) * f_px
    return np.clip(x, 0.0, width), np.clip(y, 0.0, height)


def _angle_limits(width, height, fov_v_deg):
    f_px = (height / 2.0) / math.tan(math.radians(fov_v_deg) / 2.0)
    return (math.degrees(math.atan((width / 2.0) / f_px)),
            math.degrees(math.atan((height / 2.0) / f_px)))


def saccade_trajectory(n_frames: int, width: int, height: int, fov_v_deg: float,
                       seed: int, hz: float = 90.0, max_amp_deg: float = 20.0,
                       start=(0.0, 0.0)) -> np.ndarray:
    """(n_frames, 2) float64 gaze pixel positions."""
    rng = np.random.default_rng(seed)
    ylim, plim = _angle_limits(width, height, fov_v_deg)
    yaw, pitch = float(start[0]), float(start[1])
    t = 0.0
    events = []  # (t_start, t_end, from, to)
    horizon = n_frames / hz + 1.0
    while t < horizon:
        fix = rng.uniform(0.200, 0.400)
        events.append((t, t + fix, (yaw, pitch), (yaw, pitch)))
        t += fix
        amp = rng.uniform(0.0, max_amp_deg)
        if amp == 0.0:
            amp = max_amp_deg
        ang = rng.uniform(0.0, 2 * math.pi)
        ny = float(np.clip(yaw + amp * math.cos(ang), -ylim, ylim))
        npch = float(np.clip(pitch + amp * math.sin(ang), -plim, plim))
        dur = (2.2 * amp + 21.0) / 1000.0
        events.append((t, t + dur, (yaw, pitch), (ny, npch)))
        t += dur
        yaw, pitch = ny, npch
    out = np.zeros((n_frames, 2))
    k = 0
    for i in range(n_frames):
        ti = i / hz
        while events[k][1] <= ti:
            k += 1
        t0, t1, a, b = events[k]
        s = 0.0 if t1 == t0 else (ti - t0) / (t1 - t0)
        y_ = a[0] + (b[0] - a[0]) * s
        p_ = a[1] + (b[1] - a[1]) * s
        out[i] = _to_pixels(y_, p_, width, height, fov_v_deg)
    return out


def random_walk_trajectory(n_frames: int, width: int, height: int, fov_v_deg: float,
                           seed: int, sigma_deg: float = 2.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    ylim, plim = _angle_limits(width, height, fov_v_deg)
    steps = rng.normal(0.0, sigma_deg, size=(n_frames, 2))
    yaw = np.clip(np.cumsum(steps[:, 0]), -ylim, ylim)
    pitch = np.clip(np.cumsum(steps[:, 1]), -plim, plim)
    x, y = _to_pixels(yaw, pitch, width, height, fov_v_deg)
    return np.stack([x, y], 1)
