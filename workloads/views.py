"""Camera poses and display descriptions (inputs only).

A pose is a row-major 3x4 float64 matrix [R | t] taking camera coordinates
(x right, y up, z forward) to world coordinates; ``t`` is the eye position.
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class View:
    width: int
    height: int
    fov_v_deg: float
    pose: np.ndarray  # (3, 4) float64


def look_at_pose(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(np.asarray(up, np.float64), fwd)
    right /= np.linalg.norm(right)
    upv = np.cross(fwd, right)
    P = np.zeros((3, 4))
    P[:, 0], P[:, 1], P[:, 2], P[:, 3] = right, upv, fwd, eye
    return P


def eye_pair_poses(pose: np.ndarray, ipd_m: float):
    """Left / right eye poses: the head pose shifted by -/+ ipd/2 along its right axis."""
    left, right = pose.copy(), pose.copy()
    left[:, 3] -= pose[:, 0] * ipd_m / 2
    right[:, 3] += pose[:, 0] * ipd_m / 2
    return left, right
