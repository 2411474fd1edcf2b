"""The five synthetic workloads (inputs only): display sizes, views, scenes, gaze.

1. ``random1k``   : 512x512 mono, 90 deg FOV, gaze at the centre, 1,024 random
                    triangles, camera at z=-3 looking +z; FP32 LP and display.
2. ``terrain4k``  : 3840x2160 mono, 100 deg FOV, 240-frame saccade trajectory,
                    1,069,506-triangle terrain + 2,000 boxes; FP32 LP.
3. ``objects8k``  : 7680x4320 per eye, binocular (63 mm IPD), 240-frame per-eye
                    trajectories, 1,998,088-triangle terrain + 4,000 spheres +
                    4,000 boxes; FP16 LP, FP32 accumulation.
4. ``sweep``      : the terrain4k scene, binocular, per-eye 1080p / 1440p / 4K /
                    8K / 16K displays batched together.
5. ``serving``    : 64 Poisson-arriving binocular sessions on the terrain4k
                    scene, resolutions uniform over {1080p, 1440p, 4K, 8K},
                    per-session random-walk gaze.
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from .gaze import random_walk_trajectory, saccade_trajectory
from .scenes import (Scene, random_triangles_scene, terrain_boxes_scene,
                     terrain_objects_scene)
from .views import eye_pair_poses, look_at_pose

RESOLUTIONS = {
    "1080p": (1920, 1080), "1440p": (2560, 1440), "4k": (3840, 2160),
    "8k": (7680, 4320), "16k": (15360, 8640),
}


@dataclasses.dataclass
class Display:
    width: int
    height: int
    fov_v_deg: float
    poses: List[np.ndarray]          # one (3, 4) pose per eye
    gaze: np.ndarray                 # (frames, eyes, 2) pixel positions


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    displays: List[Display]
    lp_fp16: bool = False
    display_fp16: bool = False
    frames: int = 1
    poisson_rate_hz: Optional[float] = None
    hbm_budget_bytes: Optional[int] = None


def _terrain_camera(scene: Scene, height_above: float = 10.0):
    ex, ez = scene.extent
    h = scene.heights
    nz, nx = h.shape
    z0 = -ez / 2 + 20.0
    iz = int(round((z0 + ez / 2) / ez * (nz - 1)))
    ground = float(h[iz, nx // 2])
    eye = (0.0, ground + height_above, z0)
    target = (0.0, ground, z0 + 60.0)
    return look_at_pose(eye, target)


_SCENE_CACHE = {}


def _cached(key, fn):
    if key not in _SCENE_CACHE:
        _SCENE_CACHE[key] = fn()
    return _SCENE_CACHE[key]


def workload(name: str, frames: Optional[int] = None, seed_offset: int = 0,
             small_scene: bool = False) -> Workload:
    """Build a workload by name.  ``small_scene`` swaps in a reduced terrain of the
    same structure (for quick tests); the full sizes are the default."""
    if name == "random1k":
        sc = random_triangles_scene(1024, seed=1001 + seed_offset)
        pose = look_at_pose((0.0, 0.0, -3.0), (0.0, 0.0, 0.0))
        nf = frames or 1
        gaze = np.tile(np.array([[[256.0, 256.0]]]), (nf, 1, 1))
        return Workload(name, sc, [Display(512, 512, 90.0, [pose], gaze)], frames=nf)
    if name == "terrain4k":
        if small_scene:
            sc = _cached(("tb-small", seed_offset),
                         lambda: terrain_boxes_scene(128, 256, 200, seed=1002 + seed_offset))
        else:
            sc = _cached(("tb", seed_offset),
                         lambda: terrain_boxes_scene(seed=1002 + seed_offset))
        nf = frames or 240
        W, H, fov = 3840, 2160, 100.0
        g = saccade_trajectory(nf, W, H, fov, seed=2002 + seed_offset)
        return Workload(name, sc, [Display(W, H, fov, [_terrain_camera(sc)], g[:, None, :])],
                        frames=nf)
    if name == "objects8k":
        if small_scene:
            sc = _cached(("to-small", seed_offset),
                         lambda: terrain_objects_scene(160, 200, 200, 200, seed=1003 + seed_offset))
        else:
            sc = _cached(("to", seed_offset),
                         lambda: terrain_objects_scene(seed=1003 + seed_offset))
        nf = frames or 240
        W, H, fov = 7680, 4320, 100.0
        left, right = eye_pair_poses(_terrain_camera(sc), 0.063)
        gl = saccade_trajectory(nf, W, H, fov, seed=3002 + seed_offset)
        gr = saccade_trajectory(nf, W, H, fov, seed=3003 + seed_offset)
        return Workload(name, sc, [Display(W, H, fov, [left, right], np.stack([gl, gr], 1))],
                        lp_fp16=True, display_fp16=True, frames=nf)
    if name == "sweep":
        base = workload("terrain4k", frames=1, seed_offset=seed_offset, small_scene=small_scene)
        sc = base.scene
        nf = frames or 1
        left, right = eye_pair_poses(_terrain_camera(sc), 0.063)
        disps = []
        for k, res in enumerate(["1080p", "1440p", "4k", "8k", "16k"]):
            W, H = RESOLUTIONS[res]
            gl = saccade_trajectory(nf, W, H, 100.0, seed=4000 + 2 * k + seed_offset)
            gr = saccade_trajectory(nf, W, H, 100.0, seed=4001 + 2 * k + seed_offset)
            disps.append(Display(W, H, 100.0, [left, right], np.stack([gl, gr], 1)))
        return Workload(name, sc, disps, lp_fp16=True, display_fp16=True, frames=nf)
    if name == "serving":
        base = workload("terrain4k", frames=1, seed_offset=seed_offset, small_scene=small_scene)
        sc = base.scene
        nf = frames or 60
        rng = np.random.default_rng(5000 + seed_offset)
        left, right = eye_pair_poses(_terrain_camera(sc), 0.063)
        disps = []
        names = ["1080p", "1440p", "4k", "8k"]
        for s in range(64):
            W, H = RESOLUTIONS[names[int(rng.integers(0, 4))]]
            gl = random_walk_trajectory(nf, W, H, 100.0, seed=6000 + 2 * s + seed_offset)
            gr = random_walk_trajectory(nf, W, H, 100.0, seed=6001 + 2 * s + seed_offset)
            disps.append(Display(W, H, 100.0, [left, right], np.stack([gl, gr], 1)))
        return Workload(name, sc, disps, lp_fp16=True, display_fp16=True, frames=nf,
                        poisson_rate_hz=64 * 90.0 / nf, hbm_budget_bytes=8 << 30)
    raise ValueError(f"unknown workload {name!r}")


WORKLOADS = ("random1k", "terrain4k", "objects8k", "sweep", "serving")
