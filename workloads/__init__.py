"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This package only *generates inputs*: triangle soups, per-triangle albedo,
camera poses, light directions and gaze trajectories.  It holds none of the
foveation method's arithmetic (no acuity model, no log-polar mapping, no ray
casting, no shading, no reconstruction), so both sides can take their inputs
from it without sharing any of the computation under test.

Everything is deterministic given the seed (numpy's PCG64 generator).
"""

from .scenes import (  # noqa: F401
    Scene,
    random_triangles_scene,
    terrain_boxes_scene,
    terrain_objects_scene,
    tiny_scene,
)
from .views import View, look_at_pose, eye_pair_poses  # noqa: F401
from .gaze import saccade_trajectory, random_walk_trajectory  # noqa: F401
from .configs import Workload, workload, WORKLOADS  # noqa: F401
