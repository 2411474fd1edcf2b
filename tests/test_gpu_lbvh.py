"""GPU LBVH build (Morton codes, stable radix sort, Karras hierarchy, bounds)
against the oracle's reference: bit-exact."""

import numpy as np
import pytest

import oracle
from parity import device_scene
from workloads import random_triangles_scene, terrain_boxes_scene, tiny_scene

pytestmark = pytest.mark.gpu


def _compare(V, torch_mod, scene):
    h, keep = device_scene(V, scene, torch_mod)
    try:
        codes, ids, child, nb, lb = V.vafr_scene_export_lbvh(h)
        ref = oracle.lbvh(scene.tris)
        assert np.array_equal(codes, ref.codes), "Morton codes differ"
        assert np.array_equal(ids, ref.sorted_ids), "sorted order differs"
        assert np.array_equal(child, ref.child), "topology differs"
        assert np.array_equal(nb.view(np.uint32), ref.node_box.view(np.uint32)), "node boxes differ"
        assert np.array_equal(lb.view(np.uint32), ref.leaf_box.view(np.uint32)), "leaf boxes differ"
    finally:
        V.vafr_scene_destroy(h)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (33, 3), (1024, 1001), (5000, 4),
                                    (70001, 5)])
def test_lbvh_random(V, torch_mod, n, seed):
    _compare(V, torch_mod, random_triangles_scene(n, seed=seed))


def test_lbvh_duplicate_centroids(V, torch_mod):
    rng = np.random.default_rng(3)
    pts = (rng.integers(0, 4, size=(3000, 3)) * 0.25).astype(np.float32)
    sc = random_triangles_scene(3000, seed=9)
    sc.tris[:] = pts[:, None, :]
    _compare(V, torch_mod, sc)


def test_lbvh_terrain_small(V, torch_mod):
    _compare(V, torch_mod, terrain_boxes_scene(96, 160, 150, seed=77))


@pytest.mark.parametrize("kind", ["single", "quad", "fan", "stack", "axis"])
def test_lbvh_tiny(V, torch_mod, kind):
    _compare(V, torch_mod, tiny_scene(kind))


def test_lbvh_empty(V, torch_mod):
    h, _ = device_scene(V, tiny_scene("empty"), torch_mod)
    assert V.vafr_scene_info(h)[0] == 0
    V.vafr_scene_destroy(h)
