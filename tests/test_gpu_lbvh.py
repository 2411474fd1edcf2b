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


# ---- the traversal tree (PLOC collapsed to 4-wide nodes) ---------------------------

EMPTY = np.int32(-2 ** 31)
# The traversal stack holds 128 entries and a descent pushes at most three per
# 4-wide level above the deepest one (whose children are all leaves), so the
# tree may have 1 + 128 // 3 = 43 levels.
MAX_DEPTH = 1 + 128 // 3


def check_tree4(nodes, leaves, tris):
    """Invariants of the exported traversal tree, checked level by level from
    the root: every node is reached exactly once and every leaf exactly once
    (a tree over all triangles); each node has 2-4 children, internal ones
    first (consecutive nodes, slot keys 0, 1, ...), then leaves, unused slots
    last; every child box is the exact FP32 union of its subtree's vertices
    (a leaf's box is its triangle's min/max, a node's box the min/max of its
    own children's boxes); leaves hold their triangle's vertices; the depth
    stays within what the traversal stack holds.  Returns the depth."""
    n = len(tris)
    n4 = len(nodes)
    v = leaves.reshape(n, 3, 4)[:, :, :3]
    ids = leaves[:, 3].copy().view(np.int32)
    assert np.array_equal(np.sort(ids), np.arange(n)), "leaves are not a permutation of the triangles"
    # vertices: the triangle's own, in lexicographic order
    src = tris[ids].astype(np.float32)
    order = np.lexsort((src[:, :, 2], src[:, :, 1], src[:, :, 0]), axis=1)
    assert np.array_equal(np.take_along_axis(src, order[:, :, None], 1), v)
    leaf_lo, leaf_hi = v.min(1), v.max(1)
    refs = nodes[:, 24:28].copy().view(np.int32)
    keys = nodes[:, 28:32].copy().view(np.uint32)
    lo = np.stack([nodes[:, 0:4], nodes[:, 8:12], nodes[:, 16:20]], -1)
    hi = np.stack([nodes[:, 4:8], nodes[:, 12:16], nodes[:, 20:24]], -1)
    used = refs != EMPTY
    assert np.all(used[:, :2]), "a node with fewer than two children"
    assert np.all(used[:, 1:] <= used[:, :-1]), "unused slots must come last"
    node_ref = used & (refs >= 0)
    leaf_ref = used & (refs < 0)
    assert np.all(refs[node_ref] < n4) and np.all(~refs[leaf_ref] < n)
    # internal children first, consecutive nodes, each slot's key its slot
    # number (all ones for leaves and unused slots)
    assert np.all(node_ref[:, 1:] <= node_ref[:, :-1]), "a leaf or unused slot before an internal child"
    slot = np.arange(4)
    assert np.all(~node_ref | (refs == refs[:, :1] + slot)), "internal children are not consecutive nodes"
    assert np.array_equal(keys, np.where(node_ref, slot, 0xFFFFFFFF).astype(np.uint32)), "slot keys"
    # boxes: leaf children
    lk = ~refs[leaf_ref]
    assert np.array_equal(lo[leaf_ref], leaf_lo[lk]) and np.array_equal(hi[leaf_ref], leaf_hi[lk])
    # node children: the union of that node's own child boxes
    big = np.float32(np.inf)
    ulo = np.where(used[:, :, None], lo, big).min(1)
    uhi = np.where(used[:, :, None], hi, -big).max(1)
    nk = refs[node_ref]
    assert np.array_equal(lo[node_ref], ulo[nk]) and np.array_equal(hi[node_ref], uhi[nk])
    # reachability, level by level
    seen_n = np.zeros(n4, np.int64)
    seen_l = np.zeros(n, np.int64)
    frontier = np.array([0])
    depth = 0
    while frontier.size:
        depth += 1
        assert depth <= MAX_DEPTH, "tree deeper than the traversal stack allows"
        np.add.at(seen_n, frontier, 1)
        r = refs[frontier]
        np.add.at(seen_l, ~r[(r != EMPTY) & (r < 0)], 1)
        frontier = r[(r != EMPTY) & (r >= 0)]
    assert np.all(seen_n == 1), "a node is unreachable or shared"
    assert np.all(seen_l == 1), "a leaf is unreachable or shared"
    return depth


@pytest.mark.parametrize("make", ["random70001", "duplicates", "terrain4k", "objects8k", "tiny-stack"])
def test_traversal_tree_invariants(V, torch_mod, make):
    from workloads import workload
    if make == "random70001":
        sc = random_triangles_scene(70001, seed=5)
    elif make == "duplicates":
        rng = np.random.default_rng(3)
        pts = (rng.integers(0, 4, size=(3000, 3)) * 0.25).astype(np.float32)
        sc = random_triangles_scene(3000, seed=9)
        sc.tris[:] = pts[:, None, :]
    elif make == "tiny-stack":
        sc = tiny_scene("stack")
    else:
        sc = workload(make, frames=1).scene
    h, keep = device_scene(V, sc, torch_mod)
    try:
        nodes, leaves = V.vafr_scene_export_tree4(h)
        depth = check_tree4(nodes, leaves, sc.tris.reshape(-1, 3, 3))
        print(f"{make}: {sc.n_tris} triangles, {len(nodes)} 4-wide nodes, depth {depth}")
    finally:
        V.vafr_scene_destroy(h)
