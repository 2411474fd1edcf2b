"""The host-side checker of the exported traversal tree (check_tree4) accepts a
hand-built valid tree and rejects each planted fault: a box one ulp too small,
a leaf referenced twice, a leaf missing, a node with one child, an unused slot
before a used one, and a leaf whose vertices are not its triangle's."""

import numpy as np
import pytest

from test_gpu_lbvh import EMPTY, check_tree4


def _tree():
    rng = np.random.default_rng(5)
    tris = rng.uniform(-1, 1, (6, 3, 3)).astype(np.float32)
    # leaves in the order 3, 0, 5, 1, 4, 2; vertices lexicographically sorted
    ids = np.array([3, 0, 5, 1, 4, 2])
    leaves = np.zeros((6, 12), np.float32)
    for k, i in enumerate(ids):
        t = tris[i][np.lexsort((tris[i][:, 2], tris[i][:, 1], tris[i][:, 0]))]
        leaves[k].reshape(3, 4)[:, :3] = t
    leaves[:, 3] = ids.astype(np.int32).view(np.float32)
    lo_l = leaves.reshape(6, 3, 4)[:, :, :3].min(1)
    hi_l = leaves.reshape(6, 3, 4)[:, :, :3].max(1)
    # root: leaves 0, 1 and node 1; node 1: leaves 2..5
    nodes = np.zeros((2, 32), np.float32)
    refs = np.full((2, 4), EMPTY, np.int32)
    refs[0, :3] = [~0, ~1, 1]
    refs[1, :4] = [~2, ~3, ~4, ~5]

    def put(node, slot, lo, hi):
        for a in range(3):
            nodes[node, 8 * a + slot] = lo[a]
            nodes[node, 8 * a + 4 + slot] = hi[a]
    for s in range(4):
        put(1, s, lo_l[2 + s], hi_l[2 + s])
    put(0, 0, lo_l[0], hi_l[0])
    put(0, 1, lo_l[1], hi_l[1])
    put(0, 2, lo_l[2:].min(0), hi_l[2:].max(0))
    nodes[:, 24:28] = refs.view(np.float32)
    return nodes, leaves, tris


def _refs(nodes):
    return nodes[:, 24:28].view(np.int32)


def test_valid_tree_passes():
    nodes, leaves, tris = _tree()
    assert check_tree4(nodes, leaves, tris) == 2


@pytest.mark.parametrize("fault", ["box", "dup-leaf", "one-child", "gap", "vertex", "parent-box"])
def test_planted_fault_is_rejected(fault):
    nodes, leaves, tris = _tree()
    if fault == "box":                 # a leaf box one ulp too small
        nodes[1, 0] = np.nextafter(nodes[1, 0], np.float32(np.inf))
    elif fault == "parent-box":        # a node's box one ulp too large
        nodes[0, 4 + 2] = np.nextafter(nodes[0, 4 + 2], np.float32(np.inf))
    elif fault == "dup-leaf":          # leaf 5 replaced by a second reference to leaf 4
        _refs(nodes)[1, 3] = ~4
    elif fault == "one-child":
        _refs(nodes)[1, 1:] = EMPTY
    elif fault == "gap":               # unused slot before a used one
        r = _refs(nodes)
        r[0, 1], r[0, 3] = EMPTY, ~1
    elif fault == "vertex":
        leaves[2, 0] += 1e-3
    with pytest.raises(AssertionError):
        check_tree4(nodes, leaves, tris)
