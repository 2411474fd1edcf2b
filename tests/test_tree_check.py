"""The host-side checker of the exported traversal tree (check_tree4) accepts a
hand-built valid tree and rejects each planted fault: a box one ulp too small,
a leaf referenced twice, a leaf missing, a node with one child, an unused slot
before a used one, a leaf whose vertices are not its triangle's, a leaf
before an internal child, internal children that are not consecutive nodes,
and a slot key that does not match its slot."""

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
    # root: nodes 1 and 2 (consecutive, first), then leaf 0; node 1: leaves
    # 1, 2; node 2: leaves 3, 4, 5
    nodes = np.zeros((3, 32), np.float32)
    refs = np.full((3, 4), EMPTY, np.int32)
    refs[0, :3] = [1, 2, ~0]
    refs[1, :2] = [~1, ~2]
    refs[2, :3] = [~3, ~4, ~5]
    keys = np.full((3, 4), 0xFFFFFFFF, np.uint32)
    keys[0, :2] = [0, 1]

    def put(node, slot, lo, hi):
        for a in range(3):
            nodes[node, 8 * a + slot] = lo[a]
            nodes[node, 8 * a + 4 + slot] = hi[a]
    put(1, 0, lo_l[1], hi_l[1])
    put(1, 1, lo_l[2], hi_l[2])
    for s in range(3):
        put(2, s, lo_l[3 + s], hi_l[3 + s])
    put(0, 0, lo_l[1:3].min(0), hi_l[1:3].max(0))
    put(0, 1, lo_l[3:].min(0), hi_l[3:].max(0))
    put(0, 2, lo_l[0], hi_l[0])
    nodes[:, 24:28] = refs.view(np.float32)
    nodes[:, 28:32] = keys.view(np.float32)
    return nodes, leaves, tris


def _refs(nodes):
    return nodes[:, 24:28].view(np.int32)


def test_valid_tree_passes():
    nodes, leaves, tris = _tree()
    assert check_tree4(nodes, leaves, tris) == 2


def test_slot_swap_keeps_keys_with_their_slots():
    nodes, leaves, tris = _tree()
    _swap_slots(nodes, 2, 0, 2)   # leaves of one node in another order: still valid
    assert check_tree4(nodes, leaves, tris) == 2


def _keys(nodes):
    return nodes[:, 28:32].view(np.uint32)


def _swap_slots(nodes, node, a, b):
    for off in range(0, 32, 4):   # planes, references and keys alike
        nodes[node, off + a], nodes[node, off + b] = nodes[node, off + b], nodes[node, off + a].copy()


@pytest.mark.parametrize("fault", ["box", "dup-leaf", "one-child", "gap", "vertex", "parent-box",
                                   "leaf-first", "order", "key"])
def test_planted_fault_is_rejected(fault):
    nodes, leaves, tris = _tree()
    if fault == "box":                 # a leaf box one ulp too small
        nodes[2, 0] = np.nextafter(nodes[2, 0], np.float32(np.inf))
    elif fault == "parent-box":        # a node's box one ulp too large
        nodes[0, 4 + 1] = np.nextafter(nodes[0, 4 + 1], np.float32(np.inf))
    elif fault == "dup-leaf":          # leaf 5 replaced by a second reference to leaf 4
        _refs(nodes)[2, 2] = ~4
    elif fault == "one-child":
        _refs(nodes)[1, 1:] = EMPTY
    elif fault == "gap":               # unused slot before a used one
        r = _refs(nodes)
        r[2, 1], r[2, 3] = EMPTY, ~4
    elif fault == "vertex":
        leaves[2, 0] += 1e-3
    elif fault == "leaf-first":        # the root's leaf in slot 0, its internal children after it
        _swap_slots(nodes, 0, 0, 2)
        _keys(nodes)[0, :3] = [0xFFFFFFFF, 1, 0]
    elif fault == "order":             # internal children 2, 1: not consecutive from slot 0
        _swap_slots(nodes, 0, 0, 1)
        _keys(nodes)[0, :2] = [0, 1]
    elif fault == "key":               # slot 1's key names slot 0
        _keys(nodes)[0, 1] = 0
    with pytest.raises(AssertionError):
        check_tree4(nodes, leaves, tris)
