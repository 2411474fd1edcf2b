"""Pins of the oracle's LBVH reference (Karras 2012): Morton codes on hand-computed
cases, stable sort, the binary radix tree against its definition by brute
force, and exact bounds."""

import numpy as np
import pytest

import oracle
from workloads import random_triangles_scene


def _point_tris(points):
    p = np.asarray(points, np.float32)
    return np.repeat(p[:, None, :], 3, axis=1)


def test_morton_hand_computed():
    # Degenerate triangles at integer points p: centroid sum 3p is exact, and
    # with the bounds spanning [0, 3*1024] the quantised cell is q = p (1023 at 1024).
    pts = [[0, 0, 0], [1024, 1024, 1024], [1, 0, 0], [0, 1, 0], [0, 0, 1],
           [3, 0, 0], [512, 0, 0], [1023, 1023, 1023], [5, 6, 7]]
    codes = oracle.morton(_point_tris(pts))
    want = [0, 2**30 - 1, 4, 2, 1, 4 + 32, 2**29, 2**30 - 1,
            # (5,6,7): x=101b y=110b z=111b -> bits (b2: x1 y1 z1)(b1: x0 y1 z1)(b0: x1 y0 z1)
            0b111_011_101]
    assert codes.tolist() == want


def test_morton_cubic_grid():
    # centroid-sum extents 3072 (x) and 1536 (y): every axis is scaled by the
    # largest extent, so t = 3p / 3072 = p / 1024 and q = p (1023 at 1024)
    codes = oracle.morton(_point_tris([[0, 0, 0], [1024, 512, 0], [0, 512, 0], [256, 256, 0]]))
    # (0,0,0) -> 0; (1023,512,0): x bits all set, y bit 9 -> 0x24924924 | 2**28;
    # (0,512,0) -> y bit 9 -> bit 28; (256,256,0) -> x bit 8 (bit 26) + y bit 8 (bit 25)
    assert codes.tolist() == [0, 0x24924924 | 2**28, 2**28, 2**26 + 2**25]


def test_morton_degenerate_axis():
    # y and z have zero extent (q = 0 there): only the x bits 2, 5, ..., 29 can be set
    codes = oracle.morton(_point_tris([[0, 5, 0], [1024, 5, 0], [512, 5, 0]]))
    assert codes.tolist() == [0, 0x24924924, 2**29]


def _lcp(a, b):
    x = a ^ b
    return 64 if x == 0 else 63 - int(x).bit_length() + 1


def _keys(b: oracle.LBVH):
    sc = b.codes[b.sorted_ids].astype(np.uint64)
    return [(int(c) << 32) | i for i, c in enumerate(sc)]


def _check_tree(b: oracle.LBVH, tris):
    n = len(b.sorted_ids)
    keys = _keys(b)
    # stable sort by (code, id)
    pairs = list(zip(b.codes[b.sorted_ids].tolist(), b.sorted_ids.tolist()))
    assert pairs == sorted(pairs)
    assert sorted(b.sorted_ids.tolist()) == list(range(n))
    if n == 1:
        return
    # every leaf and every non-root internal node referenced exactly once
    ref = b.child.reshape(-1)
    leaves = sorted((~ref[ref < 0]).tolist())
    inner = sorted(ref[ref >= 0].tolist())
    assert leaves == list(range(n))
    assert inner == list(range(1, n - 1))
    # definition (brute force): internal ranges are exactly the maximal ranges
    # [i, j] whose keys share a longer prefix than either extension.
    want = set()
    for i in range(n):
        for j in range(i + 1, n):
            d = _lcp(keys[i], keys[j])
            if (i == 0 or _lcp(keys[i - 1], keys[j]) < d) and (j == n - 1 or _lcp(keys[i], keys[j + 1]) < d):
                want.add((i, j))
    got = {tuple(r) for r in b.range.tolist()}
    assert got == want
    for v in range(n - 1):
        f, l = b.range[v]
        assert v in (f, l)                     # Karras numbering
        rng = []
        for c in b.child[v]:
            rng.append((~c, ~c) if c < 0 else tuple(b.range[c]))
        assert rng[0][0] == f and rng[1][1] == l and rng[0][1] + 1 == rng[1][0]
        bit = 63 - _lcp(keys[f], keys[l])
        assert all(((keys[k] >> bit) & 1) == 0 for k in range(rng[0][0], rng[0][1] + 1))
        assert all(((keys[k] >> bit) & 1) == 1 for k in range(rng[1][0], rng[1][1] + 1))
    # bounds: leaves are exact triangle boxes, nodes exact unions
    t = tris[b.sorted_ids]
    np.testing.assert_array_equal(b.leaf_box[:, :3], t.min(axis=1))
    np.testing.assert_array_equal(b.leaf_box[:, 3:], t.max(axis=1))
    for v in range(n - 1):
        f, l = b.range[v]
        np.testing.assert_array_equal(b.node_box[v, :3], b.leaf_box[f:l + 1, :3].min(0))
        np.testing.assert_array_equal(b.node_box[v, 3:], b.leaf_box[f:l + 1, 3:].max(0))


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (7, 2), (16, 3), (61, 4), (200, 5)])
def test_radix_tree_matches_definition(n, seed):
    tris = random_triangles_scene(n, seed=seed).tris
    _check_tree(oracle.lbvh(tris), tris)


def test_radix_tree_duplicate_codes():
    # many identical centroids: equal codes split by position (key concatenation)
    rng = np.random.default_rng(9)
    pts = rng.integers(0, 3, size=(40, 3)) * 512
    tris = _point_tris(pts)
    b = oracle.lbvh(tris)
    assert len(set(b.codes.tolist())) < 40
    _check_tree(b, tris)


def test_single_triangle_has_no_internal_nodes():
    tris = random_triangles_scene(1, seed=0).tris
    b = oracle.lbvh(tris)
    assert b.child.shape == (0, 2)
    assert b.sorted_ids.tolist() == [0]
