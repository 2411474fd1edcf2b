"""Pins of the oracle's ray casting (watertight test, closest hit, tie rule,
CPU BVH) and shading against closed forms and a textbook routine."""

import math

import numpy as np
import pytest

import oracle
from workloads import random_triangles_scene, tiny_scene


def _mt_brute(tris, o, d, eps=0.0):
    """Moller-Trumbore (1997), a different textbook test, vectorised in numpy."""
    v0, v1, v2 = tris[:, 0].astype(float), tris[:, 1].astype(float), tris[:, 2].astype(float)
    e1, e2 = v1 - v0, v2 - v0
    ids = np.full(len(o), -1)
    ts = np.full(len(o), np.inf)
    margin = np.full(len(o), np.inf)
    for k in range(len(o)):
        p = np.cross(d[k], e2)
        det = np.einsum("ij,ij->i", e1, p)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / det
            s = o[k] - v0
            u = np.einsum("ij,ij->i", s, p) * inv
            q = np.cross(s, e1)
            v = (q @ d[k]) * inv
            t = np.einsum("ij,ij->i", e2, q) * inv
        ok = (det != 0) & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
        if ok.any():
            i = np.flatnonzero(ok)[np.argmin(t[ok])]
            ids[k], ts[k] = i, t[i]
            margin[k] = min(u[i], v[i], 1 - u[i] - v[i])
    return ids, ts, margin


def test_single_triangle_distance():
    sc = tiny_scene("single")
    o = np.array([[0.0, 0.0, -3.0]])
    ids, t = oracle.cast_brute(sc.tris, o, np.array([[0.0, 0.0, 1.0]]))
    assert ids[0] == 0 and t[0] == 3.0
    ids, t = oracle.cast_brute(sc.tris, o, np.array([[0.0, 0.0, 2.0]]))   # unnormalised d
    assert ids[0] == 0 and t[0] == 1.5
    ids, _ = oracle.cast_brute(sc.tris, o, np.array([[0.0, 0.0, -1.0]]))  # behind
    assert ids[0] == -1
    ids, _ = oracle.cast_brute(sc.tris, o, np.array([[1.0, 0.0, 0.0]]))   # parallel
    assert ids[0] == -1
    # two-sided: reversed winding hits too
    ids, _ = oracle.cast_brute(sc.tris[:, ::-1].copy(), o, np.array([[0.0, 0.0, 1.0]]))
    assert ids[0] == 0


def test_watertight_shared_edge_and_vertex():
    # rays through the shared diagonal of a quad and the shared centre of a fan
    # always hit (no cracks); equal t goes to the lowest id.
    quad = tiny_scene("quad")
    s = np.linspace(-0.999, 0.999, 801)
    o = np.tile([0.0, 0.0, -3.0], (s.size, 1))
    d = np.stack([s, s, np.full_like(s, 3.0)], 1)       # through (s, s, 0) on the diagonal
    ids, t = oracle.cast_brute(quad.tris, o, d)
    assert np.all(ids == 0)
    np.testing.assert_allclose(t, 1.0, rtol=1e-15)
    fan = tiny_scene("fan")
    o = np.array([[0.3, -0.2, -2.0], [0.0, 0.0, -5.0]])
    d = np.array([[-0.3, 0.2, 2.0], [0.0, 0.0, 1.0]])
    ids, _ = oracle.cast_brute(fan.tris, o, d)
    assert np.all(ids == 0)


def test_tie_rule_lowest_id():
    sc = tiny_scene("stack")   # tris 0, 1 identical, 3 = 0 reversed, 2 behind
    rng = np.random.default_rng(0)
    p = np.stack([rng.uniform(-0.3, 0.3, 200), rng.uniform(-0.5, 0.3, 200), np.zeros(200)], 1)
    o = np.tile([0.0, 0.0, -3.0], (200, 1))
    ids, _ = oracle.cast_brute(sc.tris, o, p - o)
    assert np.all(ids == 0)
    ids, _ = oracle.cast_brute(sc.tris[[2, 1, 3]], o, p - o)
    assert np.all(ids == 1)   # index 1 (the copy of tri 1) is nearest; 2 ties with it but is higher


def test_brute_force_matches_textbook_test():
    sc = random_triangles_scene(200, seed=11)
    rng = np.random.default_rng(1)
    o = np.tile([0.0, 0.0, -3.0], (600, 1))
    d = np.stack([rng.uniform(-0.5, 0.5, 600), rng.uniform(-0.5, 0.5, 600), np.ones(600)], 1)
    ids, t = oracle.cast_brute(sc.tris, o, d)
    mids, mts, margin = _mt_brute(sc.tris, o, d)
    clear = margin > 1e-9
    assert clear.mean() > 0.5
    assert np.array_equal(ids[clear], mids[clear])
    np.testing.assert_allclose(t[clear], mts[clear], rtol=1e-12)
    # hit points lie on the triangle's plane
    hit = ids >= 0
    P = o[hit] + t[hit, None] * d[hit]
    tri = sc.tris[ids[hit]].astype(float)
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    dist = np.einsum("ij,ij->i", n, P - tri[:, 0]) / np.linalg.norm(n, axis=1)
    assert np.abs(dist).max() < 1e-12


def test_cpu_bvh_equals_brute_force(layout):
    sc = random_triangles_scene(1024, seed=1001)
    pose = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, -3.0]])
    tex = np.arange(0, layout.total, 13)
    o, d, _ = oracle.lp_rays(layout, 512, 512, 90.0, (256.0, 256.0), pose, tex)
    ids, t = oracle.cast_brute(sc.tris, o, d)
    bvh = oracle.CpuBVH(sc.tris)
    ids2, t2 = bvh.cast(o, d)
    assert np.array_equal(ids, ids2)
    assert np.array_equal(t, t2)
    assert 0.2 < (ids >= 0).mean() < 0.95


def test_shading_closed_forms():
    sc = tiny_scene("single")   # plane z = 0, normal +-z
    L = np.array([0.0, 0.0, 1.0])       # light travelling +z: lights the -z face
    alb = np.array([[0.5, 0.6, 0.7]], np.float32)
    d = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    rgba = oracle.shade(sc.tris, alb, L, d, np.array([0, 0]))
    # viewer on -z side sees the lit face; viewer on +z side sees the dark face
    np.testing.assert_allclose(rgba[0], [0.5, 0.6, 0.7, 1.0], rtol=1e-6)
    np.testing.assert_allclose(rgba[1], [0.05, 0.06, 0.07, 1.0], rtol=1e-6)
    L2 = np.array([0.0, math.sin(math.radians(30)), math.cos(math.radians(30))])
    rgba = oracle.shade(sc.tris, alb, L2, d[:1], np.array([0]))
    s = 0.1 + 0.9 * math.cos(math.radians(30))
    np.testing.assert_allclose(rgba[0, :3], alb[0] * s, rtol=1e-6)
    sky = oracle.shade(sc.tris, alb, L, np.array([[0, 1.0, 0], [0, -2.0, 0], [3.0, 0, 0]]),
                       np.array([-1, -1, -1]))
    np.testing.assert_allclose(sky, [[0.5, 0.7, 1.0, 1.0], [1, 1, 1, 1], [0.75, 0.85, 1.0, 1.0]])


def test_point_light_inverse_square_closed_form():
    # a point light of power rgb at height h straight above a lit plane point
    # adds albedo * rgb / h^2 there (cos = 1); two lights add up
    half = 20.0
    a, b, c, d = [-half, -half, 0], [half, -half, 0], [half, half, 0], [-half, half, 0]
    tris = np.array([[a, b, c], [a, c, d]], np.float32)
    alb = np.float32([[0.5, 0.25, 1.0]] * 2)
    L = np.array([0.0, 0.0, 1.0])                     # directional light from behind the plane
    o = np.array([[0.3, -0.2, -2.0], [1.5, 0.5, -2.0]])
    dirs = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    ids, t = oracle.cast_brute(tris, o, dirs)
    assert np.all(ids >= 0) and np.allclose(t, 2.0)
    base = oracle.shade(tris, alb, L, dirs, ids)
    pl1 = (np.array([[0.3, -0.2, -1.5]]), np.array([[2.0, 1.0, 0.5]]))
    one = oracle.shade(tris, alb, L, dirs, ids, pl1, o, t)
    np.testing.assert_allclose(one[0, :3] - base[0, :3], alb[0] * pl1[1][0] / 1.5 ** 2, rtol=1e-12)
    pl2 = (np.array([[0.3, -0.2, -1.5], [1.5, 0.5, -0.5]]), np.array([[2.0, 1.0, 0.5], [1.0, 1.0, 1.0]]))
    two = oracle.shade(tris, alb, L, dirs, ids, pl2, o, t)
    solo = oracle.shade(tris, alb, L, dirs, ids, (pl2[0][1:], pl2[1][1:]), o, t)
    np.testing.assert_allclose(two - base, (one - base) + (solo - base), atol=1e-12)
    # a light behind the surface adds nothing
    behind = oracle.shade(tris, alb, L, dirs, ids, (np.array([[0.3, -0.2, 1.0]]), np.ones((1, 3))), o, t)
    np.testing.assert_allclose(behind, base, atol=0)
