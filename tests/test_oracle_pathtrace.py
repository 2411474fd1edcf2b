"""Pins of the oracle's LP path tracer (Sec. 8): the counter-based random
numbers, the estimator on a plane whose answer has a closed form, and the
cosine distribution of bounce directions."""

import numpy as np
import pytest

import oracle
from workloads.views import look_at_pose

POSE = look_at_pose((0.0, 0.0, -3.0), (0, 0, 0))
RHO = np.float32([0.5, 0.25, 1.0])
LIGHT = np.array([-0.4, -1.0, 0.6]) / np.linalg.norm([-0.4, -1.0, 0.6])


def _plane(half=20.0):
    a, b, c, d = [-half, -half, 0], [half, -half, 0], [half, half, 0], [-half, half, 0]
    tris = np.array([[a, b, c], [a, c, d]], np.float32)
    return tris, np.stack([RHO, RHO])


def _sky(d):
    s = 0.5 * (d[:, 1] / np.linalg.norm(d, axis=1) + 1.0)
    return np.stack([1 - 0.5 * s, 1 - 0.3 * s, np.ones_like(s)], 1)


def test_uniforms_are_uniform_and_independent():
    u = np.array([[oracle.pt_uniform(11, t, k, dim) for dim in (0, 1)]
                  for t in range(4000) for k in range(3)])
    assert np.all((u >= 0) & (u < 1))
    assert np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))          # 24-bit grid
    n = u.shape[0]
    hist = np.histogram(u[:, 0], bins=20, range=(0, 1))[0]
    chi2 = ((hist - n / 20) ** 2 / (n / 20)).sum()
    assert chi2 < 45                                               # 19 dof, p ~ 1e-3
    assert abs(np.corrcoef(u[:, 0], u[:, 1])[0, 1]) < 0.05
    assert oracle.pt_uniform(11, 5, 1, 0) == oracle.pt_uniform(11, 5, 1, 0)
    assert oracle.pt_uniform(11, 5, 1, 0) != oracle.pt_uniform(12, 5, 1, 0)


def test_empty_scene_is_the_sky(layout):
    tris = np.zeros((0, 3, 3), np.float32)
    alb = np.zeros((0, 3), np.float32)
    tex = np.arange(0, layout.total, 97)
    rgba, sig = oracle.path_trace_lp(tris, alb, LIGHT, layout, 640, 480, 90.0, (320, 240), POSE,
                                     seed=3, texels=tex)
    o, d, _ = oracle.lp_rays(layout, 640, 480, 90.0, (320, 240), POSE, tex)
    np.testing.assert_allclose(rgba[:, :3], _sky(d), atol=1e-12)
    assert np.all(sig[:, 0] == -1) and np.all(sig[:, 1:-1] == -2) and np.all(sig[:, -1] == 0)


def test_plane_direct_light_only(layout):
    # D = 0: a lit Lambertian plane gives rho * cos(n, -L) exactly, nothing else
    tris, alb = _plane()
    tex = np.arange(0, layout.total, 31)
    rgba, sig = oracle.path_trace_lp(tris, alb, LIGHT, layout, 640, 480, 90.0, (320, 240), POSE,
                                     seed=5, max_diffuse=0, texels=tex)
    hit = sig[:, 0] >= 0
    assert hit.mean() > 0.9
    cos = -(np.array([0.0, 0.0, -1.0]) @ LIGHT)                     # plane faces the camera (-z)
    np.testing.assert_allclose(rgba[hit, :3], np.broadcast_to(RHO.astype(float) * cos, (hit.sum(), 3)),
                               rtol=1e-12)
    assert np.all(sig[hit, -1] == 1 | (1 << 16))        # cast and visible at segment 0


def test_plane_one_bounce_expectation(layout):
    # D = 1 over an unoccluded plane: the bounce ray always escapes, so
    # E[L] = rho cos + rho * E[sky(d)] with d cosine-distributed about n; sky
    # is affine in d_y and a cosine lobe has E[d] = (2/3) n, so
    # E[s] = (1 + (2/3) n_y)/2 = 1/2 for n = (0, 0, -1).
    tris, alb = _plane()
    tex = np.arange(layout.total)
    rgba, sig = oracle.path_trace_lp(tris, alb, LIGHT, layout, 640, 480, 90.0, (320, 240), POSE,
                                     seed=9, max_diffuse=1, texels=tex)
    hit = sig[:, 0] >= 0
    assert np.all(sig[hit, 1] == -1)                                # every bounce escapes
    cos = -(np.array([0.0, 0.0, -1.0]) @ LIGHT)
    es = 0.5
    expect = RHO.astype(float) * cos + RHO.astype(float) * np.array([1 - 0.5 * es, 1 - 0.3 * es, 1.0])
    got = rgba[hit, :3]
    se = got.std(0) / np.sqrt(hit.sum())
    assert np.all(np.abs(got.mean(0) - expect) < 5 * se + 1e-9)


def test_bounce_directions_are_cosine_distributed(layout):
    tris, alb = _plane()
    tex = np.arange(0, layout.total, 3)
    rgba, sig, seg = oracle.path_trace_lp(tris, alb, LIGHT, layout, 640, 480, 90.0, (320, 240),
                                          POSE, seed=21, max_diffuse=1, texels=tex, segments=True)
    hit = sig[:, 0] >= 0
    d = seg[hit, 1, 3:]
    n = np.array([0.0, 0.0, -1.0])
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)
    c = d @ n
    assert np.all(c > 0)
    m = c.size
    assert abs(c.mean() - 2 / 3) < 5 * c.std() / np.sqrt(m)         # E[cos] = 2/3
    assert abs((c * c).mean() - 0.5) < 5 * (c * c).std() / np.sqrt(m)   # E[cos^2] = 1/2
    assert np.all(np.abs(d[:, :2].mean(0)) < 5 * d[:, :2].std(0) / np.sqrt(m))
    # the bounce starts just off the plane (1e-5 max(1, |p|) along the normal,
    # towards the camera side) where the primary ray hit it
    pm = np.maximum(1.0, np.abs(seg[hit, 1, :3]).max(1))
    np.testing.assert_allclose(seg[hit, 1, 2], -1e-5 * pm, rtol=1e-6, atol=1e-12)


def test_occluder_shadows_direct_light(layout):
    # a small triangle between the plane and the light removes the direct term
    # exactly where the plane point's shadow ray hits it
    tris, alb = _plane()
    occ = np.array([[[-0.2, 0.2, -0.5], [0.6, 0.2, -0.5], [0.2, 0.9, -0.5]]], np.float32)
    tris = np.concatenate([tris, occ])
    alb = np.concatenate([alb, np.float32([[0.3, 0.3, 0.3]])])
    tex = np.arange(layout.total)
    rgba, sig, seg = oracle.path_trace_lp(tris, alb, LIGHT, layout, 640, 480, 90.0, (320, 240),
                                          POSE, seed=2, max_diffuse=0, texels=tex, segments=True)
    on_plane = (sig[:, 0] == 0) | (sig[:, 0] == 1)
    o, d = seg[on_plane, 0, :3], seg[on_plane, 0, 3:]
    t = -o[:, 2] / d[:, 2]
    p = o + t[:, None] * d
    p[:, 2] -= 1e-5 * np.maximum(1.0, np.abs(p).max(1))           # the shadow ray's origin
    ids, _ = oracle.cast_brute(occ, p, np.broadcast_to(-LIGHT, p.shape))
    shadowed = ids >= 0
    assert 0.001 < shadowed.mean() < 0.5
    lit = (sig[on_plane, -1] & 1) == 1
    assert np.all(sig[on_plane, -1] & (1 << 16))
    assert np.array_equal(lit, ~shadowed)
    assert np.all(rgba[on_plane][shadowed, :3] == 0.0)
