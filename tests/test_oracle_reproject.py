"""Pins of the oracle's VaFR_Rep reprojection (Sec. 5.1: the right eye's LP
buffer warped from the left eye's): the identity warp, exactness on flat
colour, and where holes may appear."""

import numpy as np

import oracle
from workloads.views import eye_pair_poses, look_at_pose

W, H, FOV = 1280, 720, 100.0
HEAD = look_at_pose((0.0, 0.2, -3.0), (0, 0, 0))


def _plane_scene(albedo=(0.6, 0.4, 0.2), half=50.0, z=2.0):
    a, b, c, d = [-half, -half, z], [half, -half, z], [half, half, z], [-half, half, z]
    tris = np.array([[a, b, c], [a, c, d]], np.float32)
    alb = np.float32([albedo, albedo])
    return tris, alb, np.float32([-0.4, -1.0, 0.6]) / np.linalg.norm([-0.4, -1.0, 0.6])


def _left(tris, alb, L, lay, gaze, pose):
    rgba, ids, t, _, _ = oracle.render_lp(tris, alb, L, lay, W, H, FOV, gaze, pose)
    return rgba, np.where(ids >= 0, t, np.inf)


def test_identity_warp_reproduces_the_buffer(layout):
    # right view == left view: every right texel centre is a left vertex
    rng = np.random.default_rng(0)
    tris = rng.uniform(-1, 1, (64, 3, 3)).astype(np.float32)
    alb = rng.uniform(0.2, 1, (64, 3)).astype(np.float32)
    L = np.float32([0, -1, 0])
    gaze = (600.5, 300.25)
    rgba, t = _left(tris, alb, L, layout, gaze, HEAD)
    right, tri = oracle.reproject_lp(layout, W, H, FOV, gaze, HEAD, gaze, HEAD, t, rgba)
    ok = tri >= 0
    assert ok.mean() > 0.95
    np.testing.assert_allclose(right[ok], rgba[ok], atol=1e-9)


def test_flat_colour_plane_is_exact_and_holes_stay_at_the_rim(layout):
    tris, alb, L = _plane_scene()
    poses = eye_pair_poses(HEAD, 0.063)
    gaze = (640.0, 360.0)
    rgba, t = _left(tris, alb, L, layout, gaze, poses[0])
    right, tri = oracle.reproject_lp(layout, W, H, FOV, gaze, poses[0], gaze, poses[1], t, rgba)
    direct, ids, _, _, _ = oracle.render_lp(tris, alb, L, layout, W, H, FOV, gaze, poses[1])
    ok = (tri >= 0) & (ids >= 0)
    # one flat-lit colour: the interpolation of equal colours is exact
    np.testing.assert_allclose(right[ok], direct[ok], atol=1e-12)
    holes = np.flatnonzero(tri < 0)
    assert holes.size < 0.02 * layout.total
    col = np.repeat(np.arange(layout.n_cols), layout.n_col)
    # holes only where the left view ends (outer rim) and at the two polar
    # centres, which no ring triangle covers: the right eye's own innermost
    # ring and the image of the left eye's centre
    assert np.sum(col[holes] < layout.n_cols - 8) <= 8


def test_occluder_opens_holes_beside_it(layout):
    # a box-like occluder in front of the plane: the right eye sees plane
    # texels the left eye does not (disocclusion) -> holes next to the object
    tris, alb, L = _plane_scene()
    q = np.array([[-0.3, -0.3, 0.5], [0.3, -0.3, 0.5], [0.3, 0.3, 0.5], [-0.3, 0.3, 0.5]], np.float32)
    occ = np.array([[q[0], q[1], q[2]], [q[0], q[2], q[3]]], np.float32)
    tris = np.concatenate([tris, occ])
    alb = np.concatenate([alb, np.float32([[0.9, 0.9, 0.9]] * 2)])
    poses = eye_pair_poses(HEAD, 0.063)
    gaze = (640.0, 380.0)
    rgba, t = _left(tris, alb, L, layout, gaze, poses[0])
    right, tri = oracle.reproject_lp(layout, W, H, FOV, gaze, poses[0], gaze, poses[1], t, rgba)
    direct, ids, _, _, _ = oracle.render_lp(tris, alb, L, layout, W, H, FOV, gaze, poses[1])
    inner = np.repeat(np.arange(layout.n_cols), layout.n_col) < layout.n_cols - 8
    holes = (tri < 0) & inner
    assert holes.sum() > 50
    # most holes are background the left eye could not see (disocclusion);
    # the rest are the object's rim, whose triangles span the depth jump
    assert np.mean(ids[holes] <= 1) > 0.5
    # elsewhere the warp agrees with the direct render, edges of the object aside
    ok = (tri >= 0) & inner
    agree = np.all(np.abs(right[ok] - direct[ok]) < 1e-9, axis=1)
    assert agree.mean() > 0.99


def _right_uf(P, pose, gaze, acuity):
    """(U, F) of world points in the right eye's LP coordinates, from the
    definitions: camera coordinates, screen point, e = atan(c_r r) (Eq. 3),
    U = u(e) - 1/2 (Eq. 12), F = angle / 360 with y down."""
    R, eye = pose[:, :3], pose[:, 3]
    c = (P - eye) @ R
    cr = 2.0 * np.tan(np.radians(FOV) / 2) / H
    px = W / 2 + c[:, 0] / (c[:, 2] * cr)
    py = H / 2 - c[:, 1] / (c[:, 2] * cr)
    dx, dy = px - gaze[0], py - gaze[1]
    e = np.minimum(np.degrees(np.arctan(cr * np.hypot(dx, dy))), 60.0)
    U = acuity.u_of_e(e) - 0.5
    F = np.mod(np.arctan2(dy, dx), 2 * np.pi) / (2 * np.pi)
    return U, F


def test_affine_data_in_lp_coordinates_is_reproduced(layout, acuity):
    # left colours that are an affine function of where each left texel's hit
    # point lands in the right eye's (U, F) plane: the barycentric
    # interpolation there must reproduce that function at every covered right
    # texel centre (U = c, F = (j + 1/2) / n_c), away from the angular seam
    tris, alb, L = _plane_scene()
    poses = eye_pair_poses(HEAD, 0.063)
    gl, gr = (610.0, 350.0), (655.0, 372.0)
    _, t = _left(tris, alb, L, layout, gl, poses[0])
    o, d, _ = oracle.lp_rays(layout, W, H, FOV, gl, poses[0])
    hit = np.isfinite(t)
    P = o + np.where(hit, t, 0.0)[:, None] * d
    U, F = _right_uf(P, poses[1], gr, acuity)
    A = np.array([[0.1, 1e-3, 0.4], [0.7, -5e-4, 0.2], [0.3, 2e-4, -0.3]])
    left = np.ones((layout.total, 4))
    left[:, :3] = A[:, 0] + np.outer(U, A[:, 1]) + np.outer(F, A[:, 2])
    right, tri = oracle.reproject_lp(layout, W, H, FOV, gl, poses[0], gr, poses[1], t, left)
    col = np.repeat(np.arange(layout.n_cols), layout.n_col)
    j = np.arange(layout.total) - layout.off_col[col]
    Fc = (j + 0.5) / layout.n_col[col]
    want = A[:, 0] + np.outer(col, A[:, 1]) + np.outer(Fc, A[:, 2])
    sel = (tri >= 0) & (Fc > 0.1) & (Fc < 0.9) & (col >= 4) & (col < layout.n_cols - 8)
    assert sel.sum() > 0.7 * layout.total
    np.testing.assert_allclose(right[sel, :3], want[sel], atol=1e-9)


def _probe_setup(layout, seed=1, k=120):
    """Identical eyes, hit distances putting every vertex 5 units from the eye,
    and random interior left texels with their first triangle's own texel."""
    gaze = (600.5, 300.25)
    _, d, _ = oracle.lp_rays(layout, W, H, FOV, gaze, HEAD)
    dn = np.linalg.norm(d, axis=1)
    t = 5.0 / dn
    col = np.repeat(np.arange(layout.n_cols), layout.n_col)
    cand = np.flatnonzero((col > 2) & (col < layout.n_cols - 3))
    rng = np.random.default_rng(seed)
    tex = rng.choice(cand, k, replace=False)
    s = rng.integers(0, 2, tex.size)
    return gaze, t, dn, tex, 2 * tex + s, col


def test_rep_probe_identity_view_closed_forms(layout):
    """With identical eyes a left texel's vertex lands on its own right texel
    centre (U = c, F = (j + 1/2)/n_c).  Every vertex 5 units away: depth ratio
    1, depth 5 at the texel; the triangle joins columns c and c +- 1 (U span
    1); the texel centre is a vertex, so it lies on the boundary (margin 0)."""
    gaze, t, dn, tex, tid, col = _probe_setup(layout)
    p = oracle.rep_probe(layout, W, H, FOV, gaze, HEAD, gaze, HEAD, t, tid, tex)
    assert np.all(p["exists"] == 1) and np.all(p["in_front"] == 1) and np.all(p["n_inf"] == 0)
    assert np.all(p["front_margin"] > 0)
    np.testing.assert_allclose(p["depth_ratio"], 1.0, atol=1e-12)
    np.testing.assert_allclose(p["u_span"], 1.0, atol=1e-8)
    np.testing.assert_allclose(p["depth"], 5.0, atol=1e-9)
    np.testing.assert_allclose(p["cover_margin"], 0.0, atol=1e-6)
    assert np.all(p["f_span"] <= 0.25)
    # a texel eight columns away is outside the triangle's U range
    far = layout.off_col[np.minimum(col[tex] + 8, layout.n_cols - 1)]
    q = oracle.rep_probe(layout, W, H, FOV, gaze, HEAD, gaze, HEAD, t, tid, far)
    assert np.all(q["cover_margin"] < -1.0)


def test_rep_probe_depths_misses_and_eyes_behind(layout):
    gaze, t, dn, tex, tid, col = _probe_setup(layout, seed=2, k=12)
    for k in range(tex.size):
        tt = t.copy()
        tt[tex[k]] = 6.0 / dn[tex[k]]          # the queried texel's own vertex at 6
        p = oracle.rep_probe(layout, W, H, FOV, gaze, HEAD, gaze, HEAD, tt, tid[k:k + 1], tex[k:k + 1])
        assert abs(p["depth_ratio"][0] - 1.2) < 1e-12     # 6 / 5
        assert abs(p["depth"][0] - 6.0) < 1e-9           # the texel centre is that vertex
        tt[tex[k]] = np.inf                       # a miss: a point at infinity
        p = oracle.rep_probe(layout, W, H, FOV, gaze, HEAD, gaze, HEAD, tt, tid[k:k + 1], tex[k:k + 1])
        assert p["n_inf"][0] == 1 and p["depth_ratio"][0] == 0.0
    # a right eye turned around sees every vertex behind it
    back = HEAD.copy()
    back[:, 0] *= -1.0
    back[:, 2] *= -1.0
    p = oracle.rep_probe(layout, W, H, FOV, gaze, HEAD, gaze, back, t, tid, tex)
    assert np.all(p["in_front"] == 0) and np.all(p["front_margin"] < 0)
    # ids that name no triangle
    p = oracle.rep_probe(layout, W, H, FOV, gaze, HEAD, gaze, HEAD, t, np.array([-1, 2 * layout.total]),
                         np.array([0, 0]))
    assert np.all(p["exists"] == 0)
