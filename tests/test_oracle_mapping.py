"""Pins of the oracle's acuity model, log-polar mapping, layout and reconstruction
filter against what the paper prints and what the mathematics fixes."""

import math

import numpy as np
import pytest

import oracle


def test_pivots_reproduce_printed_acuity(golden, acuity):
    # Sec. 3.3: the MAR segments pass through the printed pivots (E_k, f_k).
    E = np.array(golden["pivots"]["eccentricity_deg"], float)
    f = np.array(golden["pivots"]["acuity_cpd"], float)
    # approach each pivot from inside the segment that ends there and from
    # inside the one that starts there: the MAR model is continuous.
    for k, (e, fk) in enumerate(zip(E, f)):
        if k > 0:
            assert acuity.f_of_e(e - 1e-9)[0] == pytest.approx(fk, rel=1e-7)
        if k < len(E) - 1:
            assert acuity.f_of_e(e)[0] == pytest.approx(fk, rel=1e-12)


def test_shading_rate_equals_acuity(acuity):
    # Eq. 13: SR(e) = (1/2) du/de = f(e) -- central differences of u.
    rng = np.random.default_rng(0)
    e = np.concatenate([rng.uniform(0.05, 59.95, 400), [0.5, 9.9, 10.1, 19.9, 20.1, 29.9, 30.1]])
    h = 1e-5
    du = (acuity.u_of_e(e + h) - acuity.u_of_e(e - h)) / (2 * h)
    np.testing.assert_allclose(0.5 * du, acuity.f_of_e(e), rtol=2e-6)


def test_u_zero_at_fovea_and_continuous(acuity):
    assert acuity.u_of_e(0.0)[0] == pytest.approx(0.0, abs=1e-9)
    for E in (10.0, 20.0, 30.0):
        lo, hi = acuity.u_of_e(E - 1e-10)[0], acuity.u_of_e(E)[0]
        assert abs(hi - lo) < 1e-6


def test_u_first_segment_closed_form(acuity):
    # Eq. 5 on [0, 10): u(10) = (2/m1) ln(omega(10)/omega(0)) with omega = 1/f.
    m1 = (1 / 10 - 1 / 40) / 10
    assert acuity.u_of_e(10.0)[0] == pytest.approx(2 / m1 * math.log(4.0), rel=1e-12)


def test_inverse_round_trip(acuity):
    # Eq. 10 inverts Eq. 5/12 on every segment.
    e = np.linspace(0.0, 60.0, 2001)
    np.testing.assert_allclose(acuity.e_of_u(acuity.u_of_e(e)), e, atol=1e-10)
    u = np.linspace(0.0, acuity.u_of_e(60.0)[0], 2001)
    np.testing.assert_allclose(acuity.u_of_e(acuity.e_of_u(u)), u, atol=1e-9)


def test_tangential_rate_equals_radial(acuity):
    # Eq. 6: r dtheta/dv = dr/du with r = tan(e)/c_r (Eq. 3) and v = l(e) theta/360
    # (Eqs. 8-9).  Holds for any c_r; theta in radians on the left-hand side.
    cr = 3.7e-4
    u = np.linspace(5.0, 895.0, 300)
    h = 1e-4
    r = lambda uu: np.tan(np.radians(acuity.e_of_u(uu))) / cr
    dr_du = (r(u + h) - r(u - h)) / (2 * h)
    e = acuity.e_of_u(u)
    dv_dtheta = acuity.l_of_e(e) / (2 * math.pi)   # texels per radian
    np.testing.assert_allclose(r(u) / dv_dtheta, dr_du, rtol=1e-6)


def test_shading_height_shape(acuity):
    # Eq. 9: l(0) = 0 and l = v(e, 360).
    assert acuity.l_of_e(0.0)[0] == 0.0
    e = np.linspace(0.01, 60, 6000)
    l = acuity.l_of_e(e)
    assert np.all(l > 0)


def test_integrated_shading_points_match_printed_count(golden, acuity):
    # Fig. 5 caption: 1,061,735 shading points = area of the semi-ellipse
    # v < l(e(u)), u in [0, u(60)] (Sec. 3.2.2).  This pins the pivot reading.
    from scipy.integrate import quad
    umax = acuity.u_of_e(60.0)[0]
    brk = list(acuity.u_of_e([10.0, 20.0, 30.0]))
    area, _ = quad(lambda u: acuity.l_of_e(acuity.e_of_u(u))[0], 0, umax, limit=400, points=brk)
    assert area == pytest.approx(golden["shading_points"]["value"], rel=1e-4)


def test_printed_buffer_size_is_flat_5cpd_reading(golden):
    # Sec. 3.2.2 prints (w, h) = (932, 1800) with l maximal near 45 deg.  Those two
    # numbers follow from holding f at 5 cpd on [30, 60) -- the m -> 0 limit of
    # Eq. 12 -- not from the printed 4 cpd at 60 deg (whose area is the printed
    # count above).  Both readings are reproduced.
    flat = oracle.Acuity((0, 10, 20, 30, 60), (40, 10, 6, 5, 5))
    assert round(flat.u_of_e(60.0)[0]) == golden["lp_buffer_size"]["width"]
    e = np.linspace(0.01, 60, 60001)
    l = flat.l_of_e(e)
    assert round(l.max()) == golden["lp_buffer_size"]["height"]
    assert e[np.argmax(l)] == pytest.approx(golden["lp_buffer_size"]["argmax_l_deg_printed"], abs=0.01)


def test_layout_counts(golden, acuity, layout):
    # Discrete layout: columns at u = c + 0.5 below u(60); n_c = round(l(e_c)).
    assert layout.n_cols == int(math.floor(acuity.u_of_e(60.0)[0] - 0.5)) + 1
    assert np.all(layout.n_col >= 1)
    l = acuity.l_of_e(layout.e_col)
    assert np.all(np.abs(layout.n_col - l) <= 0.5)
    assert np.array_equal(layout.off_col, np.concatenate([[0], np.cumsum(layout.n_col)[:-1]]))
    assert layout.total == int(layout.n_col.sum())
    # within 0.02 % of the printed 1,061,735 (Fig. 5) and "1,061K" in Table 1
    assert abs(layout.total - golden["shading_points"]["value"]) / layout.total < 2e-4
    for res, k in golden["rays_per_eye_table"]["vafr_dup_k"].items():
        assert layout.total // 1000 == k


def test_gt_rays_table(golden):
    # Table 1, GT column: one ray per display pixel.
    tab = golden["rays_per_eye_table"]
    for res, (W, H) in tab["resolutions"].items():
        o, d = oracle.pixel_rays(W, H, 90.0, np.eye(3, 4), pixels=np.array([0, W * H - 1]))
        assert d.shape == (2, 3)
        assert (W * H) // 1000 == tab["gt_k"][res]


def test_texel_forward_inverse_round_trip(acuity, layout):
    # Eqs. 3, 10, 11: a texel's screen point maps forward to the texel centre.
    rng = np.random.default_rng(1)
    tex = rng.integers(0, layout.total, 5000)
    W, H, fov, gaze = 3840, 2160, 100.0, (1500.25, 900.75)
    _, _, xy = oracle.lp_rays(layout, W, H, fov, gaze, np.eye(3, 4), tex)
    cr = 2 * math.tan(math.radians(fov) / 2) / H
    dx, dy = xy[:, 0] - gaze[0], xy[:, 1] - gaze[1]
    r = np.hypot(dx, dy)
    e = np.degrees(np.arctan(cr * r))
    u = acuity.u_of_e(e)
    col = np.searchsorted(layout.off_col, tex, side="right") - 1
    np.testing.assert_allclose(u, col + 0.5, atol=1e-7)
    ang = np.degrees(np.arctan2(dy, dx)) % 360.0
    j = tex - layout.off_col[col]
    want = (j + 0.5) / layout.n_col[col] * 360.0
    err = (ang - want + 180.0) % 360.0 - 180.0
    assert np.abs(err).max() < 1e-7


def test_lp_rays_independent_of_resolution(layout):
    # Sec. 3.2.2: the LP buffer does not depend on the display resolution: for the
    # same FOV, pose and gaze direction the rays are the same at 1080p and 8K.
    rng = np.random.default_rng(2)
    tex = rng.integers(0, layout.total, 4000)
    pose = np.eye(3, 4)
    _, d1, _ = oracle.lp_rays(layout, 1920, 1080, 100.0, (960.0, 540.0), pose, tex)
    _, d2, _ = oracle.lp_rays(layout, 7680, 4320, 100.0, (3840.0, 2160.0), pose, tex)
    np.testing.assert_allclose(d1, d2, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------------------
# reconstruction filter (Sec. 3.4 inverse mapping; bilinear reading)

def test_reconstruct_constant_is_exact(layout):
    lp = np.tile([0.25, 0.5, 0.75, 1.0], (layout.total, 1))
    pts = oracle.pixel_centres(640, 360)
    out = oracle.reconstruct_points(lp, layout, 640, 360, 100.0, (200.3, 100.9), pts)
    np.testing.assert_allclose(out, np.broadcast_to(lp[0], out.shape), atol=1e-14)


def test_reconstruct_at_texel_centres_returns_texel(layout):
    # Sampling at a texel's inverse-mapped screen point gives weight 1 to that
    # texel: pins the half-texel offsets, the angle direction and the wrap.
    rng = np.random.default_rng(3)
    lp = rng.uniform(0, 1, (layout.total, 4))
    W, H, fov, gaze = 1920, 1080, 100.0, (700.5, 400.25)
    tex = rng.integers(0, layout.total, 3000)
    _, _, xy = oracle.lp_rays(layout, W, H, fov, gaze, np.eye(3, 4), tex)
    out = oracle.reconstruct_points(lp, layout, W, H, fov, gaze, xy)
    np.testing.assert_allclose(out, lp[tex], atol=1e-6)


def test_reconstruct_smooth_field_within_interpolation_bound(acuity, layout):
    # F(e, phi) = (e/60, (1+cos phi)/2, (1+sin phi)/2) at texel centres; the
    # bilinear reconstruction must reproduce F(e(x,y), phi(x,y)) to the
    # interpolation error bound wherever columns hold >= 100 texels.
    e_c = np.repeat(layout.e_col, layout.n_col)
    col = np.repeat(np.arange(layout.n_cols), layout.n_col)
    j = np.arange(layout.total) - layout.off_col[col]
    phi = np.radians((j + 0.5) / layout.n_col[col] * 360.0)
    lp = np.stack([e_c / 60, 0.5 + 0.5 * np.cos(phi), 0.5 + 0.5 * np.sin(phi), np.ones_like(phi)], 1)
    W, H, fov, gaze = 2560, 1440, 100.0, (1280.0, 720.0)
    rng = np.random.default_rng(4)
    pts = np.stack([rng.uniform(0, W, 20000), rng.uniform(0, H, 20000)], 1)
    out = oracle.reconstruct_points(lp, layout, W, H, fov, gaze, pts)
    cr = 2 * math.tan(math.radians(fov) / 2) / H
    dx, dy = pts[:, 0] - gaze[0], pts[:, 1] - gaze[1]
    e = np.degrees(np.arctan(cr * np.hypot(dx, dy)))
    ph = np.arctan2(dy, dx)
    ref = np.stack([np.minimum(e, 60) / 60, 0.5 + 0.5 * np.cos(ph), 0.5 + 0.5 * np.sin(ph)], 1)
    n_here = layout.n_col[np.clip(np.floor(acuity.u_of_e(np.minimum(e, 60)) - 0.5).astype(int),
                                  0, layout.n_cols - 1)]
    ok = (n_here >= 100) & (e < 59.5)
    # bilinear bound: (1/8) h^2 max|F''| with angular spacing h <= 2 pi / 100
    bound = 0.125 * (2 * math.pi / 100) ** 2 * 0.5 + 1e-4
    assert np.abs(out[ok, :3] - ref[ok]).max() < bound
    assert ok.mean() > 0.6


def test_reconstruct_clamps_beyond_e_max(layout):
    # points past 60 deg read the outermost column along the same angle
    rng = np.random.default_rng(5)
    lp = rng.uniform(0, 1, (layout.total, 4))
    W, H, fov, gaze = 3840, 2160, 110.0, (200.0, 200.0)
    cr = 2 * math.tan(math.radians(fov) / 2) / H
    r60 = math.tan(math.radians(60.0)) / cr
    ang = np.radians(np.array([10.0, 20.0, 40.0]))
    far = np.stack([gaze[0] + 1.3 * r60 * np.cos(ang), gaze[1] + 1.3 * r60 * np.sin(ang)], 1)
    edge = np.stack([gaze[0] + r60 * np.cos(ang), gaze[1] + r60 * np.sin(ang)], 1)
    a = oracle.reconstruct_points(lp, layout, W, H, fov, gaze, far)
    b = oracle.reconstruct_points(lp, layout, W, H, fov, gaze, edge)
    np.testing.assert_allclose(a, b, atol=1e-9)
