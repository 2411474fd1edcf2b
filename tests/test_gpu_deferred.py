"""GPU deferred path (Sec. 3.4, Sec. 5): the CUDA-rasterised visibility buffer
equals the GT cast's closest hits, the LP lighting equals the GT shading of
the pixel under each texel, both against the FP64 oracle; and point lights
(the deferred scenes' many lights) against the oracle's shading."""

import numpy as np
import pytest

import oracle
from parity import classify, compare_hits_and_colours, device_scene, lp_slots
from workloads import workload

pytestmark = pytest.mark.gpu


def _lights(sc, n, seed):
    rng = np.random.default_rng(seed)
    lo, hi = sc.tris.reshape(-1, 3).min(0), sc.tris.reshape(-1, 3).max(0)
    pos = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    pos[:, 1] = hi[1] + rng.uniform(0.5, 3.0, n)           # above the scene
    rgb = rng.uniform(0.2, 1.0, (n, 3)).astype(np.float32) * float(np.max(hi - lo)) ** 2 * 0.5
    return pos, rgb


@pytest.mark.parametrize("name", ["random1k", "terrain4k"])
def test_vbuffer_is_the_gt_cast(V, torch_mod, name):
    w = workload(name, frames=4)
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    pos, rgb = _lights(sc, 16, 3)
    V.vafr_scene_set_point_lights(h, pos, rgb)
    s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, d.poses))
    V.vafr_set_gaze(s, 0, *d.gaze[1, 0])
    W, H = d.width, d.height
    vb = torch_mod.empty((H, W), dtype=torch_mod.int64, device="cuda")
    V.vafr_render_vbuffer(h, s, 0, vb)
    gt = torch_mod.empty((H, W, 4), device="cuda")
    ids = torch_mod.empty(H * W, dtype=torch_mod.int32, device="cuda")
    V.vafr_render_full_gt(h, s, 0, gt, ids)
    full = torch_mod.empty((H, W, 4), device="cuda")
    V.vafr_shade_full_deferred(h, s, 0, vb, full)
    slot, n_slots, _, _ = lp_slots(V, s)
    lp = torch_mod.empty((n_slots, 4), device="cuda")
    V.vafr_shade_lp_deferred(h, s, 0, vb, lp)
    torch_mod.cuda.synchronize()
    assert V.vafr_session_check(s) == 0 and V.vafr_scene_check(h) == 0
    key = vb.cpu().numpy().reshape(-1).view(np.uint64)
    vid = np.where(key == np.uint64(2 ** 64 - 1), -1, (key & np.uint64(0xffffffff)).astype(np.int64))
    # the rasteriser's coverage and depth test reproduce the cast exactly
    assert np.array_equal(vid, ids.cpu().numpy())
    assert torch_mod.equal(full, gt)
    # LP lighting = the GT shading of the pixel under each texel
    lay = oracle.lp_layout()
    _, _, xy = oracle.lp_rays(lay, W, H, d.fov_v_deg, d.gaze[1, 0], d.poses[0])
    px = np.clip(np.floor(xy[:, 0]), 0, W - 1).astype(np.int64)
    py = np.clip(np.floor(xy[:, 1]), 0, H - 1).astype(np.int64)
    got = lp.cpu().numpy()[slot]
    ref = gt.cpu().numpy().reshape(-1, 4)[py * W + px]
    same = np.all(got == ref, axis=1)
    assert same.mean() > 0.999     # the rest sit on a pixel boundary (FP32 vs FP64 floor)
    # against the FP64 oracle on a sample of pixels, point lights included
    rng = np.random.default_rng(7)
    pix = np.sort(rng.choice(W * H, 40000, replace=False))
    bvh = oracle.CpuBVH(sc.tris) if sc.n_tris > 5000 else None
    orgba, oid, ot, o, dd = oracle.render_gt(sc.tris, sc.albedo, sc.light_dir, W, H, d.fov_v_deg,
                                             d.poses[0], pixels=pix, bvh=bvh, point_lights=(pos, rgb))
    compare_hits_and_colours(sc.tris, o, dd, vid[pix], full.cpu().numpy().reshape(-1, 4)[pix], oid, ot,
                             orgba, 1e-3 * max(1.0, float(np.abs(orgba).max())))
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_lp_lighting_against_the_oracle(V, torch_mod):
    """The LP lighting pass (Sec. 3.4 / Sec. 5: lighting at LP resolution from
    the display-resolution G-buffer) against the FP64 oracle: each texel takes
    the shading of the pixel under its screen point, so on a 65,536-texel
    sample the GPU texel must equal the oracle's GT shading of the floor pixel
    of the oracle's screen point -- hit ids exactly except ray-edge ties,
    colours within the FP32 tolerance.  Texels within 1e-2 px of a pixel
    boundary (where the GPU's FP32 screen point may floor to the neighbour)
    must match the oracle at one of the two pixels."""
    w = workload("terrain4k", frames=4)
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    pos, rgb = _lights(sc, 31, 9)
    V.vafr_scene_set_point_lights(h, pos, rgb)
    s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, d.poses))
    gaze = d.gaze[2, 0]
    V.vafr_set_gaze(s, 0, *gaze)
    W, H = d.width, d.height
    vb = torch_mod.empty((H, W), dtype=torch_mod.int64, device="cuda")
    V.vafr_render_vbuffer(h, s, 0, vb)
    slot, n_slots, _, _ = lp_slots(V, s)
    lp = torch_mod.empty((n_slots, 4), device="cuda")
    V.vafr_shade_lp_deferred(h, s, 0, vb, lp)
    torch_mod.cuda.synchronize()
    assert V.vafr_session_check(s) == 0 and V.vafr_scene_check(h) == 0
    key = vb.cpu().numpy().reshape(-1).view(np.uint64)
    vid = np.where(key == np.uint64(2 ** 64 - 1), -1, (key & np.uint64(0xffffffff)).astype(np.int64))
    lay = oracle.lp_layout()
    rng = np.random.default_rng(21)
    tex = np.sort(rng.choice(lay.total, 65536, replace=False))
    _, _, xy = oracle.lp_rays(lay, W, H, d.fov_v_deg, gaze, d.poses[0], texels=tex)
    # texels whose screen point lies on the display (the pass clamps the rest
    # to the border pixel, which the same comparison covers)
    fx, fy = np.floor(xy[:, 0]), np.floor(xy[:, 1])
    px = np.clip(fx, 0, W - 1).astype(np.int64)
    py = np.clip(fy, 0, H - 1).astype(np.int64)
    got = lp.cpu().numpy()[slot][tex]
    eps = 1e-2
    rx, ry = xy[:, 0] - fx, xy[:, 1] - fy
    inside = (xy[:, 0] >= eps) & (xy[:, 0] < W - eps) & (xy[:, 1] >= eps) & (xy[:, 1] < H - eps)
    near = inside & ((rx < eps) | (rx > 1 - eps) | (ry < eps) | (ry > 1 - eps))
    far = ~near
    bvh = oracle.CpuBVH(sc.tris)
    pix = py * W + px
    orgba, oid, ot, o, dd = oracle.render_gt(sc.tris, sc.albedo, sc.light_dir, W, H, d.fov_v_deg,
                                             d.poses[0], pixels=pix[far], bvh=bvh, point_lights=(pos, rgb))
    tol = 1e-3 * max(1.0, float(np.abs(orgba).max()))
    summ = compare_hits_and_colours(sc.tris, o, dd, vid[pix[far]], got[far], oid, ot, orgba, tol)
    print("deferred LP lighting vs oracle", summ, "boundary texels", int(near.sum()))
    # boundary texels: the oracle at the floor pixel or its neighbour across
    # the nearer boundary, hit and colour
    k = np.flatnonzero(near)
    sx = np.where(rx[k] < 0.5, -1, 1) * ((rx[k] < eps) | (rx[k] > 1 - eps))
    sy = np.where(ry[k] < 0.5, -1, 1) * ((ry[k] < eps) | (ry[k] > 1 - eps))
    cands = [pix[k], py[k] * W + np.clip(px[k] + sx, 0, W - 1), np.clip(py[k] + sy, 0, H - 1) * W + px[k],
             np.clip(py[k] + sy, 0, H - 1) * W + np.clip(px[k] + sx, 0, W - 1)]
    ok = np.zeros(k.size, bool)
    for c in cands:
        crgba, cid, _, _, _ = oracle.render_gt(sc.tris, sc.albedo, sc.light_dir, W, H, d.fov_v_deg,
                                               d.poses[0], pixels=c, bvh=bvh, point_lights=(pos, rgb))
        ok |= (vid[c] == cid) & (np.abs(got[k] - crgba).max(1) <= tol)
    # what is left are ray-edge ties at those pixels, inside the same budget
    assert (~ok).sum() <= 1e-4 * tex.size + summ["ties"], (int((~ok).sum()), summ)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_point_lights_in_the_ray_cast(V, torch_mod):
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    pos, rgb = _lights(sc, 31, 5)
    V.vafr_scene_set_point_lights(h, pos, rgb)
    s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, d.poses))
    V.vafr_set_gaze(s, 0, *d.gaze[0, 0])
    slot, n_slots, _, _ = lp_slots(V, s)
    lp = torch_mod.empty((n_slots, 4), device="cuda")
    ids = torch_mod.empty(n_slots, dtype=torch_mod.int32, device="cuda")
    V.vafr_render_lp(h, s, 1, lp, ids)
    torch_mod.cuda.synchronize()
    lay = oracle.lp_layout()
    rgba, oid, ot, o, dd = oracle.render_lp(sc.tris, sc.albedo, sc.light_dir, lay, d.width, d.height,
                                            d.fov_v_deg, d.gaze[0, 0], d.poses[0], point_lights=(pos, rgb))
    assert np.abs(rgba[oid >= 0, :3]).max() > 1.5           # the lights do add light
    compare_hits_and_colours(sc.tris, o, dd, ids.cpu().numpy()[slot], lp.cpu().numpy()[slot], oid, ot,
                             rgba, 1e-3 * max(1.0, float(np.abs(rgba).max())))
    # removing them restores the directional shading exactly
    V.vafr_scene_set_point_lights(h, np.zeros((0, 3)), np.zeros((0, 3)))
    V.vafr_render_lp(h, s, 1, lp, ids)
    torch_mod.cuda.synchronize()
    plain, _, _, _, _ = oracle.render_lp(sc.tris, sc.albedo, sc.light_dir, lay, d.width, d.height,
                                         d.fov_v_deg, d.gaze[0, 0], d.poses[0])
    assert np.abs(lp.cpu().numpy()[slot][oid >= 0] - plain[oid >= 0]).max() < 1e-3 + 1e-6
    with pytest.raises(V.VafrError):
        V.vafr_scene_set_point_lights(h, np.zeros((300, 3)), np.ones((300, 3)))
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def _edge_scene():
    """Triangles that exercise every branch of the rasteriser's set-up: one
    reaching behind the eye (near-plane clip), one wholly behind it, a
    degenerate one, sub-pixel ones, one filling the view just past the eye,
    one with far-away vertices, coplanar overlaps (equal-depth ties), and
    boxes that straddle the display edges."""
    from workloads.scenes import Scene
    rng = np.random.default_rng(11)
    t = []
    t.append([[-50, -1, -20], [50, -1, -20], [0, -1, 60]])        # ground through the eye plane
    t.append([[-1, -1, -5], [1, -1, -5], [0, 1, -5]])             # behind the eye
    t.append([[0, 0, 5], [1, 1, 5], [2, 2, 5]])                   # degenerate (collinear)
    for k in range(200):                                          # sub-pixel, far away
        c = rng.uniform([-40, -10, 300], [40, 30, 400])
        t.append(c + rng.uniform(-0.05, 0.05, (3, 3)))
    t.append([[-0.3, -0.2, 0.2], [0.3, -0.2, 0.2], [0.0, 0.3, 0.2]])   # fills the view near the eye
    t.append([[-1e5, 2, 1e5], [1e5, 2, 1e5], [0, 2, -1e5]])            # far-away vertices
    t.append([[-1, 0, 3], [1, 0, 3], [0, 1.5, 3]])                     # coplanar pair: equal t
    t.append([[-1, 0, 3], [1, 0, 3], [0, 1.5, 3]])
    t.append([[-0.5, -0.5, 3], [1.5, -0.5, 3], [0.5, 1.0, 3]])
    for k in range(300):                                          # mid-size, some off-screen
        c = rng.uniform([-8, -5, 4], [8, 5, 30])
        t.append(c + rng.uniform(-1.5, 1.5, (3, 3)))
    tris = np.asarray(t, np.float32)
    alb = rng.uniform(0.2, 1.0, (len(tris), 3)).astype(np.float32)
    return Scene(tris, alb, np.float32([-0.4, -1.0, 0.6]) / np.float32(np.linalg.norm([-0.4, -1.0, 0.6])))


@pytest.mark.parametrize("size", [(333, 197), (16, 8), (1, 1), (1031, 777)])
def test_vbuffer_edge_cases(V, torch_mod, size):
    """The V-buffer equals the GT cast's hits exactly on awkward geometry and
    on display sizes that are not multiples of the raster tiles."""
    from workloads.views import look_at_pose
    sc = _edge_scene()
    h, keep = device_scene(V, sc, torch_mod)
    W, H = size
    pose = look_at_pose((0.0, 0.5, 0.0), (0.0, 0.3, 10.0))
    s = V.vafr_session_create(V.make_session_desc(W, H, 90.0, [pose]))
    V.vafr_set_gaze(s, 0, 0.37 * W, 0.61 * H)
    vb = torch_mod.empty((H, W), dtype=torch_mod.int64, device="cuda")
    V.vafr_render_vbuffer(h, s, 0, vb)
    gt = torch_mod.empty((H, W, 4), device="cuda")
    ids = torch_mod.empty(H * W, dtype=torch_mod.int32, device="cuda")
    V.vafr_render_full_gt(h, s, 0, gt, ids)
    full = torch_mod.empty((H, W, 4), device="cuda")
    V.vafr_shade_full_deferred(h, s, 0, vb, full)
    torch_mod.cuda.synchronize()
    assert V.vafr_session_check(s) == 0 and V.vafr_scene_check(h) == 0
    key = vb.cpu().numpy().reshape(-1).view(np.uint64)
    vid = np.where(key == np.uint64(2 ** 64 - 1), -1, (key & np.uint64(0xffffffff)).astype(np.int64))
    assert np.array_equal(vid, ids.cpu().numpy())
    assert torch_mod.equal(full, gt)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_vbuffer_empty_scene(V, torch_mod):
    from workloads.scenes import Scene
    from workloads.views import look_at_pose
    sc = Scene(np.zeros((0, 3, 3), np.float32), np.zeros((0, 3), np.float32), np.float32([0, -1, 0]))
    h, keep = device_scene(V, sc, torch_mod)
    s = V.vafr_session_create(V.make_session_desc(64, 48, 60.0, [look_at_pose((0, 0, -3), (0, 0, 0))]))
    V.vafr_set_gaze(s, 0, 32.0, 24.0)
    vb = torch_mod.zeros((48, 64), dtype=torch_mod.int64, device="cuda")
    V.vafr_render_vbuffer(h, s, 0, vb)
    torch_mod.cuda.synchronize()
    assert bool((vb == -1).all())      # every pixel is sky (key ~0)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_vbuffer_stats_counts_and_buffer(V, torch_mod):
    """The instrumented rasteriser writes the same buffer, and its counters
    nest: pre-filter evaluations >= pixels past it >= exact tests >= atomics."""
    w = workload("random1k", frames=4)
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, d.poses))
    V.vafr_set_gaze(s, 0, *d.gaze[0, 0])
    vb = torch_mod.empty((d.height, d.width), dtype=torch_mod.int64, device="cuda")
    vb2 = torch_mod.empty_like(vb)
    V.vafr_render_vbuffer(h, s, 0, vb)
    st = V.vafr_vbuffer_stats(h, s, 0, vb2)
    torch_mod.cuda.synchronize()
    assert torch_mod.equal(vb, vb2)
    assert st["prefilter"] >= st["filtered"] >= st["tests"] >= st["atomics"] > 0
    covered = int((vb != -1).sum())
    assert st["atomics"] >= covered          # every covered pixel took at least one minimum
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)
