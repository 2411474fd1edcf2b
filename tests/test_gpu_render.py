"""GPU LP render (ray generation + traversal + shading) and GT render against the
FP64 oracle: hit triangle ids bit-exact except classified ray-edge / depth ties
(<= 0.01 % of rays), colours within 1e-3 (FP32) or the FP16 bound + 1e-3."""

import math

import numpy as np
import pytest

import oracle
from parity import check_guards, compare_hits_and_colours, device_scene, lp_slots
from workloads import random_triangles_scene, tiny_scene, workload
from workloads.views import look_at_pose

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lay():
    return oracle.lp_layout()


def _session(V, W, H, fov, poses, lp_fmt=0, disp_fmt=0, acuity=None):
    return V.vafr_session_create(V.make_session_desc(W, H, fov, poses, lp_fmt, disp_fmt, acuity))


def _render_lp(V, torch, scene_h, sess, n_tex, eye_mask=1, fp16=False):
    """LP render of the eyes in `eye_mask`; returns the texels (and hit ids) in
    the oracle's order, eye after eye, after checking every guard slot."""
    eyes = bin(eye_mask).count("1")
    slot, n_slots, counts, offs = lp_slots(V, sess)
    assert len(slot) == n_tex
    dt = torch.float16 if fp16 else torch.float32
    lp = torch.empty((eyes * n_slots, 4), dtype=dt, device="cuda")
    ids = torch.empty(eyes * n_slots, dtype=torch.int32, device="cuda")
    V.vafr_render_lp(scene_h, sess, eye_mask, lp, ids)
    torch.cuda.synchronize()
    assert V.vafr_session_check(sess) == 0
    lp = lp.float().cpu().numpy().reshape(eyes, n_slots, 4)
    ids = ids.cpu().numpy().reshape(eyes, n_slots)
    for e in range(eyes):
        check_guards(lp[e], counts, offs)
        check_guards(ids[e], counts, offs)
    return lp[:, slot].reshape(-1, 4), ids[:, slot].reshape(-1)


def test_layout_matches_oracle(V, lay):
    pose = look_at_pose((0, 0, -3), (0, 0, 0))
    for W, H in [(512, 512), (7680, 4320)]:
        s = _session(V, W, H, 90.0, [pose])
        counts, offs, ecc, n_tex = V.vafr_lp_layout(s)
        assert n_tex == lay.total
        assert np.array_equal(counts, lay.n_col)
        # the oracle's offsets plus a guard slot on each side of every column
        assert np.array_equal(offs, np.asarray(lay.off_col) + 2 * np.arange(len(counts)) + 1)
        lpb, _ = V.vafr_session_sizes(s)
        assert lpb == 16 * (lay.total + 2 * len(counts))
        np.testing.assert_allclose(ecc, lay.e_col, rtol=1e-6)
        V.vafr_session_destroy(s)


ANISO = (1.0, 5.0 / 6.0, 2.0 / 3.0, 0.5, 0.5)


def _acuities(V):
    """(library acuity, oracle acuity) pairs: Sec. 9 anisotropy, Sec. 3.3 display-limited curves."""
    P, F = oracle.PAPER_PIVOTS_DEG, oracle.PAPER_PIVOTS_CPD
    return [(V.vafr_acuity_anisotropic(), oracle.Acuity(P, F, delta=ANISO)),
            (V.vafr_acuity_display_limited(9.0), oracle.Acuity(P, np.minimum(F, 9.0))),
            (V.vafr_acuity_display_limited(18.0), oracle.Acuity(P, np.minimum(F, 18.0)))]


def test_layouts_of_other_acuities_match_oracle(V):
    pose = look_at_pose((0, 0, -3), (0, 0, 0))
    for acu, ora in _acuities(V):
        ref = oracle.lp_layout(ora)
        s = _session(V, 1920, 1080, 100.0, [pose], acuity=acu)
        counts, offs, ecc, n_tex = V.vafr_lp_layout(s)
        assert n_tex == ref.total
        assert np.array_equal(counts, ref.n_col)
        np.testing.assert_allclose(ecc, ref.e_col, rtol=1e-6)
        V.vafr_session_destroy(s)


def test_lp_frame_anisotropic_full(V, torch_mod):
    """Every LP ray of an anisotropic layout (Sec. 9) against the oracle."""
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    acu, ora = _acuities(V)[0]
    lay_a = oracle.lp_layout(ora)
    s = _session(V, d.width, d.height, d.fov_v_deg, d.poses, acuity=acu)
    gaze = (d.width * 0.4, d.height * 0.55)
    V.vafr_set_gaze(s, 0, *gaze)
    lp, ids = _render_lp(V, torch_mod, h, s, lay_a.total)
    rgba, oid, ot, o, dd = oracle.render_lp(sc.tris, sc.albedo, sc.light_dir, lay_a, d.width,
                                            d.height, d.fov_v_deg, gaze, d.poses[0])
    compare_hits_and_colours(sc.tris, o, dd, ids, lp, oid, ot, rgba, 1e-3)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_lp_frame_random1k_full(V, torch_mod, lay):
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    s = _session(V, d.width, d.height, d.fov_v_deg, d.poses)
    gaze = d.gaze[0, 0]
    V.vafr_set_gaze(s, 0, *gaze)
    lp, ids = _render_lp(V, torch_mod, h, s, lay.total)
    rgba, oid, ot, o, dd = oracle.render_lp(sc.tris, sc.albedo, sc.light_dir, lay, d.width,
                                            d.height, d.fov_v_deg, gaze, d.poses[0])
    summ = compare_hits_and_colours(sc.tris, o, dd, ids, lp, oid, ot, rgba, 1e-3)
    assert 0.2 < (ids >= 0).mean() < 0.95
    st = V.vafr_traversal_stats(h, s, 0)
    assert st["rays"] == lay.total and st["hits"] == int((ids >= 0).sum())
    print("random1k LP", summ, st)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


# injection kind -> (status code, status bit that must be set: 1 stack, 2 iteration limit, 4 bad node)
@pytest.mark.parametrize("kind,code,bit", [(1, (-6,), 4), (2, (-4,), 2), (3, (-4, -6), 1)])
def test_traversal_faults_reach_the_status_word(V, torch_mod, lay, kind, code, bit):
    """Failure detection without a GPU fault: a tree corrupted on the host (an
    out-of-range child, a self-loop, a stack-growing self-loop) makes the
    traversal's own bounds, iteration and stack checks stop the rays; the
    session status word reports VAFR_ERR_DEVICE / VAFR_ERR_TIMEOUT, and the
    restored tree renders the same bits as before in the same context.  In the
    stack-growing loop the rays that enter a single root box push nothing and
    reach the iteration limit, which takes precedence in the code; the stack
    bit must still be set."""
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    s = _session(V, d.width, d.height, d.fov_v_deg, d.poses)
    V.vafr_set_gaze(s, 0, *d.gaze[0, 0])
    slot, n_slots, _, _ = lp_slots(V, s)
    lp_ref, ids_ref = _render_lp(V, torch_mod, h, s, lay.total)
    lp = torch_mod.empty((n_slots, 4), dtype=torch_mod.float32, device="cuda")
    ids = torch_mod.empty(n_slots, dtype=torch_mod.int32, device="cuda")
    V.vafr_scene_inject_fault(h, kind)
    V.vafr_render_lp(h, s, 1, lp, ids)
    assert V.vafr_session_check(s) in code
    status = int(V.load().vafr_last_error_message().decode().split("0x")[-1], 16)
    assert status & bit
    assert V.vafr_session_check(s) == 0            # reading clears the word
    # the stopped rays report no hit
    assert (ids.cpu().numpy()[slot] == -1).sum() > (ids_ref == -1).sum()
    V.vafr_scene_inject_fault(h, V.INJECT_NONE)
    lp2, ids2 = _render_lp(V, torch_mod, h, s, lay.total)
    assert np.array_equal(ids2, ids_ref) and np.array_equal(lp2, lp_ref)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_gt_random1k_full(V, torch_mod):
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    s = _session(V, d.width, d.height, d.fov_v_deg, d.poses)
    out = torch_mod.empty((d.height, d.width, 4), dtype=torch_mod.float32, device="cuda")
    ids = torch_mod.empty(d.height * d.width, dtype=torch_mod.int32, device="cuda")
    V.vafr_render_full_gt(h, s, 0, out, ids)
    torch_mod.cuda.synchronize()
    rgba, oid, ot, o, dd = oracle.render_gt(sc.tris, sc.albedo, sc.light_dir, d.width, d.height,
                                            d.fov_v_deg, d.poses[0])
    compare_hits_and_colours(sc.tris, o, dd, ids.cpu().numpy(), out.cpu().numpy().reshape(-1, 4),
                             oid, ot, rgba, 1e-3)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


@pytest.mark.parametrize("kind", ["empty", "single", "quad", "fan", "stack", "axis"])
def test_lp_tiny_scenes(V, torch_mod, lay, kind):
    sc = tiny_scene(kind)
    pose = look_at_pose((0.0, 0.0, -3.0), (0, 0, 0))
    h, keep = device_scene(V, sc, torch_mod)
    s = _session(V, 640, 480, 90.0, [pose])
    V.vafr_set_gaze(s, 0, 320.0, 240.0)
    lp, ids = _render_lp(V, torch_mod, h, s, lay.total)
    rgba, oid, ot, o, dd = oracle.render_lp(sc.tris, sc.albedo, sc.light_dir, lay, 640, 480, 90.0,
                                            (320.0, 240.0), pose)
    compare_hits_and_colours(sc.tris, o, dd, ids, lp, oid, ot, rgba, 1e-3)
    if kind == "empty":
        assert (ids == -1).all()
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


@pytest.fixture(scope="module")
def terrain(V, torch_mod):
    w = workload("terrain4k", frames=240)
    h, keep = device_scene(V, w.scene, torch_mod)
    bvh = oracle.CpuBVH(w.scene.tris)
    yield w, h, bvh
    V.vafr_scene_destroy(h)


@pytest.mark.parametrize("frame", [0, 120, 239])
def test_lp_terrain_full_size_sampled(V, torch_mod, lay, terrain, frame):
    w, h, bvh = terrain
    d, sc = w.displays[0], w.scene
    s = _session(V, d.width, d.height, d.fov_v_deg, d.poses)
    gaze = d.gaze[frame, 0]
    V.vafr_set_gaze(s, 0, *gaze)
    lp, ids = _render_lp(V, torch_mod, h, s, lay.total)
    rng = np.random.default_rng(frame)
    tex = np.sort(rng.choice(lay.total, 65536, replace=False))
    rgba, oid, ot, o, dd = oracle.render_lp(sc.tris, sc.albedo, sc.light_dir, lay, d.width,
                                            d.height, d.fov_v_deg, gaze, d.poses[0], texels=tex,
                                            bvh=bvh)
    compare_hits_and_colours(sc.tris, o, dd, ids[tex], lp[tex], oid, ot, rgba, 1e-3)
    V.vafr_session_destroy(s)


def test_gt_terrain_full_size_sampled(V, torch_mod, terrain):
    w, h, bvh = terrain
    d, sc = w.displays[0], w.scene
    s = _session(V, d.width, d.height, d.fov_v_deg, d.poses)
    out = torch_mod.empty((d.height * d.width, 4), dtype=torch_mod.float32, device="cuda")
    ids = torch_mod.empty(d.height * d.width, dtype=torch_mod.int32, device="cuda")
    V.vafr_render_full_gt(h, s, 0, out, ids)
    torch_mod.cuda.synchronize()
    rng = np.random.default_rng(5)
    pix = np.sort(rng.choice(d.width * d.height, 65536, replace=False))
    rgba, oid, ot, o, dd = oracle.render_gt(sc.tris, sc.albedo, sc.light_dir, d.width, d.height,
                                            d.fov_v_deg, d.poses[0], pixels=pix, bvh=bvh)
    compare_hits_and_colours(sc.tris, o, dd, ids.cpu().numpy()[pix], out.cpu().numpy()[pix], oid,
                             ot, rgba, 1e-3)
    V.vafr_session_destroy(s)


def test_gt_terrain_16k_sampled(V, torch_mod, terrain):
    """The largest display of the resolution sweep (15360 x 8640, 132.7 M rays in
    one launch): sampled pixels against the oracle's CPU-BVH cast."""
    w, h, bvh = terrain
    d, sc = w.displays[0], w.scene
    W, H = 15360, 8640
    s = _session(V, W, H, d.fov_v_deg, d.poses)
    out = torch_mod.empty((H * W, 4), dtype=torch_mod.float32, device="cuda")
    ids = torch_mod.empty(H * W, dtype=torch_mod.int32, device="cuda")
    V.vafr_render_full_gt(h, s, 0, out, ids)
    torch_mod.cuda.synchronize()
    rng = np.random.default_rng(16)
    pix = np.sort(rng.choice(W * H, 65536, replace=False))
    sel = torch_mod.from_numpy(pix).cuda()
    got_ids, got = ids[sel].cpu().numpy(), out[sel].cpu().numpy()
    del out, ids
    rgba, oid, ot, o, dd = oracle.render_gt(sc.tris, sc.albedo, sc.light_dir, W, H, d.fov_v_deg,
                                            d.poses[0], pixels=pix, bvh=bvh)
    compare_hits_and_colours(sc.tris, o, dd, got_ids, got, oid, ot, rgba, 1e-3)
    V.vafr_session_destroy(s)


def test_lp_fp16_binocular_and_gaze_outside(V, torch_mod, lay):
    sc = random_triangles_scene(1024, seed=1001)
    head = look_at_pose((0.0, 0.2, -3.0), (0, 0, 0))
    from workloads.views import eye_pair_poses
    poses = eye_pair_poses(head, 0.063)
    W, H = 1920, 1080
    h, keep = device_scene(V, sc, torch_mod)
    s = _session(V, W, H, 100.0, poses, lp_fmt=1, disp_fmt=1)
    gazes = [(-250.0, 1300.5), (W + 0.25, -3.75)]   # both outside the display
    for e, g in enumerate(gazes):
        V.vafr_set_gaze(s, e, *g)
    lp, ids = _render_lp(V, torch_mod, h, s, lay.total, eye_mask=3, fp16=True)
    rng = np.random.default_rng(11)
    for e in range(2):
        tex = np.sort(rng.choice(lay.total, 50000, replace=False))
        rgba, oid, ot, o, dd = oracle.render_lp(sc.tris, sc.albedo, sc.light_dir, lay, W, H, 100.0,
                                                gazes[e], poses[e], texels=tex)
        # FP16 RNE: relative 2^-11 of values <= 1, plus the FP32 1e-3
        compare_hits_and_colours(sc.tris, o, dd, ids[e * lay.total + tex],
                                 lp[e * lay.total + tex], oid, ot, rgba, 1e-3 + 2.0 ** -11)
    # each eye alone is bitwise the same as both together
    for e in range(2):
        lp1, ids1 = _render_lp(V, torch_mod, h, s, lay.total, eye_mask=1 << e, fp16=True)
        assert np.array_equal(ids1, ids[e * lay.total:(e + 1) * lay.total])
        assert np.array_equal(lp1, lp[e * lay.total:(e + 1) * lay.total])
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


@pytest.fixture(scope="module")
def objects8k(V, torch_mod):
    w = workload("objects8k", frames=240)
    h, keep = device_scene(V, w.scene, torch_mod)
    bvh = oracle.CpuBVH(w.scene.tris)
    yield w, h, bvh
    V.vafr_scene_destroy(h)


@pytest.mark.parametrize("frame,variant", [(0, 4), (150, 4), (150, 2), (150, 6), (150, 7)])
def test_lp_objects8k_binocular_sampled(V, torch_mod, lay, objects8k, frame, variant):
    """The 8K binocular workload at full size (1,998,088 triangles, FP16 LP, both
    eyes in one launch, each eye on its own gaze trajectory) in the render
    variants the autotuner picks for it (4: plain order capped at 64
    registers; 7: longest-first order at 7 blocks per SM), the uncapped plain
    order (2) and the longest-first order (6): sampled texels of both eyes
    against the oracle's CPU-BVH cast."""
    w, h, bvh = objects8k
    d, sc = w.displays[0], w.scene
    s = _session(V, d.width, d.height, d.fov_v_deg, d.poses, lp_fmt=1, disp_fmt=1)
    for e in range(2):
        V.vafr_set_gaze(s, e, *d.gaze[frame, e])
    V.vafr_session_tuning(s, (variant, 2))
    lp, ids = _render_lp(V, torch_mod, h, s, lay.total, eye_mask=3, fp16=True)
    rng = np.random.default_rng(frame + variant)
    tex = np.sort(rng.choice(lay.total, 65536, replace=False))
    for e in range(2):
        rgba, oid, ot, o, dd = oracle.render_lp(sc.tris, sc.albedo, sc.light_dir, lay, d.width,
                                                d.height, d.fov_v_deg, d.gaze[frame, e], d.poses[e],
                                                texels=tex, bvh=bvh)
        compare_hits_and_colours(sc.tris, o, dd, ids[e * lay.total + tex], lp[e * lay.total + tex],
                                 oid, ot, rgba, 1e-3 + 2.0 ** -11)
    V.vafr_session_destroy(s)


def test_lp_independent_of_resolution(V, torch_mod, lay):
    # Sec. 3.2.2: same FOV, pose and gaze direction -> same LP buffer at 1080p and 8K
    sc = random_triangles_scene(1024, seed=1001)
    pose = look_at_pose((0.0, 0.0, -3.0), (0, 0, 0))
    h, keep = device_scene(V, sc, torch_mod)
    outs = []
    for W, H, g in [(1920, 1080, (1060.0, 490.0)), (7680, 4320, (4240.0, 1960.0))]:
        s = _session(V, W, H, 100.0, [pose])
        V.vafr_set_gaze(s, 0, *g)
        outs.append(_render_lp(V, torch_mod, h, s, lay.total))
        V.vafr_session_destroy(s)
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][0], outs[1][0])
    V.vafr_scene_destroy(h)


def test_invalid_arguments(V, torch_mod):
    pose = look_at_pose((0.0, 0.0, -3.0), (0, 0, 0))
    with pytest.raises(V.VafrError):
        _session(V, 0, 100, 90.0, [pose])
    with pytest.raises(V.VafrError):
        _session(V, 100, 100, 180.0, [pose])
    bad = V.make_acuity([0, 10, 5], [40, 10, 6])
    with pytest.raises(V.VafrError):
        _session(V, 100, 100, 90.0, [pose], acuity=bad)
    s = _session(V, 100, 100, 90.0, [pose])
    with pytest.raises(V.VafrError):
        V.vafr_set_gaze(s, 0, math.nan, 1.0)
    with pytest.raises(V.VafrError):
        V.vafr_set_gaze(s, 1, 1.0, 1.0)
    lp = torch_mod.empty((10, 4), device="cuda")
    sc = random_triangles_scene(8, seed=1)
    h, keep = device_scene(V, sc, torch_mod)
    with pytest.raises(V.VafrError):   # gaze never set
        V.vafr_render_lp(h, s, 1, lp)
    V.vafr_set_gaze(s, 0, 50.0, 50.0)
    with pytest.raises(V.VafrError):   # eye mask outside the session
        V.vafr_render_lp(h, s, 2, lp)
    with pytest.raises(V.VafrError):   # unknown injection
        V.vafr_scene_inject_fault(h, 7)
    one, keep1 = device_scene(V, random_triangles_scene(1, seed=2), torch_mod)
    with pytest.raises(V.VafrError):   # no tree to corrupt
        V.vafr_scene_inject_fault(one, V.INJECT_LOOP)
    V.vafr_scene_destroy(one)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_axis_parallel_rays_stay_cheap(V, torch_mod, lay, terrain):
    """Rays exactly parallel to a world axis (cos phi = 0 at the centre gaze) from
    an eye whose origin is off that axis's plane must still cull boxes: no ray
    may wander through the whole tree (that once made one launch 7x slower)."""
    w, h, bvh = terrain
    d = w.displays[0]
    from workloads.views import eye_pair_poses
    left, _ = eye_pair_poses(d.poses[0], 0.063)
    s = _session(V, d.width, d.height, d.fov_v_deg, [left])
    V.vafr_set_gaze(s, 0, d.width / 2, d.height / 2)
    st = V.vafr_traversal_stats(h, s, 0)
    assert st["max_nodes"] < 2000, st
    lp, ids = _render_lp(V, torch_mod, h, s, lay.total)
    rng = np.random.default_rng(3)
    tex = np.sort(rng.choice(lay.total, 20000, replace=False))
    rgba, oid, ot, o, dd = oracle.render_lp(w.scene.tris, w.scene.albedo, w.scene.light_dir, lay,
                                            d.width, d.height, d.fov_v_deg,
                                            (d.width / 2, d.height / 2), left, texels=tex, bvh=bvh)
    compare_hits_and_colours(w.scene.tris, o, dd, ids[tex], lp[tex], oid, ot, rgba, 1e-3)
    V.vafr_session_destroy(s)
