"""GPU path tracing into the LP buffer (Sec. 8) against the FP64 oracle: path
signatures (hit id per segment, shadow-visibility mask) identical except
classified ties, radiance within FP32 rounding where the signatures agree."""

import numpy as np
import pytest

import oracle
from parity import check_guards, classify, device_scene, lp_slots
from workloads import workload

pytestmark = pytest.mark.gpu

D = 3


def _render_pt(V, torch, h, s, seed, depth=D, eye_mask=1, fp16=False):
    slot, n_slots, counts, offs = lp_slots(V, s)
    eyes = bin(eye_mask).count("1")
    lp = torch.empty((eyes * n_slots, 4), dtype=torch.float16 if fp16 else torch.float32, device="cuda")
    sig = torch.full((eyes * n_slots, depth + 2), -7, dtype=torch.int32, device="cuda")
    V.vafr_render_lp_pt(h, s, eye_mask, lp, seed, depth, sig)
    torch.cuda.synchronize()
    assert V.vafr_session_check(s) == 0
    lp = lp.float().cpu().numpy().reshape(eyes, n_slots, 4)
    sig = sig.cpu().numpy().reshape(eyes, n_slots, depth + 2)
    for e in range(eyes):
        check_guards(lp[e], counts, offs)
    return lp[:, slot], sig[:, slot]


def _compare(sc, lay, got_rgba, got_sig, ref_rgba, ref_sig, seg, tex, tol):
    """Signatures equal except ties; radiance within tol where they agree."""
    n = len(tex)
    same = np.all(got_sig == ref_sig, axis=1)
    hit_diff = np.any(got_sig[:, :-1] != ref_sig[:, :-1], axis=1)
    shadow_only = ~same & ~hit_diff
    # first segment whose hit differs, classified on the oracle's FP64 ray
    idx = np.flatnonzero(hit_diff)
    ties = errs = 0
    for q in idx:
        k = int(np.flatnonzero(got_sig[q, :-1] != ref_sig[q, :-1])[0])
        o, d = seg[q, k, :3][None], seg[q, k, 3:][None]
        oid = ref_sig[q, k:k + 1].astype(np.int32)
        ot = oracle.ray_tri_t(sc.tris, oid, o, d) if oid[0] >= 0 else np.array([np.inf])
        t_, e_, _ = classify(sc.tris, o, d, got_sig[q, k:k + 1], oid, ot)
        ties += t_
        errs += e_
    cerr = np.abs(got_rgba[same, :3] - ref_rgba[same, :3]).max(initial=0.0)
    # rays the oracle traced: path segments (a hit id or -1 for a miss) and
    # shadow rays (bits 16-23 of the last signature word)
    segs = int((ref_sig[:, :-1] >= -1).sum())
    shadow = int(np.unpackbits(((ref_sig[:, -1] >> 16) & 0xff).astype(np.uint8)).sum())
    n_rays = segs + shadow
    summ = dict(n=n, rays=n_rays, same=float(same.mean()), hit_ties=ties, hit_errors=errs,
                shadow_only=int(shadow_only.sum()), colour_err=float(cerr))
    print("path parity", summ)
    assert errs == 0, summ
    # the ray-edge tie budget, 0.01 % of the rays cast; a shadow ray whose
    # visibility differs counts as one of its ties
    assert ties + shadow_only.sum() <= 1e-4 * n_rays, summ
    assert cerr <= tol, summ
    return summ


def test_path_trace_random1k_full(V, torch_mod):
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, d.poses))
    gaze = d.gaze[0, 0]
    V.vafr_set_gaze(s, 0, *gaze)
    lay = oracle.lp_layout()
    got, sig = _render_pt(V, torch_mod, h, s, seed=1234)
    tex = np.arange(lay.total)
    ref, rsig, seg = oracle.path_trace_lp(sc.tris, sc.albedo, sc.light_dir, lay, d.width, d.height,
                                          d.fov_v_deg, gaze, d.poses[0], seed=1234, max_diffuse=D,
                                          segments=True)
    summ = _compare(sc, lay, got[0], sig[0], ref, rsig, seg, tex, 1e-4)
    assert (rsig[:, 1] >= 0).mean() > 0.05          # bounces do hit geometry
    # deterministic per seed, different across seeds
    again, sig2 = _render_pt(V, torch_mod, h, s, seed=1234)
    assert np.array_equal(again, got) and np.array_equal(sig2, sig)
    other, _ = _render_pt(V, torch_mod, h, s, seed=1235)
    assert not np.array_equal(other, got)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_path_trace_terrain_sampled_fp16_binocular(V, torch_mod):
    w = workload("terrain4k", frames=8)
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    from workloads.views import eye_pair_poses
    poses = eye_pair_poses(d.poses[0], 0.063)
    s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, poses, 1, 1))
    gazes = [d.gaze[3, 0], d.gaze[5, 0]]
    for e, g in enumerate(gazes):
        V.vafr_set_gaze(s, e, *g)
    lay = oracle.lp_layout()
    got, sig = _render_pt(V, torch_mod, h, s, seed=99, eye_mask=3, fp16=True)
    bvh = oracle.CpuBVH(sc.tris)
    rng = np.random.default_rng(4)
    for e in range(2):
        tex = np.sort(rng.choice(lay.total, 30000, replace=False))
        ref, rsig, seg = oracle.path_trace_lp(sc.tris, sc.albedo, sc.light_dir, lay, d.width, d.height,
                                              d.fov_v_deg, gazes[e], poses[e], seed=99, max_diffuse=D,
                                              texels=tex, bvh=bvh, segments=True)
        # FP16 storage: relative 2^-11 of values up to ~3, plus the FP32 budget
        _compare(sc, lay, got[e][tex], sig[e][tex], ref, rsig, seg, tex, 1e-4 + 3 * 2.0 ** -11)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_path_trace_depth_zero_is_direct_light_only(V, torch_mod):
    """max_diffuse = 0: no bounce is traced and every signature says so."""
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, d.poses))
    V.vafr_set_gaze(s, 0, *d.gaze[0, 0])
    got, sig = _render_pt(V, torch_mod, h, s, seed=5, depth=0)
    assert sig.shape[-1] == 2
    assert np.all(np.isin(sig[0, :, 1], [0, 1 << 16, (1 << 16) | 1]))
    hit = sig[0, :, 0] >= 0
    assert np.all(got[0, hit & ((sig[0, :, 1] & 1) == 0), :3] == 0)   # unlit hits are black
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)
