"""GPU FXAA inside the LP buffer (Sec. 3.4, Sec. 7) against the oracle, on LP
buffers the oracle renders (never on CUDA-produced data), and its place in
render_frame, batches and captured graphs."""

import numpy as np
import pytest

import oracle
from parity import check_guards, device_scene, lp_slots, to_device_lp
from workloads import random_triangles_scene, workload
from workloads.views import eye_pair_poses, look_at_pose

pytestmark = pytest.mark.gpu

POSE = look_at_pose((0.0, 0.0, -3.0), (0, 0, 0))


def _fxaa(V, torch, s, lp_compact, fp16=False):
    dt = torch.float16 if fp16 else torch.float32
    lp = torch.from_numpy(np.ascontiguousarray(to_device_lp(lp_compact, V, s))).to(dt).cuda()
    out = torch.full_like(lp, float("nan"))
    V.vafr_fxaa_lp(s, 0, lp, out)
    torch.cuda.synchronize()
    slot, _, counts, offs = lp_slots(V, s)
    o = out.float().cpu().numpy()
    check_guards(o, counts, offs)
    return o[slot]


@pytest.fixture(scope="module")
def rendered():
    """An oracle LP render of the 1,024-triangle scene: edges everywhere."""
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    lay = oracle.lp_layout()
    rgba, _, _, _, _ = oracle.render_lp(sc.tris, sc.albedo, sc.light_dir, lay, d.width, d.height,
                                        d.fov_v_deg, d.gaze[0, 0], d.poses[0])
    return lay, rgba.astype(np.float32)


def test_fxaa_matches_oracle_fp32(V, torch_mod, rendered):
    lay, lp = rendered
    s = V.vafr_session_create(V.make_session_desc(512, 512, 90.0, [POSE]))
    got = _fxaa(V, torch_mod, s, lp)
    ref = oracle.fxaa_lp(lp.astype(np.float64), lay)
    changed = np.any(ref != lp, 1).mean()
    print(f"fxaa: {changed:.3f} of texels blended, max err {np.abs(got - ref).max():.2e}")
    assert 0.01 < changed < 0.9
    assert np.abs(got - ref).max() < 1e-5
    V.vafr_session_destroy(s)


def test_fxaa_matches_oracle_fp16_and_blocks(V, torch_mod):
    lay = oracle.lp_layout()
    rng = np.random.default_rng(3)
    col = np.repeat(np.arange(lay.n_cols), lay.n_col)
    j = np.arange(lay.total) - lay.off_col[col]
    # angular-radial blocks: edges along both grid directions, ragged columns
    blocks = ((col // 37) + (j * 7 // np.maximum(lay.n_col[col], 1))) % 2
    lp = np.stack([blocks * 0.9 + 0.05, blocks * 0.5 + rng.uniform(0, 0.05, lay.total),
                   1 - blocks * 0.8, np.ones(lay.total)], 1).astype(np.float16)
    s = V.vafr_session_create(V.make_session_desc(512, 512, 90.0, [POSE], 1, 1))
    got = _fxaa(V, torch_mod, s, lp, fp16=True)
    ref = oracle.fxaa_lp(lp.astype(np.float64), lay)
    assert np.any(ref != lp.astype(np.float64))
    assert np.abs(got - ref).max() < 1e-5 + 2.0 ** -11
    V.vafr_session_destroy(s)


def test_fxaa_constant_is_exact(V, torch_mod):
    lay = oracle.lp_layout()
    lp = np.tile(np.float32([0.2, 0.4, 0.6, 1.0]), (lay.total, 1))
    s = V.vafr_session_create(V.make_session_desc(512, 512, 90.0, [POSE]))
    assert np.array_equal(_fxaa(V, torch_mod, s, lp), lp)
    V.vafr_session_destroy(s)


def test_fxaa_anisotropic_layout(V, torch_mod, rendered):
    P, F = oracle.PAPER_PIVOTS_DEG, oracle.PAPER_PIVOTS_CPD
    ora = oracle.Acuity(P, F, delta=(1, 5 / 6, 2 / 3, 0.5, 0.5))
    lay_a = oracle.lp_layout(ora)
    rng = np.random.default_rng(8)
    lp = (rng.uniform(0, 1, (lay_a.total, 4)) * (rng.random((lay_a.total, 1)) < 0.3)).astype(np.float32)
    s = V.vafr_session_create(V.make_session_desc(512, 512, 90.0, [POSE],
                                                  acuity=V.vafr_acuity_anisotropic()))
    got = _fxaa(V, torch_mod, s, lp)
    ref = oracle.fxaa_lp(lp.astype(np.float64), lay_a)
    assert np.abs(got - ref).max() < 1e-5
    V.vafr_session_destroy(s)


def _setup_scene(V, torch):
    sc = random_triangles_scene(2000, seed=21)
    return device_scene(V, sc, torch)


def test_render_frame_applies_fxaa(V, torch_mod):
    """render_frame of an FXAA session == render_lp -> fxaa_lp -> reconstruct."""
    h, keep = _setup_scene(V, torch_mod)
    poses = eye_pair_poses(look_at_pose((0.0, 0.3, -3.2), (0, 0, 0)), 0.063)
    W, H = 960, 540
    s = V.vafr_session_create(V.make_session_desc(W, H, 100.0, poses, lp_fxaa=True))
    for e, g in enumerate([(400.0, 300.0), (520.5, 250.25)]):
        V.vafr_set_gaze(s, e, *g)
    got = torch_mod.empty((2, H, W, 4), device="cuda")
    V.vafr_render_frame(h, s, got)
    lpb, dpb = V.vafr_session_sizes(s)
    lp = torch_mod.empty(2 * lpb, dtype=torch_mod.uint8, device="cuda")
    aa = torch_mod.empty(2 * lpb, dtype=torch_mod.uint8, device="cuda")
    ref = torch_mod.empty((2, H, W, 4), device="cuda")
    V.vafr_render_lp(h, s, 3, lp)
    for e in range(2):
        V.vafr_fxaa_lp(s, e, lp[e * lpb:], aa[e * lpb:])
        V.vafr_reconstruct(s, e, aa[e * lpb:], ref[e])
    torch_mod.cuda.synchronize()
    assert torch_mod.equal(got, ref)
    assert not torch_mod.equal(lp, aa)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_batch_and_graph_with_fxaa(V, torch_mod):
    """A batch mixing FXAA and plain sessions, launched directly and replayed from
    a captured graph, equals the single-session calls."""
    h, keep = _setup_scene(V, torch_mod)
    poses = eye_pair_poses(look_at_pose((0.0, 0.3, -3.2), (0, 0, 0)), 0.063)
    sess, frames, bufs = [], [], []
    for k, (W, H, aa) in enumerate([(640, 360, True), (333, 211, False), (1280, 720, True)]):
        s = V.vafr_session_create(V.make_session_desc(W, H, 100.0, poses, lp_fxaa=aa))
        lpb, dpb = V.vafr_session_sizes(s)
        for e in range(2):
            V.vafr_set_gaze(s, e, W * (0.3 + 0.2 * e), H * (0.5 - 0.1 * k))
            b = [torch_mod.zeros(n, dtype=torch_mod.uint8, device="cuda") for n in (lpb, lpb, dpb)]
            bufs.append(b)
            frames.append((s, e, b[0], b[2], b[1]) if aa else (s, e, b[0], b[2]))
        sess.append((s, aa, lpb, dpb))

    def single():
        outs = []
        for s, aa, lpb, dpb in sess:
            lp = torch_mod.empty(2 * lpb, dtype=torch_mod.uint8, device="cuda")
            V.vafr_render_lp(h, s, 3, lp)
            for e in range(2):
                src = lp[e * lpb:]
                if aa:
                    src = torch_mod.empty(lpb, dtype=torch_mod.uint8, device="cuda")
                    V.vafr_fxaa_lp(s, e, lp[e * lpb:], src)
                d = torch_mod.empty(dpb, dtype=torch_mod.uint8, device="cuda")
                V.vafr_reconstruct(s, e, src, d)
                outs.append(d)
        torch_mod.cuda.synchronize()
        return [o.cpu() for o in outs]

    ref = single()
    bt = V.vafr_batch_create(h, 16)
    V.vafr_batch_render(bt, frames)
    torch_mod.cuda.synchronize()
    for b, r in zip(bufs, ref):
        assert torch_mod.equal(b[2].cpu(), r)
    V.vafr_batch_capture(bt, frames)
    for it in range(2):
        for s, aa, lpb, dpb in sess:
            V.vafr_set_gaze(s, 0, 100.0 + 50 * it, 80.0)
            V.vafr_set_gaze(s, 1, 150.0, 60.0 + 30 * it)
        V.vafr_batch_replay(bt)
        torch_mod.cuda.synchronize()
        ref = single()
        for b, r in zip(bufs, ref):
            assert torch_mod.equal(b[2].cpu(), r)
    with pytest.raises(V.VafrError):   # an FXAA session's frame without lp_aa
        V.vafr_batch_render(bt, [frames[0][:4]])
    V.vafr_batch_destroy(bt)
    for s, *_ in sess:
        V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)
