"""GPU inverse-mapping reconstruction against the FP64 oracle, on seeded LP inputs
(never on CUDA-produced data), and the whole VaFR frame end to end."""

import math

import numpy as np
import pytest

import oracle
from parity import device_scene, lp_slots, to_device_lp
from workloads import workload
from workloads.views import look_at_pose

pytestmark = pytest.mark.gpu

POSE = look_at_pose((0.0, 0.0, -3.0), (0, 0, 0))


@pytest.fixture(scope="module")
def lay():
    return oracle.lp_layout()


def _recon(V, torch, W, H, fov, gaze, lp_np, lp_fmt=0, disp_fmt=0, variant=None, acuity=None):
    s = V.vafr_session_create(V.make_session_desc(W, H, fov, [POSE], lp_fmt, disp_fmt, acuity))
    V.vafr_set_gaze(s, 0, *gaze)
    dt = torch.float16 if lp_fmt else torch.float32
    lp = torch.from_numpy(np.ascontiguousarray(to_device_lp(lp_np, V, s))).to(dt).cuda()
    out = torch.empty((H, W, 4), dtype=torch.float16 if disp_fmt else torch.float32, device="cuda")
    if variant is not None:
        V.vafr_session_tuning(s, (0, variant))
    V.vafr_reconstruct(s, 0, lp, out)
    torch.cuda.synchronize()
    res = out.float().cpu().numpy().reshape(-1, 4)
    V.vafr_session_destroy(s)
    return res


@pytest.mark.parametrize("W,H,gaze", [(640, 360, (200.3, 100.9)), (641, 357, (320.5, 178.5)),
                                      (500, 300, (0.0, 0.0)), (500, 300, (-120.0, 410.25)),
                                      (512, 512, (512.0, 512.0))])
def test_random_lp_all_pixels(V, torch_mod, lay, W, H, gaze):
    rng = np.random.default_rng(W * 7 + H)
    lp = rng.uniform(0, 1, (lay.total, 4)).astype(np.float32)
    got = _recon(V, torch_mod, W, H, 100.0, gaze, lp)
    ref = oracle.reconstruct(lp.astype(np.float64), lay, W, H, 100.0, gaze)
    err = np.abs(got - ref).max()
    print(f"recon {W}x{H} gaze {gaze}: max err {err:.2e}")
    assert err < 1e-3


@pytest.mark.parametrize("which", ["anisotropic", "display9"])
def test_other_acuity_layouts(V, torch_mod, which):
    """Reconstruction over the anisotropic (Sec. 9) and display-limited (Sec. 3.3)
    layouts against the oracle, every pixel."""
    P, F = oracle.PAPER_PIVOTS_DEG, oracle.PAPER_PIVOTS_CPD
    if which == "anisotropic":
        acu, ora = V.vafr_acuity_anisotropic(), oracle.Acuity(P, F, delta=(1, 5 / 6, 2 / 3, 0.5, 0.5))
    else:
        acu, ora = V.vafr_acuity_display_limited(9.0), oracle.Acuity(P, np.minimum(F, 9.0))
    lay_a = oracle.lp_layout(ora)
    rng = np.random.default_rng(17)
    lp = rng.uniform(0, 1, (lay_a.total, 4)).astype(np.float32)
    W, H, gaze = 801, 449, (300.5, 260.25)
    got = _recon(V, torch_mod, W, H, 100.0, gaze, lp, acuity=acu)
    ref = oracle.reconstruct(lp.astype(np.float64), lay_a, W, H, 100.0, gaze, acuity=ora)
    assert np.abs(got - ref).max() < 1e-3


def test_constant_lp_is_exact(V, torch_mod, lay):
    lp = np.tile(np.float32([0.25, 0.5, 0.75, 1.0]), (lay.total, 1))
    got = _recon(V, torch_mod, 777, 333, 90.0, (100.0, 200.0), lp)
    assert np.array_equal(got, np.broadcast_to(lp[0], got.shape))


def test_analytic_texture(V, torch_mod, lay):
    # F(e, phi) at texel centres: the smooth field reconstructs to 1e-5 of the oracle
    e_c = np.repeat(lay.e_col, lay.n_col)
    col = np.repeat(np.arange(lay.n_cols), lay.n_col)
    j = np.arange(lay.total) - lay.off_col[col]
    phi = np.radians((j + 0.5) / lay.n_col[col] * 360.0)
    lp = np.stack([e_c / 60, 0.5 + 0.5 * np.cos(phi), 0.5 + 0.5 * np.sin(phi),
                   np.ones_like(phi)], 1)
    W, H, gaze = 1280, 720, (700.25, 300.75)
    got = _recon(V, torch_mod, W, H, 100.0, gaze, lp.astype(np.float32))
    ref = oracle.reconstruct(lp.astype(np.float32).astype(np.float64), lay, W, H, 100.0, gaze)
    assert np.abs(got - ref).max() < 1e-5


def test_fp16_formats(V, torch_mod, lay):
    rng = np.random.default_rng(9)
    lp = rng.uniform(0, 1, (lay.total, 4)).astype(np.float16)
    W, H, gaze = 960, 540, (480.0, 270.0)
    got = _recon(V, torch_mod, W, H, 100.0, gaze, lp, lp_fmt=1, disp_fmt=1)
    ref = oracle.reconstruct(lp.astype(np.float64), lay, W, H, 100.0, gaze)
    assert np.abs(got - ref).max() < 1e-3 + 2.0 ** -11


@pytest.mark.parametrize("fmts", [(0, 0), (1, 1), (1, 0), (0, 1)])
def test_tile_variants_identical(V, torch_mod, lay, fmts):
    """Row tiles and column-run tiles of every shape give the same bits, for
    every LP / display format pair, on a ragged display (odd width and height)."""
    rng = np.random.default_rng(4)
    lp = rng.uniform(0, 1, (lay.total, 4)).astype(np.float32)
    n_variants = V.vafr_tuning_space()[1]
    outs = [_recon(V, torch_mod, 803, 451, 100.0, (400.0, 225.0), lp, lp_fmt=fmts[0],
                   disp_fmt=fmts[1], variant=v) for v in range(n_variants)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("W,H", [(3840, 2160), (7680, 4320)])
def test_full_size_sampled(V, torch_mod, lay, W, H):
    rng = np.random.default_rng(W)
    lp = rng.uniform(0, 1, (lay.total, 4)).astype(np.float32)
    gaze = (W * 0.37, H * 0.61)
    got = _recon(V, torch_mod, W, H, 100.0, gaze, lp)
    pix = rng.choice(W * H, 65536, replace=False)
    ref = oracle.reconstruct(lp.astype(np.float64), lay, W, H, 100.0, gaze, pix)
    assert np.abs(got[pix] - ref).max() < 1e-3


@pytest.mark.parametrize("disp_fmt", [0, 1])
def test_16k_sampled(V, torch_mod, lay, disp_fmt):
    """15360 x 8640 (the sweep's largest display, 132.7 M pixels in one launch),
    FP32 or FP16 display: sampled pixels against the oracle."""
    W, H = 15360, 8640
    rng = np.random.default_rng(15360 + disp_fmt)
    lp_np = rng.uniform(0, 1, (lay.total, 4)).astype(np.float32)
    gaze = (W * 0.58, H * 0.33)
    s = V.vafr_session_create(V.make_session_desc(W, H, 100.0, [POSE], 0, disp_fmt))
    V.vafr_set_gaze(s, 0, *gaze)
    lp = torch_mod.from_numpy(np.ascontiguousarray(to_device_lp(lp_np, V, s))).cuda()
    dt = torch_mod.float16 if disp_fmt else torch_mod.float32
    out = torch_mod.empty((H * W, 4), dtype=dt, device="cuda")
    V.vafr_reconstruct(s, 0, lp, out)
    torch_mod.cuda.synchronize()
    pix = np.sort(rng.choice(W * H, 65536, replace=False))
    got = out[torch_mod.from_numpy(pix).cuda()].float().cpu().numpy()
    del out
    V.vafr_session_destroy(s)
    ref = oracle.reconstruct(lp_np.astype(np.float64), lay, W, H, 100.0, gaze, pix)
    tol = 1e-3 + (2.0 ** -11 if disp_fmt else 0.0)
    assert np.abs(got - ref).max() < tol


@pytest.mark.parametrize("variant", [1, 2, 8])
def test_8k_fp16_sampled(V, torch_mod, lay, variant):
    """One eye of the 8K binocular configuration (FP16 LP, FP16 display) in the
    reconstruct variants the autotuner picks (2 at 8K, 1 at 4K): sampled pixels
    against the oracle fed the same FP16-rounded LP texels."""
    W, H = 7680, 4320
    rng = np.random.default_rng(8 + variant)
    lp = rng.uniform(0, 1, (lay.total, 4)).astype(np.float16).astype(np.float32)
    gaze = (W * 0.44, H * 0.57)
    got = _recon(V, torch_mod, W, H, 100.0, gaze, lp, lp_fmt=1, disp_fmt=1, variant=variant)
    pix = rng.choice(W * H, 65536, replace=False)
    ref = oracle.reconstruct(lp.astype(np.float64), lay, W, H, 100.0, gaze, pix)
    assert np.abs(got[pix] - ref).max() < 1e-3 + 2.0 ** -11


def test_whole_frame_random1k(V, torch_mod, lay):
    """render_frame (LP render + reconstruct) vs the oracle's LP render + reconstruct;
    pixels whose filter footprint touches a tie texel are excluded."""
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, d.poses))
    gaze = d.gaze[0, 0]
    V.vafr_set_gaze(s, 0, *gaze)
    host = np.zeros((d.height, d.width, 4), np.float32)
    V.vafr_render_frame(h, s, host)                        # host output: D2H inside the call
    slot, n_slots, _, _ = lp_slots(V, s)
    lp = torch_mod.empty((n_slots, 4), device="cuda")
    ids = torch_mod.empty(n_slots, dtype=torch_mod.int32, device="cuda")
    V.vafr_render_lp(h, s, 1, lp, ids)
    torch_mod.cuda.synchronize()
    rgba, oid, _, _, _ = oracle.render_lp(sc.tris, sc.albedo, sc.light_dir, lay, d.width,
                                          d.height, d.fov_v_deg, gaze, d.poses[0])
    ref = oracle.reconstruct(rgba, lay, d.width, d.height, d.fov_v_deg, gaze)
    bad = (ids.cpu().numpy()[slot] != oid).astype(np.float64)[:, None]
    touch = oracle.reconstruct(bad, lay, d.width, d.height, d.fov_v_deg, gaze)[:, 0] > 0
    got = host.reshape(-1, 4)
    assert touch.mean() < 0.01
    assert np.abs(got[~touch] - ref[~touch]).max() < 1e-3
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_render_frame_host_outputs_match_device(V, torch_mod, lay):
    """vafr_render_frame into device memory, pinned host memory (written by the
    kernel directly) and pageable host memory (copied): bitwise identical."""
    torch = torch_mod
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch)
    s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, d.poses))
    V.vafr_set_gaze(s, 0, 200.25, 300.5)
    dev = torch.empty((d.height, d.width, 4), dtype=torch.float32, device="cuda")
    pinned = torch.zeros((d.height, d.width, 4), dtype=torch.float32, pin_memory=True)
    pageable = np.zeros((d.height, d.width, 4), np.float32)
    V.vafr_render_frame(h, s, dev)
    V.vafr_render_frame(h, s, pinned)
    V.vafr_render_frame(h, s, pageable)
    torch.cuda.synchronize()
    ref = dev.cpu().numpy()
    assert np.array_equal(pinned.numpy(), ref)
    assert np.array_equal(pageable, ref)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


def test_render_frame_pinned_host_equals_device(V, torch_mod):
    """render_frame into page-locked host memory (device display + one copy)
    holds the bytes of render_frame into device memory."""
    w = workload("random1k")
    d, sc = w.displays[0], w.scene
    h, keep = device_scene(V, sc, torch_mod)
    s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, d.poses))
    V.vafr_set_gaze(s, 0, *d.gaze[0, 0])
    dev = torch_mod.empty((d.height, d.width, 4), device="cuda")
    pin = torch_mod.zeros((d.height, d.width, 4), pin_memory=True)
    V.vafr_render_frame(h, s, dev)
    V.vafr_render_frame(h, s, pin)
    torch_mod.cuda.synchronize()
    assert torch_mod.equal(dev.cpu(), pin)
    V.vafr_session_destroy(s)
    V.vafr_scene_destroy(h)


@pytest.mark.parametrize("W,H,fmt", [(3840, 2160, 0), (7680, 4320, 1)])
def test_staged_tiles_equal_plain_runs_full_size(V, torch_mod, lay, W, H, fmt):
    """Variant 8 stages each tile's LP footprint in shared memory; at the bench's
    display sizes (4K FP32, 8K FP16) and a gaze near a corner and one in the
    middle, every pixel equals the plain column run's bit for bit."""
    rng = np.random.default_rng(W + fmt)
    lp = rng.uniform(0, 1, (lay.total, 4)).astype(np.float16 if fmt else np.float32)
    for gaze in ((W * 0.5 + 0.37, H * 0.5 - 0.21), (W * 0.07, H * 0.93)):
        a = _recon(V, torch_mod, W, H, 100.0, gaze, lp, lp_fmt=fmt, disp_fmt=fmt, variant=2)
        b = _recon(V, torch_mod, W, H, 100.0, gaze, lp, lp_fmt=fmt, disp_fmt=fmt, variant=8)
        assert np.array_equal(a, b)
