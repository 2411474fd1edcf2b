"""Benchmark of the VaFR ray-casting hot path on one GB300 (or N, one per rank).

Workload (default ``objects8k``, the largest single-GPU configuration):
binocular 7680x4320 per eye, 63 mm IPD, 100 deg vertical FOV, a 240-frame
seeded saccade gaze trajectory per eye, a 1,998,088-triangle scene (fBm
terrain 829x1024 + 4,000 spheres + 4,000 boxes), FP16 LP buffer and FP16
display, FP32 shading and filter arithmetic.

A step is one binocular frame: the FP64 gaze set-up of both eyes, the LP
render of both eyes in one launch (one ray per LP texel: generation + BVH
traversal + shading) and the reconstruction of both full-resolution displays.
Inputs (scene, BVH, buffers) are resident in HBM before timing.  L2 is flushed
(256 MiB write) between steps, outside the per-step CUDA events.  The GPU's own
full-resolution ray cast (the paper's GT, one ray per display pixel) is timed
the same way for the speedup.  On one GPU the line also carries compact
results of the other configurations under extra keys: ``terrain4k`` (4K
monocular, FP32), ``sweep`` (1080p ... 16K binocular batched in one CUDA
graph, VaFR and GT per resolution) and ``serving`` (64 Poisson sessions,
frames/s and p50/p99 latency); ``--no-extra`` leaves them out.

``--impl reference`` times the FP64 CPU oracle (the reference arm here) on the
host cores over the same 240-frame trajectory: each step renders a bounded
random sample of one frame's LP texels and display pixels; ``ms_per_step`` is
the measured time of that sample and the whole-frame time extrapolated from it
is reported beside it.

Prints one JSON line (rank 0).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "display Mpix/s (VaFR frame: LP render + reconstruct)"
UNIT = "Mpix/s"
HERE_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FP32_LANES_PER_SM = 128
# FP32 operations per unit of traversal work, in two readings.
# Algorithmic counts (the traversal roofline's own units; `roofline.frac`):
# 12 per child-box test (a subtract and a multiply per slab plane), 30 per
# ray-triangle test, 20 per ray for generation and shading.
OPS_PER_BOX_ALG = 12
OPS_PER_TRI_ALG = 30
OPS_PER_RAY_ALG = 20
# Counted from the kernel source (`roofline.frac_source_count`): a child box
# test is 12 slab ops, 6 min/max (two three-input min/max and the clamps to 0
# and t_max), the far-bound scale, the compare and the select; a triangle test
# is 9 sub + 18 shear ops + 9 (U,V,W) + 2 (det) + 9 (z) + 3 (T) + 1 div + 7
# compares; ray set-up + generation + shading ~ 60.
OPS_PER_BOX = 21
OPS_PER_TRI = 58
OPS_PER_RAY = 60
PT_DIFFUSE = 3        # the paper's maximum diffuse bounces (Sec. 8.1)
# Deferred rasteriser, counted the same way from raster.cu: the screen-space
# pre-filter is 2 conversions + 2 adds + 6 FMAs + 3 compares; an exact test
# is the pixel ray (15), the shear set-up (3 abs, 5 compares/selects, 2 divides
# + 1 reciprocal, 9 selects = 20), the watertight test on eye-relative
# vertices (50) and the key (3).
LPT_VARIANTS = (6, 7)   # render variants in longest-first chunk order (k_render_lp_lpt)
OPS_PER_PREFILTER = 13
OPS_PER_PIXEL_TEST = 88


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(HERE_PEAKS) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic(kernel: str, srcs, workload: str):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel's sources changed since the counters were taken (the hash covers
    the concatenated source files) or no capture covers this workload."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        h = hashlib.sha256()
        for src in srcs:
            h.update(open(src, "rb").read())
        sha = h.hexdigest()[:16]
        for ln in open(path):
            f = ln.split()
            if len(f) >= 4 and f[0] == kernel and f[1] == sha and f[3] == workload:
                return float(f[2]), f[3]
    except OSError:
        pass
    return None, None


def _workload_desc(w):
    d = w.displays[0]
    return (f"{w.name}: {d.width}x{d.height} x {len(d.poses)} eye(s), {d.fov_v_deg:g} deg FOV, "
            f"{w.frames}-frame seeded gaze trajectory, {w.scene.n_tris:,} triangles "
            f"({w.scene.name}), LP {'FP16' if w.lp_fp16 else 'FP32'}, display "
            f"{'FP16' if w.display_fp16 else 'FP32'}")


L2_NOTE = "GPU arm: flushed between steps (256 MiB write outside the per-step events)"


def _config(w, args, ws):
    """The workload description, the same dict in both arms."""
    pt, rep, deferred = bool(args.pt), bool(args.rep), bool(args.deferred)
    return {"workload": _workload_desc(w), "l2": L2_NOTE, "acuity": args.acuity,
            "lp_fxaa": bool(args.fxaa),
            "shading": f"path traced, 1 path/texel, NEE, {PT_DIFFUSE} diffuse bounces" if pt
            else "ray cast, Lambert + ambient",
            "binocular_mode": "VaFR_Rep (right eye warped)" if rep else "VaFR_Dup",
            "pipeline": "deferred (visibility buffer + LP lighting)" if deferred else "ray casting",
            "point_lights": int(args.point_lights),
            "parallelism": f"replicas x{ws} (independent sessions, no collective)"}


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle on the host cores


def oracle_frame_sample(w, frame, n_tex, n_pix, bvh, lay, rng):
    """Seconds to render n_tex LP texels + reconstruct n_pix pixels of one frame
    (every eye), and the same scaled to a whole frame."""
    import oracle
    d = w.displays[0]
    eyes = len(d.poses)
    t_lp = t_rec = 0.0
    for e in range(eyes):
        gaze = d.gaze[frame % len(d.gaze), e]
        tex = np.sort(rng.choice(lay.total, n_tex, replace=False))
        t0 = time.perf_counter()
        rgba, ids, _, _, _ = oracle.render_lp(w.scene.tris, w.scene.albedo, w.scene.light_dir, lay,
                                              d.width, d.height, d.fov_v_deg, gaze, d.poses[e],
                                              texels=tex, bvh=bvh)
        t_lp += time.perf_counter() - t0
        lp = np.zeros((lay.total, 4))
        lp[tex] = rgba
        pix = rng.choice(d.width * d.height, n_pix, replace=False)
        t0 = time.perf_counter()
        oracle.reconstruct(lp, lay, d.width, d.height, d.fov_v_deg, gaze, pix)
        t_rec += time.perf_counter() - t0
    frame_s = t_lp * lay.total / n_tex + t_rec * d.width * d.height / n_pix
    return t_lp + t_rec, frame_s


def run_reference(args, w, ws):
    import oracle
    oracle.build()
    d = w.displays[0]
    eyes = len(d.poses)
    lay = oracle.lp_layout()
    t0 = time.perf_counter()
    bvh = oracle.CpuBVH(w.scene.tris)
    build_s = time.perf_counter() - t0
    rng = np.random.default_rng(123)
    n_tex, n_pix = args.ref_texels, args.ref_pixels
    for k in range(args.warmup):
        oracle_frame_sample(w, k, n_tex, n_pix, bvh, lay, rng)
    step_s, frame_s = [], []
    for k in range(args.steps):
        s_, f_ = oracle_frame_sample(w, args.warmup + k, n_tex, n_pix, bvh, lay, rng)
        step_s.append(s_)
        frame_s.append(f_)
    st, ft = np.array(step_s), np.array(frame_s)
    value = d.width * d.height * eyes / 1e6 / ft.mean()
    sample = (f"per step: {n_tex} random LP texels/eye (CPU BVH, FP64) + {n_pix} random display "
              f"pixels/eye reconstructed, of frame k of the {len(d.gaze)}-frame trajectory; Mpix/s "
              f"extrapolates the sample to the frame's {lay.total:,} texels and "
              f"{d.width * d.height:,} pixels per eye; BVH build {build_s:.1f} s excluded")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(st.mean() * 1e3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(w, args, ws),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "frame_ms_extrapolated": float(ft.mean() * 1e3),
        "p50_frame_ms_extrapolated": float(np.percentile(ft, 50) * 1e3),
        "p99_frame_ms_extrapolated": float(np.percentile(ft, 99) * 1e3),
        "cpu_seconds_measured": float(st.sum()),
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# the CUDA path


def run_gpu(args, w):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2503_23410_gb300 import build as B
    if rank == 0 or ws == 1:
        B.build()
    if dist:
        dist.barrier()
    from paper_2503_23410_gb300 import vafr as V
    V.load()
    peaks, peak_kind = _peaks()

    d = w.displays[0]
    eyes = len(d.poses)
    W_, H_ = d.width, d.height
    tris = torch.from_numpy(np.ascontiguousarray(w.scene.tris.reshape(-1, 9))).cuda()
    alb = torch.from_numpy(np.ascontiguousarray(w.scene.albedo)).cuda()
    scene = V.vafr_build_scene(tris, alb, w.scene.light_dir)
    lp_fmt = V.FMT_RGBA16F if w.lp_fp16 else V.FMT_RGBA32F
    dp_fmt = V.FMT_RGBA16F if w.display_fp16 else V.FMT_RGBA32F
    fxaa = bool(args.fxaa)
    pt = bool(args.pt)
    rep = bool(args.rep)
    deferred = bool(args.deferred)
    if rep and (pt or len(w.displays[0].poses) != 2):
        raise SystemExit("--rep needs a binocular workload and ray casting")
    if deferred and (pt or rep):
        raise SystemExit("--deferred excludes --pt and --rep")
    acuity = {"paper": None, "anisotropic": V.vafr_acuity_anisotropic,
              "display9": lambda: V.vafr_acuity_display_limited(9.0),
              "display18": lambda: V.vafr_acuity_display_limited(18.0)}[args.acuity]
    sess = V.vafr_session_create(V.make_session_desc(W_, H_, d.fov_v_deg, d.poses, lp_fmt, dp_fmt,
                                                     acuity() if acuity else None, lp_fxaa=fxaa))
    lp_b, dp_b = V.vafr_session_sizes(sess)
    lp = torch.empty(eyes * lp_b, dtype=torch.uint8, device="cuda")
    lp_aa = torch.empty(eyes * lp_b, dtype=torch.uint8, device="cuda") if fxaa else lp
    vbuf = torch.empty((H_, W_), dtype=torch.int64, device="cuda") if deferred else None
    if args.point_lights:
        rng_l = np.random.default_rng(1234)
        pts = w.scene.tris.reshape(-1, 3)
        lo, hi = pts.min(0), pts.max(0)
        lpos = rng_l.uniform(lo, hi, (args.point_lights, 3)).astype(np.float32)
        lpos[:, 1] = hi[1] + rng_l.uniform(1.0, 10.0, args.point_lights)
        lrgb = (rng_l.uniform(0.2, 1.0, (args.point_lights, 3)) * 400.0).astype(np.float32)
        V.vafr_scene_set_point_lights(scene, lpos, lrgb)
    disp = torch.empty(eyes * dp_b, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    nf = len(d.gaze)
    tuning = None
    if args.tuning:
        tuning = tuple(int(x) for x in args.tuning.split(","))
        V.vafr_session_tuning(sess, tuning)
    elif not (pt or rep or deferred or args.no_tune):
        # kernel variants picked on whole frames at the first gaze (untimed set-up)
        g0 = d.gaze[0]
        for e in range(eyes):
            V.vafr_set_gaze(sess, e, g0[e, 0], g0[e, 1])
        tuning = V.vafr_session_autotune(scene, sess, lp, disp, warm=3, iters=5)
    torch.cuda.synchronize()
    mask = (1 << eyes) - 1

    def frame(k, evs=None):
        g = d.gaze[k % nf]
        for e in range(eyes):
            V.vafr_set_gaze(sess, e, g[e, 0], g[e, 1])
        if evs:
            evs[0].record()
        if pt:                                     # path-traced LP buffer (Sec. 8)
            V.vafr_render_lp_pt(scene, sess, mask, lp, seed=k, max_diffuse=PT_DIFFUSE)
        elif rep:                                  # VaFR_Rep: left cast, right warped (Sec. 5.1)
            V.vafr_render_lp_rep(scene, sess, lp)
        elif deferred:                             # G-buffer at native resolution, LP lighting
            for e in range(eyes):
                V.vafr_render_vbuffer(scene, sess, e, vbuf)
                V.vafr_shade_lp_deferred(scene, sess, e, vbuf, lp[e * lp_b:])
        else:
            V.vafr_render_lp(scene, sess, mask, lp)
        if evs:
            evs[1].record()
        if fxaa:                                   # FXAA inside the LP buffer (Sec. 3.4)
            for e in range(eyes):
                V.vafr_fxaa_lp(sess, e, lp[e * lp_b:], lp_aa[e * lp_b:])
            if evs:
                evs[2].record()
        for e in range(eyes):
            V.vafr_reconstruct(sess, e, lp_aa[e * lp_b:], disp[e * dp_b:])
        if evs:
            evs[-1].record()

    # The GT cast is timed in its own fastest kernel, whichever variant the
    # VaFR frames use (the longest-first variants cast the GT with variant
    # 0's kernel, which is not the fastest GT cast on every scene).
    gt_variant = None

    def gt_frame(k, evs=None):
        vafr_cfg = None
        if gt_variant is not None:
            vafr_cfg = V.vafr_session_tuning(sess)
            V.vafr_session_tuning(sess, (gt_variant, vafr_cfg[1]))
        if evs:
            evs[0].record()
        for e in range(eyes):
            if pt:
                V.vafr_render_full_gt_pt(scene, sess, e, disp[e * dp_b:], seed=k, max_diffuse=PT_DIFFUSE)
            elif deferred:
                V.vafr_render_vbuffer(scene, sess, e, vbuf)
                V.vafr_shade_full_deferred(scene, sess, e, vbuf, disp[e * dp_b:])
            else:
                V.vafr_render_full_gt(scene, sess, e, disp[e * dp_b:])
        if evs:
            evs[1].record()
        if vafr_cfg is not None:
            V.vafr_session_tuning(sess, vafr_cfg)

    if not (pt or deferred):
        # pick it: every plain-order render variant casts one untimed and two
        # timed GT frames (CUDA events), the fastest is kept
        vafr_cfg = V.vafr_session_tuning(sess)
        best = None
        for v in range(V.vafr_tuning_space()[0]):
            if v in LPT_VARIANTS:
                continue
            V.vafr_session_tuning(sess, (v, vafr_cfg[1]))
            for e in range(eyes):
                V.vafr_render_full_gt(scene, sess, e, disp[e * dp_b:])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(2):
                for e in range(eyes):
                    V.vafr_render_full_gt(scene, sess, e, disp[e * dp_b:])
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                best = (ms, v)
        V.vafr_session_tuning(sess, vafr_cfg)
        gt_variant = best[1]

    def timed(fn, K, n_ev):
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(K)]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = V.vafr_kernel_launch_count()
        t0 = time.perf_counter()
        for k in range(K):
            flush.fill_(k & 0xff)
            fn(args.warmup + k, evs[k])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if dist:
            dist.barrier()
        launches = V.vafr_kernel_launch_count() - l0
        per = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(n_ev - 1)]
                        for k in range(K)])
        return per, wall, launches

    for k in range(args.warmup):
        frame(k)
        gt_frame(k)
    torch.cuda.synchronize()
    assert V.vafr_session_check(sess) == 0

    with ClockSampler(local) as clk:
        per, wall, launches = timed(frame, args.steps, 4 if fxaa else 3)
        gt_steps = max(3, min(args.steps, args.gt_steps))
        gper, gwall, _ = timed(gt_frame, gt_steps, 2)
        # end to end through the C ABI with HOST buffers, two ways:
        #  (a) vafr_render_frame into pinned host memory, one synchronous call
        #      per frame;
        #  (b) a 2-deep pipeline through the batch API: frame k renders on
        #      stream k % 2 into pinned host buffer k % 2 (the reconstruction
        #      writes the host memory directly), and a frame's buffer is
        #      reused only after its stream has finished, so frame k + 1
        #      computes while frame k crosses the CPU-GPU link.
        e2e_steps = max(3, min(args.steps, args.e2e_steps))
        host = [torch.empty(eyes * dp_b, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        if pt or rep or deferred:
            # (a) only: the frame as timed above, then one device-to-host copy
            def pt_e2e(k):
                g = d.gaze[k % nf]
                for e in range(eyes):
                    V.vafr_set_gaze(sess, e, g[e, 0], g[e, 1])
                frame(k)
                host[0].copy_(disp)
                torch.cuda.synchronize()
            for k in range(2):
                pt_e2e(k)
            te = time.perf_counter()
            for k in range(e2e_steps):
                pt_e2e(k)
            e2e_sync_s = e2e_s = time.perf_counter() - te
        else:
            for k in range(2):
                V.vafr_render_frame(scene, sess, host[0])
            torch.cuda.synchronize()
            te = time.perf_counter()
            for k in range(e2e_steps):
                g = d.gaze[k % nf]
                for e in range(eyes):
                    V.vafr_set_gaze(sess, e, g[e, 0], g[e, 1])
                V.vafr_render_frame(scene, sess, host[0])
            e2e_sync_s = time.perf_counter() - te
        if not (pt or rep or deferred):
            lps = [torch.empty(eyes * lp_b, dtype=torch.uint8, device="cuda") for _ in range(2)]
            aas = [torch.empty(eyes * lp_b, dtype=torch.uint8, device="cuda") for _ in range(2)] if fxaa else None
            streams = [torch.cuda.Stream() for _ in range(2)]
            batches = [V.vafr_batch_create(scene, 2 * eyes) for _ in range(2)]

            def frames_for(slot):
                if fxaa:
                    return [(sess, e, lps[slot][e * lp_b:], host[slot][e * dp_b:], aas[slot][e * lp_b:])
                            for e in range(eyes)]
                return [(sess, e, lps[slot][e * lp_b:], host[slot][e * dp_b:]) for e in range(eyes)]
            for k in range(4):
                V.vafr_batch_render(batches[k % 2], frames_for(k % 2), stream=streams[k % 2])
            torch.cuda.synchronize()
            te = time.perf_counter()
            for k in range(e2e_steps):
                slot = k % 2
                streams[slot].synchronize()          # frame k - 2 has landed in host[slot]
                g = d.gaze[k % nf]
                for e in range(eyes):
                    V.vafr_set_gaze(sess, e, g[e, 0], g[e, 1])
                V.vafr_batch_render(batches[slot], frames_for(slot), stream=streams[slot])
            for st_ in streams:
                st_.synchronize()
            e2e_s = time.perf_counter() - te
            for bt in batches:
                V.vafr_batch_destroy(bt)
    assert V.vafr_session_check(sess) == 0

    step_ms = per.sum(1)
    render_ms, recon_ms = per[:, 0], per[:, -1]
    gt_ms = gper[:, 0]
    total_s = step_ms.sum() / 1e3
    from paper_2503_23410_gb300.dist import max_over_ranks
    total_s, e2e_s, e2e_sync_s, gt_mean = max_over_ranks(
        [total_s, e2e_s, e2e_sync_s, float(gt_ms.mean())], "cuda")
    mpix_frame = W_ * H_ * eyes / 1e6
    value = mpix_frame * args.steps * ws / total_s
    e2e_value = mpix_frame * e2e_steps * ws / e2e_s
    e2e_sync_value = mpix_frame * e2e_steps * ws / e2e_sync_s

    # roofline of the dominant kernel
    stats = V.vafr_traversal_stats(scene, sess, 0)
    rays = stats["rays"] * eyes
    ops = (stats["box_tests"] * OPS_PER_BOX_ALG + stats["tri_tests"] * OPS_PER_TRI_ALG
           + stats["rays"] * OPS_PER_RAY_ALG) * eyes
    src_ratio = ((stats["box_tests"] * OPS_PER_BOX + stats["tri_tests"] * OPS_PER_TRI
                  + stats["rays"] * OPS_PER_RAY) /
                 max(stats["box_tests"] * OPS_PER_BOX_ALG + stats["tri_tests"] * OPS_PER_TRI_ALG
                     + stats["rays"] * OPS_PER_RAY_ALG, 1))
    pt_rays = None
    if pt:
        # rays per path from one signature run (segments traced + shadow rays
        # cast); the ops estimate scales the primary rays' per-ray cost
        sig = torch.empty((eyes * (lp_b // (8 if w.lp_fp16 else 16)), PT_DIFFUSE + 2), dtype=torch.int32,
                          device="cuda")
        sig.fill_(-2)
        V.vafr_render_lp_pt(scene, sess, mask, lp, seed=0, max_diffuse=PT_DIFFUSE, path_sig_out=sig)
        sg = sig.cpu().numpy()
        sg = sg[sg[:, 0] >= -1]                      # texel slots (guard slots stay -2)
        seg = int((sg[:, :PT_DIFFUSE + 1] >= -1).sum())
        shadow = int(np.unpackbits(((sg[:, -1] >> 16) & 0xff).astype(np.uint8)).sum())
        pt_rays = seg + shadow
        ops = ops / max(rays, 1) * pt_rays
        rays = pt_rays
    if rep:
        # the VaFR_Rep render stage casts the left eye's rays and the right
        # eye's holes (the last timed frame's count); the warp itself is
        # counted as no FP32 work, so the fraction is a lower bound
        rep_rays = stats["rays"] + V.vafr_rep_hole_count(sess)
        ops = ops / max(rays, 1) * rep_rays
        rays = rep_rays
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    derived_peak = n_sms * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12  # T FP32 ops/s
    ffma, ffma2 = V.vafr_measure_fp32_peak()                        # FMAs/s, measured here
    alu_peak = ffma / 1e12 if ffma > 0 else derived_peak
    render_s = float(render_ms.mean()) / 1e3
    recon_s = float(recon_ms.mean()) / 1e3
    lp_bytes = lp_b * eyes
    recon_bytes = dp_b * eyes + lp_bytes                            # display write + LP read once
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    csrc = os.path.join(ROOT, "paper_2503_23410_gb300", "csrc")
    # traffic lines were captured with the paper's acuity model; another model
    # changes the ray count and the LP buffer, so it needs captures of its own
    traffic_key = args.workload if args.acuity == "paper" else f"{args.workload}+{args.acuity}"
    lpt = bool(tuning) and tuning[0] in LPT_VARIANTS
    if pt:
        tr_render, _ = _traffic("path_lp", [os.path.join(csrc, f) for f in ("pathtrace.cu", "trace.cuh")],
                                traffic_key)
    elif rep:
        tr_render = None      # no capture covers the Rep stage's kernels together
    else:
        tr_render, _ = _traffic("render_lp_lpt" if lpt else "render_lp",
                                [os.path.join(csrc, f) for f in ("render.cu", "trace.cuh")], traffic_key)
    tr_recon, _ = _traffic("reconstruct", [os.path.join(csrc, f) for f in ("reconstruct.cu", "lp_map.cuh")],
                           traffic_key)
    render_kernel = ("k_path_lp" if pt else
                     "k_render_lp (left eye) + k_rep_* warp + k_render_list (holes)" if rep else
                     "k_render_lp_lpt" if lpt else "k_render_lp")
    roof_render = {"kernel": render_kernel, "bound": "alu",
                   "achieved": ops / render_s / 1e12,
                   "peak": alu_peak, "unit": "TFLOP/s", "frac": ops / render_s / 1e12 / alu_peak,
                   "ops_counted": (f"algorithmic: {OPS_PER_BOX_ALG} per child-box test, {OPS_PER_TRI_ALG} per "
                                   f"triangle test, {OPS_PER_RAY_ALG} per ray (generation + shading), with "
                                   "the box and triangle tests counted by an instrumented traversal"),
                   "frac_source_count": ops * src_ratio / render_s / 1e12 / alu_peak,
                   "ops_source_count": (f"{OPS_PER_BOX} per child-box test, {OPS_PER_TRI} per triangle test, "
                                        f"{OPS_PER_RAY} per ray, counted from the kernel source (robust slab "
                                        "form, watertight test with its division and compares)"),
                   "traffic": tr_render,
                   "peak_kind": (f"measured: scalar FFMA issue rate of this GPU (vafr_measure_fp32_peak; "
                                 f"paired FFMA2 {ffma2 / 1e12:.1f} T FMA/s; lane count x max clock "
                                 f"{derived_peak:.1f})") if ffma > 0 else
                                f"derived: {n_sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                f"{sm_mhz:g} MHz (1 op/lane/clk)",
                   "ops_per_launch": ops, "rays_per_launch": rays,
                   "nodes4_per_ray": stats["nodes"] / max(stats["rays"], 1),
                   "box_tests_per_ray": stats["box_tests"] / max(stats["rays"], 1),
                   "tri_tests_per_ray": stats["tri_tests"] / max(stats["rays"], 1),
                   "mrays_per_s": rays / render_s / 1e6, "avg_ms": render_s * 1e3}
    roof_recon = {"kernel": "k_reconstruct_runs", "bound": "hbm",
                  "achieved": recon_bytes / recon_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                  "frac": recon_bytes / recon_s / 1e9 / hbm_peak, "traffic": tr_recon,
                  "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured"
                  else "fallback 6.8 TB/s",
                  "bytes_per_launch": recon_bytes / eyes, "avg_ms": recon_s * 1e3 / eyes,
                  "launches_per_frame": eyes}
    if deferred:
        # the render stage is the V-buffer rasteriser (+ the LP lighting pass, a
        # few % of it): FP32 ops counted from the raster source per pre-filter
        # evaluation, per pixel past it (depth pre-test) and per exact
        # pixel-ray test, with the counts of an instrumented launch
        g = d.gaze[0]
        for q in range(eyes):
            V.vafr_set_gaze(sess, q, g[q, 0], g[q, 1])
        rs = {k: 0 for k in ("prefilter", "filtered", "tests", "atomics")}
        for q in range(eyes):
            for k, v in V.vafr_vbuffer_stats(scene, sess, q, vbuf).items():
                rs[k] += v
        r_ops = rs["prefilter"] * OPS_PER_PREFILTER + rs["filtered"] * 2 + rs["tests"] * OPS_PER_PIXEL_TEST
        roof_render = {"kernel": "k_vbuf_raster + k_vbuf_tiles (+ k_shade_lp_vbuf)", "bound": "alu",
                       "achieved": r_ops / render_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                       "frac": r_ops / render_s / 1e12 / alu_peak, "traffic": None,
                       "ops_counted": "counted from the rasteriser source per pre-filter evaluation, "
                                      "pixel past it and exact pixel-ray test",
                       "peak_kind": roof_render["peak_kind"], "ops_per_launch": r_ops,
                       "raster_counts_per_frame": rs, "avg_ms": render_s * 1e3}
    dominant = roof_render if render_s >= recon_s else roof_recon

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(step_ms.mean()), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(w, args, ws),
        "tuning": ({"render_variant": tuning[0], "reconstruct_variant": tuning[1],
                    "by": "--tuning" if args.tuning else
                    "vafr_session_autotune on whole frames at the first gaze, before warm-up"}
                   if tuning else "default variants (0, 0)"),
        "storage": {"lp": "f16" if w.lp_fp16 else "f32", "display": "f16" if w.display_fp16 else "f32",
                    "arithmetic": "f32 (shading, filter accumulation); f64 host gaze set-up"},
        "fps": 1e3 / float(step_ms.mean()),
        "p50_frame_ms": float(np.percentile(step_ms, 50)),
        "p99_frame_ms": float(np.percentile(step_ms, 99)),
        "gt": {"fps": 1e3 / gt_mean, "ms_per_frame": gt_mean,
               "mpix_per_s": mpix_frame * 1e3 / gt_mean, "rays_per_frame": W_ * H_ * eyes,
               "steps": gt_steps,
               "render_variant": (gt_variant if gt_variant is not None else
                                  V.vafr_session_tuning(sess)[0]),
               "variant_by": ("fastest plain-order variant on 2 GT frames, picked before warm-up"
                              if gt_variant is not None else "the VaFR frames' variant")},
        "speedup_vs_gt": gt_mean / float(step_ms.mean()),
        "stage_ms": dict({"render_lp": float(render_ms.mean()), "reconstruct": float(recon_ms.mean())},
                         **({"fxaa_lp": float(per[:, 1].mean())} if fxaa else {})),
        "roofline": dominant,
        "roofline_other": roof_recon if dominant is roof_render else roof_render,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 16 * eyes,
                "d2h_bytes_per_step": dp_b * eyes, "steps": e2e_steps,
                "path": ("the timed frame (path-traced, VaFR_Rep or deferred LP buffer, then "
                         "vafr_reconstruct), then one device-to-host copy into pinned memory, "
                         "synchronous per frame") if (pt or rep or deferred) else
                        ("vafr_batch_render into pinned host frames (reconstruction into the "
                         "batch's device staging buffers, copy-engine transfer to the host), 2 "
                         "frames in flight on 2 streams (C ABI); gaze passed by value each step"),
                "sync_per_frame_value": e2e_sync_value,
                "sync_per_frame_path": "vafr_render_frame into pinned host memory (the "
                                       "reconstruction writes it through its device alias), one "
                                       "synchronous call per frame"},
        "gpu_launches": int(launches),
        "wall_s_timed_loop": wall,
        "clocks": clk.summary(),
    }
    def gpu_eval(k, e):
        """One eye of frame k on the GPU (hit ids included), for the precision
        report: LP colours and ids in the oracle's texel order, display pixels."""
        g = d.gaze[k % nf]
        for q in range(eyes):
            V.vafr_set_gaze(sess, q, g[q, 0], g[q, 1])
        counts, offs, _, n_tex = V.vafr_lp_layout(sess)
        counts = counts.astype(np.int64)
        starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
        slot = np.repeat(offs - starts, counts) + np.arange(n_tex)
        tdt = torch.float16 if w.lp_fp16 else torch.float32
        lp1 = torch.empty(lp_b, dtype=torch.uint8, device="cuda")
        ids1 = torch.empty(lp_b // (8 if w.lp_fp16 else 16), dtype=torch.int32, device="cuda")
        disp1 = torch.empty(dp_b, dtype=torch.uint8, device="cuda")
        V.vafr_render_lp(scene, sess, 1 << e, lp1, ids1)
        V.vafr_reconstruct(sess, e, lp1, disp1)
        torch.cuda.synchronize()
        lp_h = lp1.view(tdt).view(-1, 4).float().cpu().numpy()[slot]
        dd = disp1.view(torch.float16 if w.display_fp16 else torch.float32).view(H_, W_, 4).float().cpu().numpy()
        return lp_h, ids1.cpu().numpy()[slot], dd

    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        plain = not (pt or rep or deferred or fxaa)
        line["cpu_baseline"], prec = cpu_baseline(args, w, gpu_eval if plain else None)
        if prec is not None:
            prec.update({"lp": "f16" if w.lp_fp16 else "f32", "display": "f16" if w.display_fp16 else "f32",
                         "accumulate": "f32", "frame": 0,
                         "note": "GPU frame against the FP64 oracle's frame at the same gaze; ids differ "
                                 "only at ray-edge ties, and display pixels whose filter footprint holds "
                                 "such a texel make the max"})
            line["precision"] = prec
    V.vafr_session_destroy(sess)
    V.vafr_scene_destroy(scene)
    if dist:
        dist.destroy_process_group()
    return line if rank == 0 else None


def _device_scene(V, torch, w):
    tris = torch.from_numpy(np.ascontiguousarray(w.scene.tris.reshape(-1, 9))).cuda()
    alb = torch.from_numpy(np.ascontiguousarray(w.scene.albedo)).cuda()
    return V.vafr_build_scene(tris, alb, w.scene.light_dir), (tris, alb)


def run_sweep(args):
    """Resolution sweep (binocular, 1080p ... 16K per eye, FP16 LP and display):
    all ten frame-eyes rendered by ONE batched render launch + ONE batched
    reconstruct launch per frame; GT timed per resolution."""
    import torch
    torch.cuda.set_device(0)
    from paper_2503_23410_gb300 import build as B
    B.build()
    from paper_2503_23410_gb300 import vafr as V
    from workloads import workload
    V.load()
    w = workload("sweep", frames=args.steps + args.warmup)
    scene, keep = _device_scene(V, torch, w)
    sess, bufs, frames = [], [], []
    for d in w.displays:
        s = V.vafr_session_create(V.make_session_desc(d.width, d.height, d.fov_v_deg, d.poses,
                                                      V.FMT_RGBA16F, V.FMT_RGBA16F))
        lpb, dpb = V.vafr_session_sizes(s)
        lp = torch.empty(2 * lpb, dtype=torch.uint8, device="cuda")
        dp = torch.empty(2 * dpb, dtype=torch.uint8, device="cuda")
        sess.append(s)
        bufs.append((lp, dp, lpb, dpb))
        for e in range(2):
            frames.append((s, e, lp[e * lpb:], dp[e * dpb:]))
    batch = V.vafr_batch_create(scene, V.MAX_BATCH)

    def set_gaze(k):
        for s, d in zip(sess, w.displays):
            for e in range(2):
                V.vafr_set_gaze(s, e, *d.gaze[k % len(d.gaze), e])
    set_gaze(0)
    V.vafr_batch_autotune(batch, frames, iters=3)
    V.vafr_batch_capture(batch, frames)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for k in range(args.warmup):
        set_gaze(k)
        V.vafr_batch_replay(batch)
    torch.cuda.synchronize()
    times = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        set_gaze(args.warmup + k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        V.vafr_batch_replay(batch)
        e1.record()
        times.append((e0, e1))
    torch.cuda.synchronize()
    batch_ms = np.array([a.elapsed_time(b) for a, b in times])
    per_res = []
    for (s, (lp, dp, lpb, dpb), d) in zip(sess, bufs, w.displays):
        gts = []
        for k in range(max(3, args.gt_steps // 4) + 2):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for e in range(2):
                V.vafr_render_full_gt(scene, s, e, dp[e * dpb:])
            e1.record()
            torch.cuda.synchronize()
            if k >= 2:
                gts.append(e0.elapsed_time(e1))
        vs = []
        for k in range(8):
            flush.fill_(2)
            for e in range(2):
                V.vafr_set_gaze(s, e, *d.gaze[k, e])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            V.vafr_render_lp(scene, s, 3, lp)
            for e in range(2):
                V.vafr_reconstruct(s, e, lp[e * lpb:], dp[e * dpb:])
            e1.record()
            torch.cuda.synchronize()
            if k >= 2:
                vs.append(e0.elapsed_time(e1))
        _, _, _, n_tex = V.vafr_lp_layout(s)
        per_res.append({"width": d.width, "height": d.height, "lp_rays": 2 * n_tex,
                        "gt_rays": 2 * d.width * d.height, "vafr_ms": float(np.median(vs)),
                        "gt_ms": float(np.median(gts)),
                        "speedup_vs_gt": float(np.median(gts) / np.median(vs))})
    mpix = sum(2 * d.width * d.height for d in w.displays) / 1e6
    line = {"metric": "display Mpix/s, resolution sweep batched in one launch", "unit": "Mpix/s",
            "value": mpix * 1e3 / float(batch_ms.mean()), "ms_per_step": float(batch_ms.mean()),
            "p50_frame_ms": float(np.percentile(batch_ms, 50)),
            "p99_frame_ms": float(np.percentile(batch_ms, 99)), "steps": args.steps,
            "warmup": args.warmup, "n_gpus": 1, "higher_is_better": True, "dtype": "f16 store, f32 math",
            "data": "synthetic", "config": {"workload": "sweep: terrain4k scene, binocular, per eye "
            "1920x1080, 2560x1440, 3840x2160, 7680x4320, 15360x8640; FP16 LP + display; one CUDA "
            "graph (render + reconstruct launch) per frame",
            "l2": "flushed between steps"},
            "tuning": V.vafr_batch_tuning(batch), "per_resolution": per_res}
    V.vafr_batch_destroy(batch)
    for s in sess:
        V.vafr_session_destroy(s)
    V.vafr_scene_destroy(scene)
    return line


def run_serving(args):
    """64 Poisson-arriving binocular sessions (1080p/1440p/4K/8K), admitted by
    an 8 GB HBM budget and continuously batched on two streams."""
    import torch
    torch.cuda.set_device(0)
    from paper_2503_23410_gb300 import build as B
    B.build()
    from paper_2503_23410_gb300 import vafr as V
    from paper_2503_23410_gb300.serve import Server, VafrBackend, poisson_requests
    from workloads import workload
    V.load()
    w = workload("serving", frames=args.serve_frames)
    scene, keep = _device_scene(V, torch, w)
    reqs = poisson_requests(w, seed=1)
    warm = poisson_requests(workload("serving", frames=3), seed=2, n_sessions=8)
    be = VafrBackend(scene, n_slots=2, autotune=True)
    Server(be, w.hbm_budget_bytes).run(warm)            # warm-up (tuning, allocator)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        st = Server(be, w.hbm_budget_bytes).run(reqs, time_limit_s=600)
    be.close_all()
    sm = st.summary()
    line = {"metric": "served frames/s and p50/p99 frame latency, 64 Poisson sessions",
            "unit": "frames/s", "value": sm["frames_per_s"], "higher_is_better": True,
            "n_gpus": 1, "data": "synthetic", "dtype": "f16 store, f32 math",
            "config": {"workload": f"serving: {len(reqs)} binocular sessions x {args.serve_frames} "
                       "frames, resolution uniform over 1080p/1440p/4K/8K, Poisson arrivals "
                       f"({w.poisson_rate_hz:.0f}/s), random-walk gaze, terrain4k scene, HBM "
                       f"budget {w.hbm_budget_bytes >> 30} GB, 2 in-flight batches"},
            "serving": sm, "clocks": clk.summary()}
    V.vafr_scene_destroy(scene)
    return line


def cpu_baseline(args, w, gpu_eval=None):
    """The FP64 oracle on the host cores: whole LP buffers (every texel through
    the CPU BVH) and the display reconstructed at up to --cpu-pixels pixels per
    eye (all of them at 4K), frame after frame along the gaze trajectory until
    --cpu-seconds of oracle work; Mpix/s extrapolates the pixel sample to whole
    frames.  With gpu_eval, the first frame is also compared with the GPU's
    (precision against the FP64 oracle)."""
    import oracle
    oracle.build()
    lay = oracle.lp_layout()
    d = w.displays[0]
    eyes = len(d.poses)
    npx = d.width * d.height
    bvh = oracle.CpuBVH(w.scene.tris)
    rng = np.random.default_rng(7)
    cpu_s, frame_s, k = 0.0, [], 0
    precision = None
    while k < 1 or (cpu_s < args.cpu_seconds and k < 240):
        t_lp = t_rec = 0.0
        n_pix = min(npx, args.cpu_pixels)
        for e in range(eyes):
            gaze = d.gaze[k % len(d.gaze), e]
            t0 = time.perf_counter()
            rgba, ids, _, _, _ = oracle.render_lp(w.scene.tris, w.scene.albedo, w.scene.light_dir, lay,
                                                  d.width, d.height, d.fov_v_deg, gaze, d.poses[e], bvh=bvh)
            t_lp += time.perf_counter() - t0
            pix = None if n_pix == npx else np.sort(rng.choice(npx, n_pix, replace=False))
            t0 = time.perf_counter()
            disp = oracle.reconstruct(rgba, lay, d.width, d.height, d.fov_v_deg, gaze, pix)
            t_rec += time.perf_counter() - t0
            if gpu_eval is not None and k == 0:
                precision = _precision(precision, gpu_eval(k, e), rgba, ids, disp, pix)
        cpu_s += t_lp + t_rec
        frame_s.append(t_lp + t_rec * npx / n_pix)
        k += 1
    ft = float(np.mean(frame_s))
    n_pix = min(npx, args.cpu_pixels)
    out = {"value": npx * eyes / 1e6 / ft, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{k} frames x (all {lay.total} LP texels via CPU BVH + "
                     f"{'all' if n_pix == npx else n_pix} of {npx} display pixels) per eye, FP64, "
                     f"ray-cast pipeline{'' if n_pix == npx else ', pixels extrapolated to whole frames'}; "
                     f"{cpu_s:.1f} s of oracle work"}
    return out, precision


def _precision(acc, gpu, rgba, ids, disp, pix):
    """Error of one GPU eye (LP slots in oracle texel order, hit ids, display
    pixels) against the FP64 oracle's frame: hit-id agreement, the LP colour
    error where the hits agree, and quantiles of the display error."""
    g_lp, g_ids, g_disp = gpu
    same = g_ids == ids
    lp_err = np.abs(g_lp[same] - rgba[same]).max() if same.any() else 0.0
    gd = g_disp.reshape(-1, 4)
    if pix is not None:
        gd = gd[pix]
    de = np.abs(gd - disp.reshape(-1, 4)).max(axis=1)
    cur = {"lp_hit_id_mismatch_frac": float(1.0 - same.mean()),
           "lp_max_abs_err_where_hits_agree": float(lp_err),
           "display_abs_err": {"p50": float(np.quantile(de, 0.5)), "p99": float(np.quantile(de, 0.99)),
                               "p99.9": float(np.quantile(de, 0.999)), "max": float(de.max())},
           "display_frac_err_above_1e-3": float((de > 1e-3).mean())}
    if acc is None:
        return cur
    # worst over eyes
    acc["lp_hit_id_mismatch_frac"] = max(acc["lp_hit_id_mismatch_frac"], cur["lp_hit_id_mismatch_frac"])
    acc["lp_max_abs_err_where_hits_agree"] = max(acc["lp_max_abs_err_where_hits_agree"],
                                                 cur["lp_max_abs_err_where_hits_agree"])
    for q in acc["display_abs_err"]:
        acc["display_abs_err"][q] = max(acc["display_abs_err"][q], cur["display_abs_err"][q])
    acc["display_frac_err_above_1e-3"] = max(acc["display_frac_err_above_1e-3"],
                                             cur["display_frac_err_above_1e-3"])
    return acc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=240)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="vafr", choices=["vafr", "reference"])
    ap.add_argument("--workload", default="objects8k",
                    choices=["random1k", "terrain4k", "objects8k", "sweep", "serving"])
    ap.add_argument("--serve-frames", type=int, default=60)
    ap.add_argument("--gt-steps", type=int, default=60)
    ap.add_argument("--e2e-steps", type=int, default=60)
    ap.add_argument("--ref-texels", type=int, default=65536)
    ap.add_argument("--ref-pixels", type=int, default=524288)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-pixels", type=int, default=1 << 23,
                    help="display pixels per eye the oracle reconstructs in each baseline frame")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--acuity", default="paper", choices=["paper", "anisotropic", "display9", "display18"],
                    help="acuity model: the paper's pivots, the Sec. 9 anisotropy, or the Sec. 3.3 "
                         "display-limited curves at 9 / 18 cpd")
    ap.add_argument("--pt", action="store_true",
                    help="path-trace the LP buffer (Sec. 8: 1 path per texel, NEE, 3 diffuse bounces) "
                         "and compare with the path-traced full-resolution GT")
    ap.add_argument("--deferred", action="store_true",
                    help="deferred pipeline (Sec. 3.4 / 5): visibility buffer rasterised at display "
                         "resolution, lighting in the LP buffer; GT lights every pixel")
    ap.add_argument("--point-lights", type=int, default=0,
                    help="seeded unshadowed point lights added to the scene (the deferred scenes "
                         "carry many lights; the Sun Temple has 31)")
    ap.add_argument("--rep", action="store_true",
                    help="VaFR_Rep (Sec. 5.1): the right eye's LP buffer warped from the left eye's, "
                         "holes ray cast (binocular workloads)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default kernel variants instead of vafr_session_autotune's choice")
    ap.add_argument("--tuning", default=None,
                    help="render,reconstruct variants to use instead of autotuning (e.g. 6,2; for "
                         "profiling runs, where the tuner's timings are distorted)")
    ap.add_argument("--fxaa", action="store_true",
                    help="run the LP-space FXAA pass (Sec. 3.4) inside each timed frame")
    ap.add_argument("--no-extra", action="store_true",
                    help="leave out the terrain4k, sweep and serving summaries of the default line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    from workloads import workload
    ws, rank, _ = _dist()
    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, workload(args.workload), ws)
        return
    if args.workload == "sweep":
        print(json.dumps(run_sweep(args)))
        return
    if args.workload == "serving":
        print(json.dumps(run_serving(args)))
        return
    line = run_gpu(args, workload(args.workload))
    if line is None:
        return
    plain = not (args.pt or args.rep or args.deferred or args.fxaa or args.tuning or args.acuity != "paper")
    if ws == 1 and args.workload == "objects8k" and plain and not args.no_extra:
        line["extra_configs"] = ("terrain4k, sweep and serving: the other single-GPU configurations, "
                                 "measured in the same process after the headline, L2 flushed between steps")
        sub = argparse.Namespace(**vars(args))
        sub.cpu_seconds = 0.0           # one oracle frame: the precision report, no baseline loop
        line["terrain4k"] = _compact(run_gpu(sub, workload("terrain4k")))
        line["sweep"] = {k: v for k, v in run_sweep(args).items()
                         if k not in ("metric", "n_gpus", "higher_is_better", "data", "steps", "warmup")}
        line["serving"] = {k: v for k, v in run_serving(args).items()
                           if k not in ("metric", "n_gpus", "higher_is_better", "data")}
    print(json.dumps(line))


def _compact(line):
    """The figures of a secondary configuration's line worth keeping."""
    keep = ("value", "unit", "ms_per_step", "fps", "p50_frame_ms", "p99_frame_ms", "speedup_vs_gt",
            "stage_ms", "tuning", "precision", "storage")
    out = {k: line[k] for k in keep if k in line}
    out["workload"] = line["config"]["workload"]
    out["gt_ms_per_frame"] = line["gt"]["ms_per_frame"]
    out["e2e_value"] = line["e2e"]["value"]
    for key in ("roofline", "roofline_other"):
        r = line[key]
        out[key] = {k: r[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac",
                                      "frac_source_count", "traffic", "avg_ms") if k in r}
    if "cpu_baseline" in line:
        out["cpu_oracle_one_frame"] = line["cpu_baseline"]
    return out


if __name__ == "__main__":
    main()
