"""Host-side logic of bench.py (no GPU): the precision summary against the
oracle and the whole-frame oracle baseline on a small workload."""

import types

import numpy as np

import bench
import oracle
from workloads import workload


def test_precision_summary():
    rng = np.random.default_rng(3)
    n, W, H = 1000, 8, 4
    ref = rng.uniform(0, 1, (n, 4))
    ids = np.arange(n)
    gpu_lp = ref + 1e-6
    gids = ids.copy()
    gids[7] = -1                                  # one disagreeing hit
    gpu_lp[7] = 0.0                               # ... whose colour is not counted
    disp = rng.uniform(0, 1, (H * W, 4))
    gdisp = disp.copy()
    gdisp[5, 2] += 0.5                            # one bad pixel
    p = bench._precision(None, (gpu_lp, gids, gdisp.reshape(H, W, 4)), ref, ids, disp, None)
    assert abs(p["lp_hit_id_mismatch_frac"] - 1.0 / n) < 1e-12
    assert abs(p["lp_max_abs_err_where_hits_agree"] - 1e-6) < 1e-9
    assert abs(p["display_abs_err"]["max"] - 0.5) < 1e-12
    assert abs(p["display_frac_err_above_1e-3"] - 1.0 / (H * W)) < 1e-12
    # a second eye keeps the worst of both
    q = bench._precision(dict(p, display_abs_err=dict(p["display_abs_err"])),
                         (ref, ids, disp.reshape(H, W, 4)), ref, ids, disp, None)
    assert q["display_abs_err"]["max"] == p["display_abs_err"]["max"]
    # a pixel sample selects the same pixels on both sides
    pix = np.array([1, 5, 9])
    r = bench._precision(None, (gpu_lp, gids, gdisp.reshape(H, W, 4)), ref, ids, disp[pix], pix)
    assert abs(r["display_abs_err"]["max"] - 0.5) < 1e-12


def test_cpu_baseline_small_workload():
    w = workload("random1k", frames=4)
    args = types.SimpleNamespace(cpu_seconds=0.0, cpu_pixels=1 << 23)
    lay = oracle.lp_layout()
    d = w.displays[0]

    def gpu_eval(k, e):     # the oracle standing in for the GPU: zero error
        rgba, ids, _, _, _ = oracle.render_lp(w.scene.tris, w.scene.albedo, w.scene.light_dir, lay,
                                              d.width, d.height, d.fov_v_deg, d.gaze[k, e], d.poses[e])
        out = oracle.reconstruct(rgba, lay, d.width, d.height, d.fov_v_deg, d.gaze[k, e])
        return rgba, ids, out.reshape(d.height, d.width, 4)

    line, prec = bench.cpu_baseline(args, w, gpu_eval)
    assert line["kind"] == "oracle" and line["value"] > 0 and line["cores"] >= 1
    assert "all 1061630 LP texels" in line["sample"]
    assert prec["lp_hit_id_mismatch_frac"] == 0.0
    assert prec["display_abs_err"]["max"] == 0.0


def test_traffic_lines_match_sources_and_workload(tmp_path):
    """A committed DRAM-traffic line is used only for the kernel, source hash and
    workload it was captured on."""
    import hashlib
    import os
    csrc = os.path.join(bench.ROOT, "paper_2503_23410_gb300", "csrc")
    srcs = [os.path.join(csrc, f) for f in ("render.cu", "trace.cuh")]
    h = hashlib.sha256()
    for s in srcs:
        h.update(open(s, "rb").read())
    sha = h.hexdigest()[:16]
    lines = [ln.split() for ln in open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.txt"))
             if ln.strip() and not ln.startswith("#")]
    want = {(f[0], f[3]): float(f[2]) for f in lines if f[1] == sha}
    for (kernel, wl), b in want.items():
        assert bench._traffic(kernel, srcs, wl) == (b, wl)
    assert bench._traffic("render_lp", srcs, "no-such-workload") == (None, None)
    other = tmp_path / "edited.cu"
    other.write_bytes(open(srcs[0], "rb").read() + b"\n")
    assert bench._traffic("render_lp", [str(other), srcs[1]], "terrain4k") == (None, None)


def test_reference_arm_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints one
    JSON line with the benchmark contract's keys."""
    import json
    import os
    import subprocess
    import sys
    import time
    t0 = time.perf_counter()
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "random1k", "--steps", "2", "--warmup", "0",
                          "--ref-texels", "512", "--ref-pixels", "4096"],
                         capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    wall = time.perf_counter() - t0
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # the measured per-step time fits inside the process's own run time
    assert d["ms_per_step"] * d["steps"] / 1e3 < wall
    assert d["frame_ms_extrapolated"] > 0
    # the same workload description as the GPU arm, trajectory included
    args = bench.argparse.Namespace(pt=False, rep=False, deferred=False, fxaa=False, acuity="paper",
                                    point_lights=0)
    assert d["config"] == bench._config(workload("random1k"), args, 1)
