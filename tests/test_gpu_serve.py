"""Serving on the GPU: Poisson sessions of mixed resolutions (1080p to 8K,
binocular), admitted by HBM budget, continuously batched; each frame rendered
in the mix, 8K binocular sessions included, is bitwise the same as that frame
rendered alone."""

import numpy as np
import pytest

from parity import device_scene
from paper_2503_23410_gb300.serve import Server, VafrBackend, poisson_requests
from workloads import workload

pytestmark = pytest.mark.gpu


def test_served_mix_equals_alone(V, torch_mod):
    torch = torch_mod
    w = workload("serving", frames=6)     # the serving configuration's scene (1.07 M triangles)
    h, keep = device_scene(V, w.scene, torch)
    reqs = poisson_requests(w, seed=1, n_sessions=24, rate_hz=2000.0)
    big = [i for i, r in enumerate(reqs) if r.width >= 7680 and r.eyes == 2]
    small = [i for i, r in enumerate(reqs) if r.width < 7680]
    assert big and len(small) >= 2, "the seeded mix holds 8K binocular and smaller sessions"
    # session -> frame to snapshot: an 8K binocular session among them
    watch = {big[0]: 2, small[0]: 0, small[-1]: 5}
    if len(big) > 1:
        watch[big[-1]] = 4
    snaps = {}

    def on_done(sid, frame, handle):
        if watch.get(sid) == frame:
            snaps[sid] = handle["disp"].cpu().numpy().copy()

    be = VafrBackend(h, n_slots=2)
    budget = 3 << 30                      # room for about five 8K binocular sessions at once
    st = Server(be, hbm_budget_bytes=budget, on_frame_done=on_done).run(reqs, time_limit_s=300)
    be.close_all()
    s = st.summary()
    print("serving", s)
    assert st.frames_done == sum(r.frames for r in reqs)
    assert not st.failed and not st.rejected
    assert st.peak_bytes <= budget
    assert max(st.batch_sizes) > 1
    assert set(snaps) == set(watch)
    # the same frames rendered alone
    for sid, frame in watch.items():
        r = reqs[sid]
        sess = V.vafr_session_create(V.make_session_desc(
            r.width, r.height, r.fov_v_deg, r.poses, V.FMT_RGBA16F, V.FMT_RGBA16F))
        for e in range(r.eyes):
            V.vafr_set_gaze(sess, e, *r.gaze[frame, e])
        lpb, dpb = V.vafr_session_sizes(sess)
        lp = torch.empty(r.eyes * lpb, dtype=torch.uint8, device="cuda")
        disp = torch.empty(r.eyes * dpb, dtype=torch.uint8, device="cuda")
        V.vafr_render_lp(h, sess, (1 << r.eyes) - 1, lp)
        for e in range(r.eyes):
            V.vafr_reconstruct(sess, e, lp[e * lpb:], disp[e * dpb:])
        torch.cuda.synchronize()
        assert np.array_equal(disp.cpu().numpy(), snaps[sid]), f"session {sid} frame {frame}"
        V.vafr_session_destroy(sess)
    V.vafr_scene_destroy(h)
