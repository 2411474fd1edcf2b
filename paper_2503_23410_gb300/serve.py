"""Continuous-batching request loop for foveated rendering sessions.

Sessions (a display size, FOV, eye poses and a gaze trajectory of N frames)
arrive over time.  The server

* admits waiting sessions in arrival order while their LP + display buffers
  fit the HBM budget (a session that could never fit is rejected);
* keeps every admitted session's buffers, and the one scene, resident;
* at every scheduling step gathers the next frame of every admitted session
  that has no frame in flight and launches them together -- both eyes of all
  of them -- as ONE batched render launch + ONE batched reconstruct launch;
* keeps up to ``max_inflight`` batches on the GPU at once (one stream each),
  so requests that arrive while a batch runs are admitted and launched
  without waiting for it;
* frees a session's memory when its last frame completes, letting waiting
  sessions in.

A frame's latency runs from the moment it was requestable (the session's
arrival for its first frame, the completion of the previous frame after that)
to the completion of the batch that rendered it.

The scheduler is independent of the device: ``VafrBackend`` drives libvafr
through its C ABI with PyTorch streams and memory; tests drive the same
scheduler with a simulated backend on the CPU.
"""

from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class SessionRequest:
    sid: int
    arrival_s: float
    width: int
    height: int
    fov_v_deg: float
    poses: Sequence[np.ndarray]     # one (3, 4) pose per eye
    gaze: np.ndarray                # (frames, eyes, 2) pixel positions
    lp_fp16: bool = True
    display_fp16: bool = True

    @property
    def frames(self) -> int:
        return int(self.gaze.shape[0])

    @property
    def eyes(self) -> int:
        return len(self.poses)


@dataclasses.dataclass
class _Active:
    req: SessionRequest
    handle: object
    nbytes: int
    next_frame: int = 0
    in_flight: bool = False
    ready_t: float = 0.0


@dataclasses.dataclass
class ServeStats:
    frames_done: int = 0            # session-frames (all eyes of a session)
    eye_frames_done: int = 0
    mpix_done: float = 0.0
    wall_s: float = 0.0
    latencies_ms: List[float] = dataclasses.field(default_factory=list)
    batches: int = 0
    batch_sizes: List[int] = dataclasses.field(default_factory=list)
    admitted: int = 0
    rejected: Dict[int, str] = dataclasses.field(default_factory=dict)
    cancelled: List[int] = dataclasses.field(default_factory=list)
    failed: Dict[int, str] = dataclasses.field(default_factory=dict)
    peak_bytes: int = 0
    max_concurrent: int = 0
    overlapped_launches: int = 0    # launches issued while another batch was in flight

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {
            "frames_per_s": self.frames_done / max(self.wall_s, 1e-9),
            "eye_frames_per_s": self.eye_frames_done / max(self.wall_s, 1e-9),
            "mpix_per_s": self.mpix_done / max(self.wall_s, 1e-9),
            "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)),
            "frames": self.frames_done,
            "batches": self.batches,
            "mean_batch_sessions": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
            "admitted": self.admitted,
            "rejected": len(self.rejected),
            "cancelled": len(self.cancelled),
            "failed": len(self.failed),
            "peak_bytes": self.peak_bytes,
            "max_concurrent_sessions": self.max_concurrent,
            "overlapped_launches": self.overlapped_launches,
            "wall_s": self.wall_s,
        }


class Server:
    """Backend-agnostic continuous-batching scheduler (see module docstring)."""

    def __init__(self, backend, hbm_budget_bytes: int, max_batch_sessions: int = 64,
                 max_inflight: int = 2, clock: Callable[[], float] = time.perf_counter,
                 on_frame_done: Optional[Callable[[int, int, object], None]] = None):
        self.backend = backend
        self.budget = int(hbm_budget_bytes)
        self.max_batch = int(max_batch_sessions)
        self.max_inflight = int(max_inflight)
        self.clock = clock
        self.on_frame_done = on_frame_done
        self._cancel = set()

    def cancel(self, sid: int) -> None:
        """Stop a session: it is dropped when waiting, or after its in-flight frame."""
        self._cancel.add(sid)

    def run(self, requests: Sequence[SessionRequest], time_limit_s: float = 600.0) -> ServeStats:
        st = ServeStats()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting: collections.deque = collections.deque()
        active: Dict[int, _Active] = {}
        inflight: collections.deque = collections.deque()   # (token, slot, [(sid, frame)])
        free_slots = list(range(self.max_inflight))
        used = 0
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            if now > time_limit_s:
                raise TimeoutError(f"serving did not finish within {time_limit_s} s")
            while pending and pending[0].arrival_s <= now:
                waiting.append(pending.popleft())
            # completions, in launch order
            while inflight and self.backend.done(inflight[0][0]):
                token, slot, items = inflight.popleft()
                free_slots.append(slot)
                t_done = self.clock() - t0
                fault = self.backend.check(token)
                for sid, frame in items:
                    a = active[sid]
                    a.in_flight = False
                    if fault:
                        st.failed[sid] = fault
                        a.next_frame = a.req.frames
                    else:
                        st.latencies_ms.append((t_done - a.ready_t) * 1e3)
                        st.frames_done += 1
                        st.eye_frames_done += a.req.eyes
                        st.mpix_done += a.req.width * a.req.height * a.req.eyes / 1e6
                        if self.on_frame_done:
                            self.on_frame_done(sid, frame, a.handle)
                        a.next_frame = frame + 1
                    a.ready_t = t_done
                    if a.next_frame >= a.req.frames or sid in self._cancel:
                        if sid in self._cancel and a.next_frame < a.req.frames:
                            st.cancelled.append(sid)
                        bad = self.backend.close(a.handle)
                        if bad:
                            st.failed[sid] = bad
                        used -= a.nbytes
                        del active[sid]
            # cancellations of sessions that are waiting or idle
            for sid in list(self._cancel):
                for r in list(waiting):
                    if r.sid == sid:
                        waiting.remove(r)
                        st.cancelled.append(sid)
                a = active.get(sid)
                if a is not None and not a.in_flight:
                    st.cancelled.append(sid)
                    bad = self.backend.close(a.handle)
                    if bad:
                        st.failed[sid] = bad
                    used -= a.nbytes
                    del active[sid]
            # admission: arrival order, by HBM budget
            while waiting:
                r = waiting[0]
                need = self.backend.bytes_needed(r)
                if need > self.budget:
                    waiting.popleft()
                    st.rejected[r.sid] = f"needs {need} B > budget {self.budget} B"
                    continue
                if used + need > self.budget:
                    break
                waiting.popleft()
                try:
                    h = self.backend.open(r)
                except Exception as exc:   # malformed request: reject it, keep serving
                    st.rejected[r.sid] = f"{type(exc).__name__}: {exc}"
                    continue
                used += need
                st.admitted += 1
                active[r.sid] = _Active(r, h, need, ready_t=self.clock() - t0)
                st.peak_bytes = max(st.peak_bytes, used)
            st.max_concurrent = max(st.max_concurrent, len(active))
            # launch every ready session's next frame as one batch
            ready = [a for a in active.values() if not a.in_flight]
            if ready and free_slots:
                ready = ready[:self.max_batch]
                slot = free_slots.pop(0)
                items = [(a.req.sid, a.next_frame) for a in ready]
                if inflight:
                    st.overlapped_launches += 1
                token = self.backend.launch(slot, [(a.handle, a.req, a.next_frame) for a in ready])
                for a in ready:
                    a.in_flight = True
                inflight.append((token, slot, items))
                st.batches += 1
                st.batch_sizes.append(len(ready))
            elif not inflight and not active and waiting and pending:
                time.sleep(0)
            else:
                self.backend.idle()
        st.wall_s = self.clock() - t0
        return st


class VafrBackend:
    """libvafr through its C ABI: one vafr batch object + one CUDA stream per slot."""

    def __init__(self, scene_handle: int, n_slots: int = 2, autotune: bool = False):
        import torch

        from . import vafr as V
        self.V = V
        self.torch = torch
        self.scene = scene_handle
        self.streams = [torch.cuda.Stream() for _ in range(n_slots)]
        self.batches = [V.vafr_batch_create(scene_handle, V.MAX_BATCH) for _ in range(n_slots)]
        self.autotune = autotune
        self._tuned = False

    def bytes_needed(self, r: SessionRequest) -> int:
        lp = 1061630 * (8 if r.lp_fp16 else 16)      # refined once the session exists
        disp = r.width * r.height * (8 if r.display_fp16 else 16)
        return (lp + disp) * r.eyes

    def open(self, r: SessionRequest):
        V, torch = self.V, self.torch
        desc = V.make_session_desc(r.width, r.height, r.fov_v_deg, r.poses,
                                   V.FMT_RGBA16F if r.lp_fp16 else V.FMT_RGBA32F,
                                   V.FMT_RGBA16F if r.display_fp16 else V.FMT_RGBA32F)
        s = V.vafr_session_create(desc)
        lpb, dpb = V.vafr_session_sizes(s)
        lp = torch.empty(r.eyes * lpb, dtype=torch.uint8, device="cuda")
        disp = torch.empty(r.eyes * dpb, dtype=torch.uint8, device="cuda")
        return {"s": s, "lp": lp, "disp": disp, "lpb": lpb, "dpb": dpb, "eyes": r.eyes}

    def close(self, h) -> Optional[str]:
        """Frees the session; returns a fault description if its device status
        word recorded one (read once per session, at close)."""
        rc = self.V.load().vafr_session_check(h["s"], None)
        self.V.vafr_session_destroy(h["s"])
        h["lp"] = h["disp"] = None
        return None if rc == 0 else "device status %d" % rc

    def launch(self, slot: int, items):
        V, torch = self.V, self.torch
        frames = []
        for h, r, f in items:
            g = r.gaze[min(f, r.frames - 1)]
            for e in range(r.eyes):
                V.vafr_set_gaze(h["s"], e, float(g[e, 0]), float(g[e, 1]))
                frames.append((h["s"], e, h["lp"][e * h["lpb"]:], h["disp"][e * h["dpb"]:]))
        stream = self.streams[slot]
        stream.wait_stream(torch.cuda.current_stream())
        if self.autotune and not self._tuned:
            with torch.cuda.stream(stream):
                V.vafr_batch_autotune(self.batches[slot], frames, stream=stream, iters=2)
                cfg = V.vafr_batch_tuning(self.batches[slot])
                for b in self.batches:
                    V.vafr_batch_tuning(b, cfg)
            self._tuned = True
        V.vafr_batch_render(self.batches[slot], frames, stream=stream)
        ev = torch.cuda.Event()
        ev.record(stream)
        return (ev, [h for h, _, _ in items])

    def done(self, token) -> bool:
        return token[0].query()

    def check(self, token) -> Optional[str]:
        return None    # device status words are read once per session, at close

    def idle(self) -> None:
        pass

    def close_all(self) -> None:
        for b in self.batches:
            self.V.vafr_batch_destroy(b)
        self.batches = []


def poisson_requests(workload, seed: int = 0, n_sessions: Optional[int] = None,
                     rate_hz: Optional[float] = None) -> List[SessionRequest]:
    """Requests of a serving workload: Poisson arrivals at ``rate_hz``."""
    rng = np.random.default_rng(seed)
    disps = workload.displays[:n_sessions] if n_sessions else workload.displays
    rate = rate_hz or workload.poisson_rate_hz or 100.0
    t = np.cumsum(rng.exponential(1.0 / rate, size=len(disps)))
    t -= t[0]
    return [SessionRequest(i, float(t[i]), d.width, d.height, d.fov_v_deg, d.poses, d.gaze,
                           workload.lp_fp16, workload.display_fp16)
            for i, d in enumerate(disps)]
