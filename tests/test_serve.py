"""Continuous-batching scheduler on the CPU with a simulated device: admission by
HBM budget, overlap of in-flight batches, latency accounting, and host-side
fault handling (oversized / malformed requests, cancellation, a device fault
reported by the backend).  No GPU is touched."""

import numpy as np
import pytest

from paper_2503_23410_gb300.serve import Server, SessionRequest


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """A batch takes 1 ms + 0.1 ms per session; idle() advances the clock."""

    def __init__(self, clock, fault_on_batch=None):
        self.clock = clock
        self.open_handles = set()
        self.launches = []
        self.fault_on_batch = fault_on_batch

    def bytes_needed(self, r):
        return r.width * r.height * r.eyes

    def open(self, r):
        if r.width <= 0:
            raise ValueError("width must be positive")
        h = object()
        self.open_handles.add(h)
        return h

    def close(self, h):
        self.open_handles.remove(h)
        return None

    def launch(self, slot, items):
        done = self.clock.t + 1e-3 + 1e-4 * len(items)
        self.launches.append((self.clock.t, slot, len(items)))
        return (done, len(self.launches) - 1)

    def done(self, token):
        return self.clock.t >= token[0]

    def check(self, token):
        return "injected fault" if token[1] == self.fault_on_batch else None

    def idle(self):
        self.clock.t += 5e-5


def _reqs(n, frames=5, rate=2000.0, seed=0, w=100, h=100):
    rng = np.random.default_rng(seed)
    t = np.concatenate([[0.0], np.cumsum(rng.exponential(1 / rate, n - 1))])
    poses = [np.eye(3, 4), np.eye(3, 4)]
    return [SessionRequest(i, float(t[i]), w, h, 90.0, poses, np.zeros((frames, 2, 2)))
            for i in range(n)]


def test_all_frames_served_and_memory_released():
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _reqs(40)
    st = Server(be, hbm_budget_bytes=10 * 100 * 100 * 2, clock=clk).run(reqs)
    assert st.frames_done == 40 * 5
    assert len(st.latencies_ms) == 200
    assert not be.open_handles
    assert st.peak_bytes <= 10 * 100 * 100 * 2
    assert st.max_concurrent == 10           # the budget, not the arrivals, limits the mix
    assert st.overlapped_launches > 0        # a batch was launched while another ran
    assert max(n for _, _, n in be.launches) > 1
    s = st.summary()
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_continuous_batching_admits_mid_flight():
    # sessions arriving while a batch is in flight join the next batch
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _reqs(6, frames=50, rate=5000.0)
    st = Server(be, hbm_budget_bytes=10 ** 9, clock=clk).run(reqs)
    sizes = [n for _, _, n in be.launches]
    assert sizes[0] < 6 and max(sizes) == 6
    assert st.frames_done == 300


def test_oversized_and_malformed_requests_rejected():
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _reqs(5)
    reqs[1].width = 10_000                   # can never fit the budget
    reqs[3].width = 0                        # the backend refuses it
    st = Server(be, hbm_budget_bytes=100 * 100 * 2 * 2, clock=clk).run(reqs)
    assert set(st.rejected) == {1, 3}
    assert st.frames_done == 3 * 5
    assert not be.open_handles


def test_cancellation():
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _reqs(4, frames=1000)
    srv = Server(be, hbm_budget_bytes=10 ** 9, clock=clk)
    srv.cancel(2)
    orig_idle = be.idle

    def idle():
        orig_idle()
        if clk.t > 0.05:
            srv.cancel(0)
    be.idle = idle
    st = srv.run(reqs)
    assert 2 in st.cancelled and 0 in st.cancelled
    assert not be.open_handles
    assert st.frames_done < 4 * 1000


def test_device_fault_marks_sessions_failed():
    clk = FakeClock()
    be = FakeBackend(clk, fault_on_batch=3)
    st = Server(be, hbm_budget_bytes=10 ** 9, clock=clk).run(_reqs(8, frames=10))
    assert st.failed, "the injected fault must be reported"
    assert all(v == "injected fault" for v in st.failed.values())
    assert not be.open_handles
    assert st.frames_done + len(st.failed) <= 80


def test_time_limit():
    clk = FakeClock()
    be = FakeBackend(clk)
    be.done = lambda token: False           # a device that never completes
    with pytest.raises(TimeoutError):
        Server(be, hbm_budget_bytes=10 ** 9, clock=clk).run(_reqs(2), time_limit_s=0.01)
