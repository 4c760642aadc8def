"""Host logic of the serving loop, against a simulated device (CPU only).

The fake models only scheduling: admission limits (E_AGAIN), launch slots,
continuous batching of frames queued while every slot is busy, and a
service time per batch. It computes nothing; the real path runs in the
library's kernels (tests/test_gpu_serving.py).
"""
import pytest

from paper_2601_01210_gb300.densify import DENSIFY_E_AGAIN, DENSIFY_OK, DENSIFY_PENDING
from paper_2601_01210_gb300.serve import ServeLoop, poisson_arrivals


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-5          # every call advances simulated time by 10 us
        return self.t


class FakeDevice:
    def __init__(self, clock, max_inflight=4, slots=1, per_batch_s=2e-3, per_frame_s=2e-4, max_batch=16):
        self.clock, self.max_inflight, self.slots = clock, max_inflight, slots
        self.per_batch_s, self.per_frame_s, self.max_batch = per_batch_s, per_frame_s, max_batch
        self.queue, self.running, self.done, self.admitted = [], [], set(), set()
        self.next_ticket, self.batch_sizes, self.frames_seen = 1, [], []

    def try_submit(self, frame):
        if len(self.admitted) >= self.max_inflight:
            return DENSIFY_E_AGAIN, 0
        t = self.next_ticket
        self.next_ticket += 1
        self.admitted.add(t)
        self.queue.append(t)
        self.frames_seen.append(frame)
        return DENSIFY_OK, t

    def _progress(self):
        now = self.clock.t
        for b in list(self.running):
            if b[0] <= now:
                self.done.update(b[1])
                self.running.remove(b)
        while self.queue and len(self.running) < self.slots:
            batch = self.queue[: self.max_batch]
            del self.queue[: len(batch)]
            self.batch_sizes.append(len(batch))
            self.running.append((now + self.per_batch_s + self.per_frame_s * len(batch), batch))

    def flush(self, timeout_ns):
        self._progress()
        return DENSIFY_OK

    def poll(self, ticket, timeout_ns):
        self._progress()
        if ticket in self.done:
            self.done.discard(ticket)
            self.admitted.discard(ticket)
            return DENSIFY_OK
        return DENSIFY_PENDING


def test_every_frame_completes_with_latency_at_least_service_time():
    clock = FakeClock()
    dev = FakeDevice(clock, max_inflight=64)
    frames = [[("view", v, s) for s in range(3)] for v in range(4)]
    arr = poisson_arrivals(4, 30.0, 0.5, seed=1)
    st = ServeLoop(dev, frames, clock=clock).run(arr, 0.5, drain_s=1.0)
    assert st.completed == st.offered == len(arr) > 40
    assert min(st.latencies_ms) >= 1000 * (dev.per_batch_s + dev.per_frame_s) - 1e-6
    s = st.summary()
    assert s["latency_ms"]["p50"] <= s["latency_ms"]["p99"] <= s["latency_ms"]["max"]


def test_busy_gpu_batches_arrivals_together():
    clock = FakeClock()
    dev = FakeDevice(clock, max_inflight=64, per_batch_s=20e-3)   # slow device
    frames = [[("view", v, s) for s in range(4)] for v in range(16)]
    arr = poisson_arrivals(16, 30.0, 0.5, seed=2)
    st = ServeLoop(dev, frames, clock=clock).run(arr, 0.5, drain_s=2.0)
    assert st.completed == len(arr)
    assert max(dev.batch_sizes) > 4            # frames that arrived during a batch went out together
    assert sum(dev.batch_sizes) == len(arr)


def test_admission_limit_backs_off_and_recovers():
    clock = FakeClock()
    dev = FakeDevice(clock, max_inflight=2, per_batch_s=5e-3)
    frames = [[("view", v, s) for s in range(4)] for v in range(8)]
    arr = poisson_arrivals(8, 60.0, 0.3, seed=3)
    st = ServeLoop(dev, frames, clock=clock).run(arr, 0.3, drain_s=3.0)
    assert st.refused_again > 0
    assert st.completed == len(arr)


def test_output_slots_are_never_reused_while_in_flight():
    clock = FakeClock()
    dev = FakeDevice(clock, max_inflight=64, per_batch_s=50e-3)
    ring = 2
    frames = [[("view", v, s) for s in range(ring)] for v in range(2)]
    arr = [(0.001 * k, 0) for k in range(10)]          # one view, bursts faster than the device
    in_flight = {}

    orig_submit, orig_poll = dev.try_submit, dev.poll

    def submit(frame):
        st, t = orig_submit(frame)
        if st == DENSIFY_OK:
            assert frame not in in_flight.values(), "output slot reused while in flight"
            in_flight[t] = frame
        return st, t

    def poll(t, timeout):
        r = orig_poll(t, timeout)
        if r == DENSIFY_OK:
            in_flight.pop(t)
        return r

    dev.try_submit, dev.poll = submit, poll
    st = ServeLoop(dev, frames, clock=clock).run(arr, 0.01, drain_s=2.0)
    assert st.completed == 10


def test_poisson_arrivals_rate():
    arr = poisson_arrivals(16, 30.0, 60.0, seed=4)
    assert len(arr) == pytest.approx(16 * 30 * 60, rel=0.05)
    assert all(a[0] <= b[0] for a, b in zip(arr, arr[1:]))


def test_a_full_viewpoint_does_not_hold_up_the_others():
    """Frames wait in one queue per viewpoint: a viewpoint whose output buffers are all in flight
    keeps its later frames back without blocking another viewpoint's frame that arrived after
    them, and each viewpoint's frames are admitted in arrival order."""
    clock = FakeClock()
    dev = FakeDevice(clock, max_inflight=64, per_batch_s=20e-3)
    frames = [[("view", v, s) for s in range(1)] for v in range(2)]   # one output buffer each
    arr = [(0.0001 * k, 0) for k in range(5)] + [(0.0008, 1)]
    st = ServeLoop(dev, frames, clock=clock).run(arr, 0.001, drain_s=2.0)
    assert st.completed == 6
    seen = [f[1] for f in dev.frames_seen]
    # view 1's frame (arrived after all of view 0's) goes out before view 0's second frame
    assert seen.index(1) == 1, seen


def test_a_large_backlog_completes_in_order():
    """Thousands of frames arriving at once: a viewpoint whose output buffers are busy is not offered
    to the device (no refused submits), every frame completes, and each viewpoint's buffers are used
    round-robin."""
    clock = FakeClock()
    dev = FakeDevice(clock, max_inflight=64, per_batch_s=1e-3, per_frame_s=0.0)
    frames = [[("view", v, s) for s in range(2)] for v in range(4)]
    arr = sorted((0.0, v) for v in range(4) for _ in range(500))      # 2000 frames at once
    attempts = []
    orig = dev.try_submit

    def submit(frame):
        attempts.append(frame)
        return orig(frame)

    dev.try_submit = submit
    st = ServeLoop(dev, frames, clock=clock).run(arr, 0.0, drain_s=10.0)
    assert st.completed == 2000
    assert len(attempts) == 2000            # no refusals: a busy viewpoint is not offered at all
    for v in range(4):                      # each viewpoint's buffers are used round-robin
        slots = [f[2] for f in attempts if f[1] == v]
        assert slots == [k % 2 for k in range(500)]
