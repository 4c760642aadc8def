"""Serving loop over a densify context: many viewpoints, frames arriving in
real time, continuous batching.

Each viewpoint produces frames at ``fps`` with Poisson-jittered arrival times
(exponential inter-arrival gaps of mean 1/fps). The loop

  1. admits every frame whose arrival time has passed with densify_submit,
     in arrival order over the viewpoints (each viewpoint's frames wait in
     its own queue, so a turn costs the same whatever the backlog); a frame
     refused with DENSIFY_E_AGAIN (all slots admitted or the scratch arena
     full) stays queued and is retried on the next turn,
  2. calls densify_flush(ctx, 0), which sends the queued frames to the GPU as
     one batch as soon as a launch slot is free (frames that arrived while the
     GPU was busy go out together),
  3. polls outstanding tickets without blocking and records each frame's
     latency (completion time minus arrival time).

Inputs and outputs stay on the device: each viewpoint owns ``ring`` output
buffer sets, reused round-robin, so a frame never overwrites the outputs of
one still in flight (a viewpoint whose ring is full backs off like E_AGAIN).

The loop only orders calls; all densification runs in the library.
"""
from __future__ import annotations

import heapq
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from .densify import DENSIFY_E_AGAIN, DENSIFY_OK, DENSIFY_PENDING


@dataclass
class ServeStats:
    offered: int = 0
    completed: int = 0
    refused_again: int = 0
    duration_s: float = 0.0
    latencies_ms: list = field(default_factory=list)
    batches: int = 0

    def summary(self):
        lat = np.asarray(self.latencies_ms, dtype=np.float64)
        pct = (lambda q: float(np.percentile(lat, q))) if lat.size else (lambda q: None)
        return {
            "offered_frames": self.offered,
            "completed_frames": self.completed,
            "frames_per_s": self.completed / self.duration_s if self.duration_s > 0 else 0.0,
            "latency_ms": {"p50": pct(50), "p90": pct(90), "p99": pct(99),
                           "max": float(lat.max()) if lat.size else None},
            "e_again_retries": self.refused_again,
        }


def poisson_arrivals(n_views: int, fps: float, duration_s: float, seed: int = 0):
    """Sorted (time, view) arrivals: per view, exponential gaps of mean 1/fps."""
    rng = np.random.default_rng(seed)
    out = []
    for v in range(n_views):
        t = rng.uniform(0.0, 1.0 / fps)
        while t < duration_s:
            out.append((t, v))
            t += rng.exponential(1.0 / fps)
    out.sort()
    return out


class ServeLoop:
    """``densifier`` exposes try_submit(frame) -> (status, ticket),
    flush(timeout_ns) and poll(ticket, timeout_ns) -> status (the Densifier
    class, or a stand-in with the same methods). ``frames[v][slot]`` is the
    densify_frame of viewpoint v's output slot."""

    def __init__(self, densifier, frames, clock=time.perf_counter, idle_sleep_s: float = 0.0):
        self.d = densifier
        self.frames = frames
        self.ring = len(frames[0])
        self.clock = clock
        self.idle_sleep_s = idle_sleep_s

    def run(self, arrivals, duration_s: float, drain_s: float = 5.0) -> ServeStats:
        st = ServeStats(offered=len(arrivals))
        waiting = [deque() for _ in self.frames]   # per viewpoint: arrival times not yet admitted
        outstanding = {}              # ticket -> (arrival time, view, slot)
        busy = [[False] * self.ring for _ in self.frames]
        next_slot = [0] * len(self.frames)
        backlog = 0
        i = 0
        t0 = self.clock()
        end = duration_s + drain_s
        while True:
            now = self.clock() - t0
            while i < len(arrivals) and arrivals[i][0] <= now:
                waiting[arrivals[i][1]].append(arrivals[i][0])
                backlog += 1
                i += 1
            # admit in arrival order over the viewpoints whose next output slot is free (a viewpoint's
            # later frames wait behind its first); E_AGAIN ends admission for this turn. The heap holds
            # one entry per viewpoint, so a turn costs O(viewpoints), whatever the backlog.
            heads = [(q[0], v) for v, q in enumerate(waiting) if q and not busy[v][next_slot[v]]]
            heapq.heapify(heads)
            while heads:
                ta, v = heapq.heappop(heads)
                slot = next_slot[v]
                status, ticket = self.d.try_submit(self.frames[v][slot])
                if status == DENSIFY_E_AGAIN:
                    st.refused_again += 1
                    break
                waiting[v].popleft()
                backlog -= 1
                busy[v][slot] = True
                next_slot[v] = (slot + 1) % self.ring
                outstanding[ticket] = (ta, v, slot)
                if waiting[v] and not busy[v][next_slot[v]]:
                    heapq.heappush(heads, (waiting[v][0], v))
            self.d.flush(0)
            done = []
            for ticket, (ta, v, slot) in outstanding.items():
                r = self.d.poll(ticket, 0)
                if r == DENSIFY_OK:
                    done.append(ticket)
                    st.latencies_ms.append(1000.0 * (self.clock() - t0 - ta))
                    busy[v][slot] = False
                elif r != DENSIFY_PENDING:
                    raise RuntimeError(f"poll failed with status {r}")
            for t in done:
                del outstanding[t]
            st.completed += len(done)
            if i >= len(arrivals) and not backlog and not outstanding:
                break
            if now > end:
                break
            if not done and self.idle_sleep_s:
                time.sleep(self.idle_sleep_s)
        st.duration_s = max(self.clock() - t0, 1e-9)
        return st
