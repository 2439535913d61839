"""Depth-request server: continuous batching of frames from many cameras.

Each camera has resident device buffers (left, right, depth) sized for its
sensor.  Requests (a camera delivered a new pair) arrive over time; the
server keeps a FIFO of waiting requests per sensor size class and a pool of
compute slots per class.  A slot is one matcher handle (its own scratch memory)
with its own CUDA stream, so the work of all busy slots overlaps on the GPU;
the number of slots per class is decided at start-up from the free device
memory (admission by free HBM).  The loop:

  1. polls the busy slots' completion events and records each finished
     request's latency (arrival to depth ready);
  2. admits, in arrival order within each class, waiting requests into the
     class's free slots (a camera never has two frames in flight, since its
     buffers are reused): uploads the camera's new frame into its resident
     buffers (optional host-to-device copy from pinned memory, on the slot's
     stream), enqueues the depth computation and an event on the slot's
     stream.

Requests that arrive while others run are admitted as soon as a slot of
their class frees up, without waiting for the others: that is the continuous
batching.  All device work goes through the C ABI (libsimsense); torch only
provides memory, streams and events.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass

import numpy as np

from . import simsense


@dataclass
class Request:
    rid: int
    camera: int
    arrival: float               # seconds on the trace clock
    admitted: float = -1.0
    done: float = -1.0


@dataclass
class Slot:
    cls: tuple
    handle: object
    stream: object
    event: object
    req: Request | None = None


def poisson_trace(n_cameras: int, rate: float, duration: float, seed: int):
    """Arrival times (s) and camera ids of a Poisson request stream."""
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate * duration))
    times = np.sort(rng.uniform(0.0, duration, size=n))
    cams = rng.integers(0, n_cameras, size=n)
    return [Request(i, int(c), float(t)) for i, (t, c) in enumerate(zip(times, cams))]


class DepthServer:
    def __init__(self, cameras, frames, slots_per_class: int = 4, hbm_reserve_gb: float = 8.0,
                 upload: bool = True, device=None):
        """cameras: list of Workload (one per camera); frames: dict mapping a
        camera's (W, H, D) class to a list of (left, right) uint8 numpy pairs,
        camera c uses pair c % len(list)."""
        import torch
        self.torch = torch
        self.dev = device or torch.device("cuda", 0)
        self.cameras = cameras
        self.upload = upload
        self.classes = sorted({(w.W, w.H, w.D) for w in cameras})
        # resident per-camera buffers and pinned host frames
        self.left, self.right, self.depth, self.host = [], [], [], []
        pinned = {}
        for c, w in enumerate(cameras):
            key = (w.W, w.H, w.D)
            pool = frames[key]
            k = c % len(pool)
            if (key, k) not in pinned:
                l, r = pool[k]
                pinned[(key, k)] = (torch.from_numpy(l).pin_memory(), torch.from_numpy(r).pin_memory())
            hl, hr = pinned[(key, k)]
            self.host.append((hl, hr))
            self.left.append(hl.to(self.dev))
            self.right.append(hr.to(self.dev))
            self.depth.append(torch.empty((w.H, w.W), dtype=torch.float32, device=self.dev))
        # compute slots per class, as many as free HBM allows (at most slots_per_class)
        self.slots = {k: [] for k in self.classes}
        proto = {}
        for w in cameras:
            proto.setdefault((w.W, w.H, w.D), w)
        for k in self.classes:
            for _ in range(slots_per_class):
                free, _total = torch.cuda.mem_get_info(self.dev)
                h = simsense.SimSense.from_workload(proto[k])
                if free - h.scratch_bytes() < hbm_reserve_gb * 2**30 and self.slots[k]:
                    h.close()
                    break
                self.slots[k].append(Slot(k, h, torch.cuda.Stream(self.dev),
                                          torch.cuda.Event(enable_timing=False)))
        self.free = {k: collections.deque(self.slots[k]) for k in self.classes}
        self.busy: list[Slot] = []

    def slot_counts(self):
        return {f"{k[0]}x{k[1]}_D{k[2]}": len(v) for k, v in self.slots.items()}

    def _launch(self, slot: Slot, req: Request):
        torch = self.torch
        c = req.camera
        with torch.cuda.stream(slot.stream):
            if self.upload:
                self.left[c].copy_(self.host[c][0], non_blocking=True)
                self.right[c].copy_(self.host[c][1], non_blocking=True)
            slot.handle.compute(self.left[c], self.right[c], self.depth[c], stream=slot.stream)
            slot.event.record(slot.stream)
        slot.req = req

    def run(self, trace, time_limit: float | None = None, sequential: bool = False, on_done=None,
            policy: str = "fifo"):
        """Serve a trace in real time; returns the finished requests.

        time_limit: stop admitting and return after this many seconds (the
        requests still waiting are not served).  sequential: at most one
        request on the GPU at a time (the plain per-request path).
        on_done(req, depth): called when a request's depth is ready, before
        its camera's buffers can be reused.
        policy: "fifo" admits strictly in arrival order (a request waits
        while an older one has no free slot, so the served mix is the
        arrival mix); "per_class" lets each class fill its own free slots
        (more concurrency, but under overload the classes' shares of the GPU
        follow their slot counts, not the arrival mix).
        A request from a camera the server does not know is not served: it
        is listed in ``self.rejected`` after the run."""
        waiting = {k: collections.deque() for k in self.classes}
        rejected = []
        busy_cams = set()
        pending = collections.deque(trace)
        finished = []
        t0 = time.perf_counter()
        iters = 0
        busy_sum = 0
        while pending or any(waiting.values()) or self.busy:
            now = time.perf_counter() - t0
            iters += 1
            busy_sum += len(self.busy)
            if time_limit is not None and now > time_limit:
                break
            # 1. completions
            still = []
            for s in self.busy:
                if s.event.query():
                    r = s.req
                    r.done = time.perf_counter() - t0
                    if on_done is not None:
                        on_done(r, self.depth[r.camera])
                    finished.append(r)
                    busy_cams.discard(r.camera)
                    s.req = None
                    self.free[s.cls].append(s)
                else:
                    still.append(s)
            self.busy = still
            # 2. arrivals up to now join their class's queue
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                if not 0 <= r.camera < len(self.cameras):
                    rejected.append(r)
                    continue
                w = self.cameras[r.camera]
                waiting[(w.W, w.H, w.D)].append(r)
            # 3. admissions: classes by the arrival of their oldest waiting
            #    request, each in arrival order into its free slots; a request
            #    whose camera still has a frame in flight waits
            order = sorted(self.classes, key=lambda c: waiting[c][0].arrival if waiting[c] else 1e30)
            for k in order:
                q = waiting[k]
                if policy == "fifo" and q and not self.free[k]:
                    break                       # the oldest waiting request blocks younger ones
                while q and self.free[k] and not (sequential and self.busy):
                    if policy == "fifo":
                        heads = [waiting[c][0].arrival for c in self.classes if c != k and waiting[c]]
                        if heads and q[0].arrival > min(heads):
                            break               # another class holds an older request
                    pick = None
                    for j in range(min(len(q), 8)):
                        if q[j].camera not in busy_cams:
                            pick = j
                            break
                    if pick is None:
                        break
                    r = q[pick]
                    del q[pick]
                    s = self.free[k].popleft()
                    r.admitted = time.perf_counter() - t0
                    self._launch(s, r)
                    busy_cams.add(r.camera)
                    self.busy.append(s)
            if not self.busy and not any(waiting.values()) and pending:
                dt = pending[0].arrival - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(min(dt, 0.001))
        self.torch.cuda.synchronize(self.dev)
        # requests still on the GPU at a time-limit stop finish unrecorded
        for s in self.busy:
            s.req = None
            self.free[s.cls].append(s)
        self.busy = []
        self.backlog = sum(len(q) for q in waiting.values()) + len(pending)
        self.rejected = rejected
        self.stats = {"iterations": iters, "mean_busy_slots": busy_sum / max(1, iters)}
        return finished

    def close(self):
        for v in self.slots.values():
            for s in v:
                s.handle.close()


def latency_stats(finished, duration, cameras=None):
    lat = np.array([r.done - r.arrival for r in finished]) if finished else np.zeros(0)
    cells = sum(cameras[r.camera].cells for r in finished) if cameras is not None else None
    return {
        "served": len(finished),
        "served_cells_per_s": cells / duration if cells is not None and duration > 0 else None,
        "served_per_s": len(finished) / duration if duration > 0 else 0.0,
        "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
        "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
        "mean_ms": float(lat.mean() * 1e3) if len(lat) else None,
    }
