"""Depth-request server: continuous batching of frames from many cameras.

Each camera has resident device buffers (left, right, depth) sized for its
sensor.  Requests (a camera delivered a new pair) arrive over time; the
server keeps a FIFO of waiting requests per sensor size class and, per class,
compute slots.  A slot is one matcher handle (its own scratch memory) with its
own CUDA stream, so the work of all busy slots overlaps on the GPU.

Admission by free HBM: the server owns a device-memory budget (the free
memory at start-up minus a reserve, or a given number of bytes) and tracks
what its slots hold.  A request is admitted into a free slot of its class; if
there is none, a new slot is created only when the budget still covers its
scratch, otherwise idle slots of other classes are released (least recently
used first) to make room as the request mix changes; if that is not enough
either, the request waits until a slot or memory frees up.

The loop:
  1. takes the completion notices of finished requests (the library writes a
     request's tag to a pipe once its stream has reached it) and records each
     request's latency (arrival to depth ready);
  2. moves the requests that have arrived into their class's queue;
  3. admits waiting requests in arrival order (a camera never has two frames
     in flight, since its buffers are reused): uploads the camera's new frame
     into its resident buffers (optional host-to-device copy from pinned
     memory, on the slot's stream), enqueues the depth computation and the
     completion notice on the slot's stream;
  4. blocks on the notice pipe until the next completion or the next arrival,
     whichever comes first (no spinning on events).

Requests that arrive while others run are admitted as soon as a slot of their
class (or the memory for one) is free, without waiting for the others: that is
the continuous batching.  All device work goes through the C ABI
(libsimsense); torch only provides memory and streams.  The device side sits
behind a small backend interface (GpuBackend), so the scheduling rules are
tested on the CPU with a fake backend on a simulated clock.
"""
from __future__ import annotations

import collections
import ctypes
import os
import select
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
    tag: int
    handle: object = None
    stream: object = None
    req: Request | None = None
    last_used: float = 0.0


def poisson_trace(n_cameras: int, rate: float, duration: float, seed: int):
    """Arrival times (s) and camera ids of a Poisson request stream."""
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate * duration))
    times = np.sort(rng.uniform(0.0, duration, size=n))
    cams = rng.integers(0, n_cameras, size=n)
    return [Request(i, int(c), float(t)) for i, (t, c) in enumerate(zip(times, cams))]


class GpuBackend:
    """Device side of the server: per-camera resident buffers, slots (a
    handle and a stream each), launches, and completion notices through a
    pipe that the library writes when a slot's stream has finished."""

    def __init__(self, device=None, upload: bool = True):
        import torch
        self.torch = torch
        self.dev = device or torch.device("cuda", 0)
        self.upload = upload
        self.lib = simsense.load()
        self.lib.simsense_notify_on_completion.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_ulonglong]
        self.lib.simsense_notify_on_completion.restype = ctypes.c_int
        self.rfd, self.wfd = os.pipe()
        os.set_blocking(self.rfd, False)
        self._scratch = {}

    def clock(self):
        return time.perf_counter()

    def sleep(self, dt):
        if dt > 0:
            time.sleep(dt)

    def free_memory(self):
        free, _total = self.torch.cuda.mem_get_info(self.dev)
        return free

    def prepare(self, cameras, frames):
        """Resident device buffers of every camera and its pinned host frame."""
        torch = self.torch
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

    def scratch_bytes(self, wl) -> int:
        """Device bytes one slot of wl's class holds (measured once per class)."""
        key = (wl.W, wl.H, wl.D)
        if key not in self._scratch:
            with simsense.SimSense.from_workload(wl) as h:
                self._scratch[key] = h.scratch_bytes()
        return self._scratch[key]

    def create_slot(self, slot: Slot, wl):
        slot.handle = simsense.SimSense.from_workload(wl)
        slot.stream = self.torch.cuda.Stream(self.dev)

    def destroy_slot(self, slot: Slot):
        slot.handle.close()
        slot.handle = None
        slot.stream = None

    def launch(self, slot: Slot, req: Request):
        torch = self.torch
        c = req.camera
        with torch.cuda.stream(slot.stream):
            if self.upload:
                self.left[c].copy_(self.host[c][0], non_blocking=True)
                self.right[c].copy_(self.host[c][1], non_blocking=True)
            slot.handle.compute(self.left[c], self.right[c], self.depth[c], stream=slot.stream)
        rc = self.lib.simsense_notify_on_completion(ctypes.c_void_p(slot.stream.cuda_stream), self.wfd, slot.tag)
        if rc != 0:
            raise simsense.SimsenseError(rc, "simsense_notify_on_completion")

    def result(self, req: Request):
        return self.depth[req.camera]

    def wait(self, timeout):
        """Tags of finished slots: blocks up to `timeout` seconds (None =
        until one finishes) when none is ready."""
        if timeout is None or timeout > 0:
            select.select([self.rfd], [], [], timeout)
        tags = []
        while True:
            try:
                b = os.read(self.rfd, 8 * 256)
            except BlockingIOError:
                break
            if not b:
                break
            tags.extend(int(t) for t in np.frombuffer(b[: len(b) // 8 * 8], dtype=np.uint64))
            if len(b) % 8:                          # a notice is one 8-byte write: never split
                raise RuntimeError("partial completion notice")
        return tags

    def synchronize(self):
        self.torch.cuda.synchronize(self.dev)

    def close(self):
        os.close(self.rfd)
        os.close(self.wfd)


class DepthServer:
    def __init__(self, cameras, frames, slots_per_class: int = 4, hbm_budget: int | None = None,
                 hbm_reserve_gb: float = 8.0, upload: bool = True, device=None, backend=None):
        """cameras: list of Workload (one per camera); frames: dict mapping a
        camera's (W, H, D) class to a list of (left, right) uint8 numpy pairs,
        camera c uses pair c % len(list).  slots_per_class caps the slots of
        one class; hbm_budget (bytes) is the device memory the slots may hold,
        by default the free memory now minus hbm_reserve_gb."""
        self.backend = backend or GpuBackend(device, upload)
        self.cameras = cameras
        self.classes = sorted({(w.W, w.H, w.D) for w in cameras})
        self.proto = {}
        for w in cameras:
            self.proto.setdefault((w.W, w.H, w.D), w)
        self.backend.prepare(cameras, frames)
        self.max_slots = slots_per_class
        self.scratch = {k: int(self.backend.scratch_bytes(self.proto[k])) for k in self.classes}
        if hbm_budget is None:
            hbm_budget = max(0, int(self.backend.free_memory() - hbm_reserve_gb * 2**30))
        self.hbm_budget = int(hbm_budget)
        self.hbm_used = 0
        self.hbm_peak = 0
        self.slots = {k: [] for k in self.classes}
        self.free = {k: collections.deque() for k in self.classes}
        self.by_tag = {}
        self._next_tag = 0
        self.created = 0
        self.released = 0
        self.busy: list[Slot] = []
        # one slot per class up front, where the budget allows
        for k in self.classes:
            s = self._grow(k, now=0.0)
            if s is not None:
                self.free[k].append(s)

    # ------------------------------------------------------------ slots
    def slot_counts(self):
        return {f"{k[0]}x{k[1]}_D{k[2]}": len(v) for k, v in self.slots.items()}

    def hbm_summary(self):
        return {"budget_bytes": self.hbm_budget, "used_bytes": self.hbm_used, "peak_bytes": self.hbm_peak,
                "slot_bytes": {f"{k[0]}x{k[1]}_D{k[2]}": v for k, v in self.scratch.items()},
                "slots_created": self.created, "slots_released": self.released}

    def _release(self, s: Slot):
        self.backend.destroy_slot(s)
        self.slots[s.cls].remove(s)
        del self.by_tag[s.tag]
        self.hbm_used -= self.scratch[s.cls]
        self.released += 1

    def _grow(self, k, now):
        """A new slot of class k if the cap and the HBM budget allow, after
        releasing idle slots of other classes (least recently used first) as
        far as needed; None otherwise."""
        if len(self.slots[k]) >= self.max_slots:
            return None
        need = self.scratch[k]
        if self.hbm_used + need > self.hbm_budget:
            idle = sorted((s for c in self.classes if c != k for s in self.free[c]), key=lambda s: s.last_used)
            freeable = sum(self.scratch[s.cls] for s in idle)
            if self.hbm_used - freeable + need > self.hbm_budget:
                return None                      # even releasing every idle slot would not make room
            for s in idle:
                if self.hbm_used + need <= self.hbm_budget:
                    break
                self.free[s.cls].remove(s)
                self._release(s)
        s = Slot(k, self._next_tag, last_used=now)
        self._next_tag += 1
        self.backend.create_slot(s, self.proto[k])
        self.slots[k].append(s)
        self.by_tag[s.tag] = s
        self.hbm_used += need
        self.hbm_peak = max(self.hbm_peak, self.hbm_used)
        self.created += 1
        return s

    # ------------------------------------------------------------ loop
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
        be = self.backend
        waiting = {k: collections.deque() for k in self.classes}
        rejected = []
        busy_cams = set()
        pending = collections.deque(trace)
        finished = []
        t0 = be.clock()
        iters = 0
        busy_sum = 0
        waits = 0
        tags = []
        while pending or any(waiting.values()) or self.busy:
            now = be.clock() - t0
            iters += 1
            busy_sum += len(self.busy)
            if time_limit is not None and now > time_limit:
                break
            # 1. completions (notices taken by the last wait)
            for tag in tags:
                s = self.by_tag.get(tag)
                if s is None or s.req is None:
                    continue                    # a notice of work abandoned at an earlier time-limit stop
                r = s.req
                r.done = be.clock() - t0
                if on_done is not None:
                    on_done(r, be.result(r))
                finished.append(r)
                busy_cams.discard(r.camera)
                s.req = None
                s.last_used = r.done
                self.busy.remove(s)
                self.free[s.cls].append(s)
            tags = []
            # 2. arrivals up to now join their class's queue
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                if not 0 <= r.camera < len(self.cameras):
                    rejected.append(r)
                    continue
                w = self.cameras[r.camera]
                waiting[(w.W, w.H, w.D)].append(r)
            # 3. admissions: classes by the arrival of their oldest waiting
            #    request, each in arrival order into its free slots (new ones
            #    while the HBM budget allows); a request whose camera still
            #    has a frame in flight waits
            order = sorted(self.classes, key=lambda c: waiting[c][0].arrival if waiting[c] else 1e30)
            for k in order:
                q = waiting[k]
                blocked = False
                while q and not (sequential and self.busy):
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
                    if self.free[k]:
                        s = self.free[k].popleft()
                    else:
                        s = self._grow(k, now)
                        if s is None:
                            blocked = True      # no slot and no memory for one: wait
                            break
                    r = q[pick]
                    del q[pick]
                    r.admitted = be.clock() - t0
                    s.req = r
                    s.last_used = r.admitted
                    be.launch(s, r)
                    busy_cams.add(r.camera)
                    self.busy.append(s)
                if policy == "fifo" and blocked:
                    break                       # the oldest waiting request blocks younger ones
            # 4. block until the next completion or the next arrival (or the
            #    time limit), if there is anything left to wait for
            if not self.busy and not pending:
                # done; or requests wait that nothing will ever admit (no
                # work in flight to free a slot, a camera or memory)
                break
            now = be.clock() - t0
            timeout = None
            if pending:
                timeout = max(0.0, pending[0].arrival - now)
            if time_limit is not None:
                timeout = max(0.0, min(timeout if timeout is not None else 1e30, time_limit - now))
            if self.busy:
                waits += 1
                tags = be.wait(timeout)
            elif timeout is not None and timeout > 0:
                be.sleep(timeout)
        be.synchronize()
        # requests still on the GPU at a time-limit stop finish unrecorded
        for s in self.busy:
            s.req = None
            self.free[s.cls].append(s)
        be.wait(0.0)                            # drain their notices
        self.busy = []
        self.backlog = sum(len(q) for q in waiting.values()) + len(pending)
        self.rejected = rejected
        self.stats = {"iterations": iters, "blocking_waits": waits, "mean_busy_slots": busy_sum / max(1, iters)}
        return finished

    def close(self):
        for k in self.classes:
            for s in list(self.slots[k]):
                self._release(s)
            self.free[k].clear()
        self.backend.close()


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
