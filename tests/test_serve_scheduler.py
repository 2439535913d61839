"""Host logic of the depth-request server (serve.DepthServer.run), on CPU.

The device side is replaced by a fake backend: a slot's "computation" is a
completion notice that arrives a fixed service time after the launch, on a
simulated clock that advances 10 microseconds per reading, by the requested
amount per sleep, and to the next notice (or the time-out) per blocking wait.
What is checked are the scheduling rules themselves:
- every request is served exactly once;
- a camera never has two frames in flight, and its frames go in arrival order;
- a class never has more requests in flight than its slot cap;
- the slots never hold more device memory than the server's budget: slots are
  created when a request needs one and the budget covers it, idle slots of
  other classes are released when a class needs their memory, and a request
  waits when neither is possible;
- under "fifo" no request is admitted while an older request of another class
  waits;
- "sequential" runs one request at a time;
- a time limit stops admissions and counts the backlog;
- requests from unknown cameras are rejected;
- the loop blocks on completions instead of spinning.
The same loop drives the GPU (tests/test_gpu_serve.py checks that each served
depth equals the pair computed alone).
"""
import collections

import pytest

from paper_2201_11924_gb300 import configs, serve

TICK = 1e-5
GB = 2**30


class FakeBackend:
    def __init__(self, service, scratch):
        self.t = 0.0
        self.service = service          # class -> seconds
        self.scratch = scratch          # class -> bytes
        self.inflight = {}              # tag -> completion time
        self.launches = []              # (time, request id, class)
        self.events = []                # (time, +bytes / -bytes) of slot creation and release
        self.sleeps = 0

    def clock(self):
        self.t += TICK
        return self.t

    def sleep(self, dt):
        self.sleeps += 1
        self.t += max(float(dt), 0.0)

    def free_memory(self):
        return 1 << 50

    def prepare(self, cameras, frames):
        self.cameras = cameras

    def scratch_bytes(self, wl):
        return self.scratch[(wl.W, wl.H, wl.D)]

    def create_slot(self, slot, wl):
        self.events.append((self.t, self.scratch[slot.cls]))

    def destroy_slot(self, slot):
        assert slot.req is None and slot.tag not in self.inflight
        self.events.append((self.t, -self.scratch[slot.cls]))

    def launch(self, slot, req):
        assert slot.tag not in self.inflight
        self.inflight[slot.tag] = self.t + self.service[slot.cls]
        self.launches.append((self.t, req.rid, slot.cls))

    def result(self, req):
        return f"depth of camera {req.camera}"

    def wait(self, timeout):
        if self.inflight:
            nxt = min(self.inflight.values())
            if timeout is None or nxt <= self.t + timeout:
                self.t = max(self.t, nxt)
            else:
                self.t += timeout
        elif timeout:
            self.t += timeout
        done = [tag for tag, at in self.inflight.items() if at <= self.t]
        for tag in done:
            del self.inflight[tag]
        return done

    def synchronize(self):
        if self.inflight:
            self.t = max(self.t, max(self.inflight.values()))

    def close(self):
        pass


def _cam(c, W, H, D):
    return configs.Workload(name=f"cam{c}", W=W, H=H, D=D, win_w=7, win_h=7, P1=7, P2=86, paths=8, uniq=15,
                            lr_max_diff=1, subpixel=True, f=300.0, baseline=0.055, seed=c,
                            scene=configs.SMALL_320.scene)


SIZES = [(160, 96, 48), (224, 128, 96), (320, 180, 128)]


def _server(n_cams, cap, service, scratch=(1 * GB, 2 * GB, 3 * GB), budget=64 * GB, sizes=SIZES):
    """A DepthServer on the fake backend: slot cap per class, service time
    (s) and slot bytes per class index, and the server's HBM budget."""
    cams = [_cam(c, *sizes[c % len(sizes)]) for c in range(n_cams)]
    classes = sorted({(w.W, w.H, w.D) for w in cams})
    be = FakeBackend({k: service[i] for i, k in enumerate(classes)}, {k: scratch[i] for i, k in enumerate(classes)})
    srv = serve.DepthServer(cams, {}, slots_per_class=cap, hbm_budget=budget, backend=be)
    return srv, be


def _cls(srv, r):
    w = srv.cameras[r.camera]
    return (w.W, w.H, w.D)


def _check_memory(srv, be):
    used = 0
    for _, b in sorted(be.events, key=lambda e: e[0]):
        used += b
        assert 0 <= used <= srv.hbm_budget
    assert used == srv.hbm_used


def _check_served(srv, be, trace, done, calls):
    assert sorted(r.rid for r in done) == sorted(r.rid for r in trace)
    assert sorted(rid for rid, _ in calls) == sorted(r.rid for r in trace)       # on_done once each
    assert all(d == f"depth of camera {r.camera}" for (rid, d), r in zip(calls, done))
    for r in done:
        assert r.arrival <= r.admitted < r.done
    # a camera: one frame in flight at a time, in arrival order
    by_cam = collections.defaultdict(list)
    for r in done:
        by_cam[r.camera].append(r)
    for rs in by_cam.values():
        rs.sort(key=lambda r: r.admitted)
        assert [r.arrival for r in rs] == sorted(r.arrival for r in rs)
        for a, b in zip(rs, rs[1:]):
            assert a.done <= b.admitted
    # a class: never more requests in flight than its slot cap
    for k in srv.classes:
        ev = sorted([(r.admitted, 1) for r in done if _cls(srv, r) == k] +
                    [(r.done, -1) for r in done if _cls(srv, r) == k], key=lambda e: (e[0], e[1]))
        n = 0
        for _, d in ev:
            n += d
            assert n <= srv.max_slots
    _check_memory(srv, be)


@pytest.mark.parametrize("policy", ["fifo", "per_class"])
def test_every_request_is_served_once_within_the_rules(policy):
    srv, be = _server(12, cap=2, service=[0.002, 0.003, 0.005])
    trace = serve.poisson_trace(12, rate=1500.0, duration=0.2, seed=11)
    calls = []
    done = srv.run(trace, policy=policy, on_done=lambda r, d: calls.append((r.rid, d)))
    _check_served(srv, be, trace, done, calls)
    assert srv.backlog == 0 and srv.rejected == []


def test_fifo_admits_no_request_past_an_older_one_of_another_class():
    srv, _ = _server(9, cap=1, service=[0.004, 0.004, 0.004])
    trace = serve.poisson_trace(9, rate=1000.0, duration=0.1, seed=3)
    done = srv.run(trace, policy="fifo")
    assert len(done) == len(trace)
    eps = 50 * TICK                        # a loop iteration reads the clock a few times
    for b in done:
        for a in done:
            if a.arrival < b.arrival and _cls(srv, a) != _cls(srv, b):
                waiting_then = a.arrival + eps < b.admitted and a.admitted > b.admitted + eps
                assert not waiting_then, (a.rid, b.rid)


def test_sequential_runs_one_request_at_a_time():
    srv, _ = _server(6, cap=2, service=[0.001, 0.001, 0.001])
    trace = serve.poisson_trace(6, rate=2000.0, duration=0.05, seed=4)
    done = sorted(srv.run(trace, sequential=True), key=lambda r: r.admitted)
    assert len(done) == len(trace)
    for a, b in zip(done, done[1:]):
        assert a.done <= b.admitted


def test_time_limit_stops_admissions_and_counts_the_backlog():
    # offered load far above capacity: 1 slot per class, 10 ms per request
    srv, be = _server(6, cap=1, service=[0.01, 0.01, 0.01])
    trace = serve.poisson_trace(6, rate=3000.0, duration=0.1, seed=5)
    limit = 0.05
    done = srv.run(trace, time_limit=limit)
    assert 0 < len(done) < len(trace)
    assert all(t <= limit + 1e-3 for t, _, _ in be.launches)
    # every request is finished, lost with the slots at the stop, or backlog
    in_flight_at_stop = len(be.launches) - len(done)
    assert len(done) + in_flight_at_stop + srv.backlog == len(trace)
    assert all(len(srv.free[k]) == len(v) for k, v in srv.slots.items())     # slots returned


def test_requests_from_unknown_cameras_are_rejected():
    srv, be = _server(6, cap=1, service=[0.001, 0.001, 0.001])
    trace = serve.poisson_trace(6, rate=1000.0, duration=0.05, seed=6)
    bad = [serve.Request(10_000 + i, cam, trace[i].arrival) for i, cam in enumerate((-1, 6, 99))]
    mixed = sorted(trace + bad, key=lambda r: r.arrival)
    calls = []
    done = srv.run(mixed, on_done=lambda r, d: calls.append((r.rid, d)))
    assert sorted(r.rid for r in srv.rejected) == [10_000, 10_001, 10_002]
    _check_served(srv, be, trace, done, calls)


def test_admission_is_limited_by_the_hbm_budget():
    # slots of 1, 2 and 3 GB under a 4 GB budget, up to 3 slots per class: at
    # most 4 small or 2 medium slots fit, and a large request has to wait for
    # memory that in-flight work of other classes holds
    srv, be = _server(12, cap=3, service=[0.002, 0.003, 0.004], budget=4 * GB)
    trace = serve.poisson_trace(12, rate=2000.0, duration=0.2, seed=21)
    calls = []
    done = srv.run(trace, on_done=lambda r, d: calls.append((r.rid, d)))
    _check_served(srv, be, trace, done, calls)
    assert srv.hbm_peak <= 4 * GB
    assert srv.released > 0                          # idle slots gave their memory to other classes
    assert srv.created > len(srv.classes)
    # some request waited for memory while a slot of its class was missing
    # and another class held the budget
    large = max(srv.classes)
    assert any(r.admitted - r.arrival > 0.001 for r in done if _cls(srv, r) == large)


def test_slots_follow_the_request_mix():
    # first only small cameras, then only large ones: the large class gets
    # the memory the idle small slots held
    sizes = [(160, 96, 48), (320, 180, 128)]
    srv, be = _server(8, cap=4, service=[0.002, 0.002], scratch=(1 * GB, 3 * GB), budget=6 * GB, sizes=sizes)
    small = [c for c in range(8) if c % 2 == 0]
    large = [c for c in range(8) if c % 2 == 1]
    trace = [serve.Request(i, small[i % 4], 0.0005 * i) for i in range(40)]
    trace += [serve.Request(100 + i, large[i % 4], 0.05 + 0.0005 * i) for i in range(40)]
    done = srv.run(trace)
    assert len(done) == len(trace)
    k_small, k_large = sorted(srv.classes)
    assert len(srv.slots[k_large]) == 2                 # 2 x 3 GB once the small slots are gone
    assert len(srv.slots[k_small]) == 0
    _check_memory(srv, be)


def test_a_request_whose_slot_can_never_fit_is_not_admitted():
    # a budget below one slot of the class: its requests stay in the backlog,
    # the other classes are served (per-class admission)
    srv, _ = _server(6, cap=2, service=[0.001, 0.001, 0.001], scratch=(1 * GB, 1 * GB, 8 * GB), budget=4 * GB)
    trace = serve.poisson_trace(6, rate=1000.0, duration=0.05, seed=8)
    big = max(srv.classes)
    done = srv.run(trace, time_limit=0.2, policy="per_class")
    assert all(_cls(srv, r) != big for r in done)
    assert srv.backlog == sum(1 for r in trace if _cls(srv, r) == big)


def test_the_loop_blocks_instead_of_spinning():
    # with 1 ms requests arriving every ~2 ms the loop wakes for arrivals and
    # completions only: a few iterations per request, not thousands
    srv, _ = _server(6, cap=2, service=[0.001, 0.001, 0.001])
    trace = serve.poisson_trace(6, rate=500.0, duration=0.2, seed=9)
    done = srv.run(trace)
    assert len(done) == len(trace)
    assert srv.stats["iterations"] <= 4 * len(trace) + 10
