"""Host logic of the depth-request server (serve.DepthServer.run), on CPU.

The device work is replaced by fakes: a slot's "computation" is a completion
event that fires a fixed service time after the launch, on a simulated clock
that advances 10 microseconds per reading and by the requested amount per
sleep.  What is checked are the scheduling rules themselves:
- every request is served exactly once;
- a camera never has two frames in flight, and its frames go in arrival order;
- a class never has more requests in flight than slots;
- under "fifo" no request is admitted while an older request of another class
  waits;
- "sequential" runs one request at a time;
- a time limit stops admissions and counts the backlog;
- requests from unknown cameras are rejected.
The same loop drives the GPU (tests/test_gpu_serve.py checks that each served
depth equals the pair computed alone).
"""
import collections

import pytest

from paper_2201_11924_gb300 import configs, serve

TICK = 1e-5


class Clock:
    def __init__(self):
        self.t = 0.0

    def perf_counter(self):
        self.t += TICK
        return self.t

    def sleep(self, dt):
        self.t += max(float(dt), 0.0)


class FakeEvent:
    def __init__(self, clock):
        self.clock, self.at = clock, None

    def query(self):
        return self.at is not None and self.clock.t >= self.at


class _Cuda:
    @staticmethod
    def synchronize(dev=None):
        pass


class FakeTorch:
    cuda = _Cuda


def _cam(c, W, H, D):
    return configs.Workload(name=f"cam{c}", W=W, H=H, D=D, win_w=7, win_h=7, P1=7, P2=86, paths=8, uniq=15,
                            lr_max_diff=1, subpixel=True, f=300.0, baseline=0.055, seed=c,
                            scene=configs.SMALL_320.scene)


SIZES = [(160, 96, 48), (224, 128, 96), (320, 180, 128)]


def _server(monkeypatch, n_cams, slots, service):
    """A DepthServer whose launches only schedule a fake completion;
    slots and service (seconds) per class index."""
    clock = Clock()
    monkeypatch.setattr(serve, "time", clock)
    cams = [_cam(c, *SIZES[c % len(SIZES)]) for c in range(n_cams)]
    srv = object.__new__(serve.DepthServer)
    srv.torch, srv.dev, srv.cameras, srv.upload = FakeTorch, None, cams, False
    srv.classes = sorted({(w.W, w.H, w.D) for w in cams})
    srv.slots = {k: [serve.Slot(k, None, None, FakeEvent(clock)) for _ in range(slots[i])]
                 for i, k in enumerate(srv.classes)}
    srv.free = {k: collections.deque(v) for k, v in srv.slots.items()}
    srv.busy = []
    srv.depth = [f"depth of camera {c}" for c in range(n_cams)]
    srv.launches = []

    def launch(slot, req):
        slot.event.at = clock.t + service[srv.classes.index(slot.cls)]
        slot.req = req
        srv.launches.append((clock.t, req.rid))

    srv._launch = launch
    return srv, clock


def _cls(srv, r):
    w = srv.cameras[r.camera]
    return (w.W, w.H, w.D)


def _check_served(srv, trace, done, calls):
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
    # a class: never more requests in flight than slots
    for k, sl in srv.slots.items():
        ev = sorted([(r.admitted, 1) for r in done if _cls(srv, r) == k] +
                    [(r.done, -1) for r in done if _cls(srv, r) == k], key=lambda e: (e[0], e[1]))
        n = 0
        for _, d in ev:
            n += d
            assert n <= len(sl)


@pytest.mark.parametrize("policy", ["fifo", "per_class"])
def test_every_request_is_served_once_within_the_rules(monkeypatch, policy):
    srv, _ = _server(monkeypatch, 12, slots=[2, 2, 1], service=[0.002, 0.003, 0.005])
    trace = serve.poisson_trace(12, rate=1500.0, duration=0.2, seed=11)
    calls = []
    done = srv.run(trace, policy=policy, on_done=lambda r, d: calls.append((r.rid, d)))
    _check_served(srv, trace, done, calls)
    assert srv.backlog == 0 and srv.rejected == []


def test_fifo_admits_no_request_past_an_older_one_of_another_class(monkeypatch):
    srv, _ = _server(monkeypatch, 9, slots=[1, 1, 1], service=[0.004, 0.004, 0.004])
    trace = serve.poisson_trace(9, rate=1000.0, duration=0.1, seed=3)
    done = srv.run(trace, policy="fifo")
    assert len(done) == len(trace)
    eps = 50 * TICK                        # a loop iteration reads the clock a few times
    for b in done:
        for a in done:
            if a.arrival < b.arrival and _cls(srv, a) != _cls(srv, b):
                waiting_then = a.arrival + eps < b.admitted and a.admitted > b.admitted + eps
                assert not waiting_then, (a.rid, b.rid)


def test_sequential_runs_one_request_at_a_time(monkeypatch):
    srv, _ = _server(monkeypatch, 6, slots=[2, 2, 2], service=[0.001, 0.001, 0.001])
    trace = serve.poisson_trace(6, rate=2000.0, duration=0.05, seed=4)
    done = sorted(srv.run(trace, sequential=True), key=lambda r: r.admitted)
    assert len(done) == len(trace)
    for a, b in zip(done, done[1:]):
        assert a.done <= b.admitted


def test_time_limit_stops_admissions_and_counts_the_backlog(monkeypatch):
    # offered load far above capacity: 1 slot per class, 10 ms per request
    srv, _ = _server(monkeypatch, 6, slots=[1, 1, 1], service=[0.01, 0.01, 0.01])
    trace = serve.poisson_trace(6, rate=3000.0, duration=0.1, seed=5)
    limit = 0.05
    done = srv.run(trace, time_limit=limit)
    assert 0 < len(done) < len(trace)
    assert all(t <= limit + 1e-3 for t, _ in srv.launches)
    # every request is finished, lost with the slots at the stop, or backlog
    in_flight_at_stop = len(srv.launches) - len(done)
    assert len(done) + in_flight_at_stop + srv.backlog == len(trace)
    assert all(len(srv.free[k]) == len(v) for k, v in srv.slots.items())     # slots returned


def test_requests_from_unknown_cameras_are_rejected(monkeypatch):
    srv, _ = _server(monkeypatch, 6, slots=[1, 1, 1], service=[0.001, 0.001, 0.001])
    trace = serve.poisson_trace(6, rate=1000.0, duration=0.05, seed=6)
    bad = [serve.Request(10_000 + i, cam, trace[i].arrival) for i, cam in enumerate((-1, 6, 99))]
    mixed = sorted(trace + bad, key=lambda r: r.arrival)
    calls = []
    done = srv.run(mixed, on_done=lambda r, d: calls.append((r.rid, d)))
    assert sorted(r.rid for r in srv.rejected) == [10_000, 10_001, 10_002]
    _check_served(srv, trace, done, calls)
