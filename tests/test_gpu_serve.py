"""Continuous-batching server: the depth of every request served in a mix of
overlapping requests from many cameras is exactly the depth of the same pair
computed alone (same kernels, each slot with its own scratch and stream)."""
import numpy as np
import pytest

from paper_2201_11924_gb300 import configs, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2201_11924_gb300 import _build, simsense
    _build.build()
    return simsense


def _cam(c, W, H, D):
    return configs.Workload(name=f"cam{c}", W=W, H=H, D=D, win_w=7, win_h=7, P1=7, P2=86, paths=8, uniq=15,
                            lr_max_diff=1, subpixel=True, f=300.0, baseline=0.055, seed=7000 + c,
                            scene=configs.SMALL_320.scene)


def test_served_results_equal_alone(lib):
    import torch
    from paper_2201_11924_gb300 import serve
    sizes = [(160, 96, 48), (224, 128, 96), (320, 180, 128)]
    cams = [_cam(c, *sizes[c % 3]) for c in range(12)]
    frames = {}
    for w in cams:
        key = (w.W, w.H, w.D)
        frames.setdefault(key, [])
        if len(frames[key]) < 2:
            p = scenes.make_pair(w)
            frames[key].append((p["left"], p["right"]))
    srv = serve.DepthServer(cams, frames, slots_per_class=3, hbm_reserve_gb=1.0)
    trace = serve.poisson_trace(len(cams), rate=3000.0, duration=0.15, seed=5)
    got = {}
    done = srv.run(trace, on_done=lambda r, d: got.__setitem__(r.rid, d.clone()))
    assert len(done) == len(trace) and len(got) == len(trace)
    # requests really overlapped on the device: some request was admitted while
    # an earlier-admitted one was still running
    by_adm = sorted(done, key=lambda q: q.admitted)
    assert any(b.admitted < a.done for a, b in zip(by_adm, by_adm[1:]))
    alone = {}
    for c, w in enumerate(cams):
        key = (w.W, w.H, w.D)
        l, r = frames[key][c % len(frames[key])]
        with lib.SimSense.from_workload(w) as m:
            alone[c] = m.compute(torch.from_numpy(l).cuda(), torch.from_numpy(r).cuda()).cpu().numpy()
    for r in done:
        np.testing.assert_array_equal(got[r.rid].cpu().numpy(), alone[r.camera])
    srv.close()
