"""IR image formation on the GPU (arxiv 2201.11924 Sec. VI-A/VI-B) against the
CPU oracle, through the C ABI: both evaluate the scene in fp64 with correctly
rounded operations in the same order, so the rendered images agree bit for
bit.  Then the whole simulated sensor runs on the device (render, noise,
depth) and matches the oracle stage on the same noisy pair."""
import numpy as np
import pytest

import oracle
from paper_2201_11924_gb300 import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2201_11924_gb300 import _build, simsense
    _build.build()
    return simsense


def _scene(seed, n_spheres=6, n_rects=4):
    rng = np.random.default_rng(seed)
    prims = [oracle.rectangle((0.0, 0.0, 2.5), (3.0, 0.0, 0.0), (0.0, 2.0, 0.0), albedo=0.7)]   # back wall
    for _ in range(n_rects):
        c = (rng.uniform(-0.6, 0.6), rng.uniform(-0.4, 0.4), rng.uniform(0.8, 2.2))
        a, b = rng.uniform(-0.4, 0.4, 2)
        u = (rng.uniform(0.1, 0.4) * np.cos(a), 0.0, rng.uniform(0.1, 0.4) * np.sin(a))
        v = (0.0, rng.uniform(0.1, 0.3) * np.cos(b), rng.uniform(0.1, 0.3) * np.sin(b))
        prims.append(oracle.rectangle(c, u, v, albedo=rng.uniform(0.2, 1.0), metallic=rng.uniform(0, 1),
                                      roughness=rng.uniform(0.1, 0.9), transmission=rng.uniform(0, 0.5)))
    for _ in range(n_spheres):
        c = (rng.uniform(-0.6, 0.6), rng.uniform(-0.4, 0.4), rng.uniform(0.6, 2.2))
        prims.append(oracle.sphere(c, rng.uniform(0.05, 0.2), albedo=rng.uniform(0.2, 1.0),
                                   metallic=rng.uniform(0, 1), roughness=rng.uniform(0.1, 0.9),
                                   transmission=rng.uniform(0, 0.5)))
    return prims


def _args(W, H):
    f = 0.9 * W
    return dict(W=W, H=H, f=f, cx=(W - 1) / 2, cy=(H - 1) / 2, baseline=0.055, proj=(0.02, 0.0, 0.0), pf=f,
                pcx=(W - 1) / 2, pcy=(H - 1) / 2, power=1.2, ambient=0.04, gain=350.0)


@pytest.mark.parametrize("W,H,seed", [(160, 120, 1), (333, 97, 2), (640, 360, 3)])
def test_render_matches_oracle_bit_for_bit(lib, W, H, seed):
    import torch
    pat = (np.random.default_rng(seed).random((H, W)) < 0.15).astype(np.uint8) * 230 + 20
    prims = _scene(seed)
    a = _args(W, H)
    gl, gr = lib.render_ir(prims, torch.from_numpy(pat).cuda(), **a)
    ol, orr, _, _ = oracle.render(prims, pat, **a)
    assert np.array_equal(gl.cpu().numpy(), ol)
    assert np.array_equal(gr.cpu().numpy(), orr)
    assert (ol > 0).mean() > 0.5                       # the scene fills the view


def test_simulated_sensor_end_to_end_on_the_device(lib):
    # render -> sensor noise -> depth stage, all on the GPU; the depth matches
    # the oracle stage run on the same noisy pair
    import torch
    W, H, D = 320, 240, 64
    pat = (np.random.default_rng(9).random((H, W)) < 0.15).astype(np.uint8) * 230 + 20
    prims = _scene(9)
    a = _args(W, H)
    gl, gr = lib.render_ir(prims, torch.from_numpy(pat).cuda(), **a)
    ol, orr, _, _ = oracle.render(prims, pat, **a)
    assert np.array_equal(gl.cpu().numpy(), ol) and np.array_equal(gr.cpu().numpy(), orr)
    wl = configs.Workload(name="sim", W=W, H=H, D=D, win_w=7, win_h=7, paths=8, uniq=10, lr_max_diff=1,
                          subpixel=True, f=a["f"], baseline=a["baseline"], seed=5)
    with lib.SimSense.from_workload(wl) as m:
        m.set_noise(True, seed=5)
        d = m.compute(gl, gr).cpu().numpy()
    nl = lib.add_noise(gl, seed=5, frame=0, view=0).cpu().numpy()
    nr = lib.add_noise(gr, seed=5, frame=0, view=1).cpu().numpy()
    o = oracle.compute(nl, nr, D, 7, 7, wl.P1, wl.P2, 8, 10, 1, True, wl.f, wl.baseline)
    valid = o["mask"] == 0
    assert np.array_equal(d > 0, valid)
    np.testing.assert_allclose(d[valid], o["depth"][valid], rtol=1e-5)
    assert valid.mean() > 0.3
