"""Rectification and depth registration on the GPU (arxiv 2201.11924 Sec.
VI-D) against the CPU oracle, through the C ABI.

Both sides evaluate the camera model in fp64 with + - * / only and no fused
multiply-adds, then quantise to 1/256 px and interpolate in integers, so the
rectified images and the registered depth maps are compared bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2201_11924_gb300 import configs, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2201_11924_gb300 import _build, simsense
    _build.build()
    return simsense


def _rot(ax, ay, az):
    cx, sx, cy, sy, cz, sz = np.cos(ax), np.sin(ax), np.cos(ay), np.sin(ay), np.cos(az), np.sin(az)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _cam(W, H, seed):
    rng = np.random.default_rng(seed)
    f = 0.9 * W
    return oracle.camera(f * (1 + 0.01 * rng.standard_normal()), f, (W - 1) / 2 + rng.uniform(-5, 5),
                         (H - 1) / 2 + rng.uniform(-5, 5), k1=rng.uniform(-0.2, 0.2), k2=rng.uniform(-0.05, 0.05),
                         p1=rng.uniform(-2e-3, 2e-3), p2=rng.uniform(-2e-3, 2e-3), k3=rng.uniform(-0.01, 0.01),
                         R=_rot(*rng.uniform(-0.02, 0.02, 3)), rfx=f, rfy=f, rcx=(W - 1) / 2, rcy=(H - 1) / 2)


@pytest.mark.parametrize("W,H,seed", [(160, 90, 1), (97, 45, 2), (960, 540, 3)])
def test_rectify_matches_oracle_bit_for_bit(lib, W, H, seed):
    import torch
    img = np.random.default_rng(seed).integers(0, 256, (H, W), dtype=np.uint8)
    cam = _cam(W, H, seed)
    got = lib.rectify(torch.from_numpy(img).cuda(), cam).cpu().numpy()
    assert np.array_equal(got, oracle.rectify(img, cam))


def test_registration_matches_oracle_bit_for_bit(lib):
    import torch
    rng = np.random.default_rng(5)
    W, H = 200, 120
    depth = rng.uniform(0.3, 3.0, (H, W)).astype(np.float32)
    depth[rng.random(depth.shape) < 0.15] = 0.0
    R, t = _rot(0.01, -0.02, 0.005), [0.015, -0.002, 0.001]
    args = (180.0, 181.0, 99.5, 59.5, 360.0, 362.0, 199.5, 119.5, R, t, 400, 240)   # 2x the resolution
    got = lib.register_depth(torch.from_numpy(depth).cuda(), lib.registration_t(*args)).cpu().numpy()
    want = oracle.register(depth, *args)
    assert np.array_equal(got, want)
    assert (got > 0).sum() > 0.5 * (depth > 0).sum()


def test_stage_with_rectification_equals_oracle_on_rectified_pair(lib):
    import torch
    wl = configs.SMALL_320
    p = scenes.make_pair(wl)
    cl, cr = _cam(wl.W, wl.H, 11), _cam(wl.W, wl.H, 12)
    with lib.SimSense.from_workload(wl) as m:
        m.set_rectify(cl, cr)
        d = m.compute(torch.from_numpy(p["left"]).cuda(), torch.from_numpy(p["right"]).cuda()).cpu().numpy()
        rl, rr = oracle.rectify(p["left"], cl), oracle.rectify(p["right"], cr)
        o = oracle.compute(rl, rr, wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq, wl.lr_max_diff,
                           wl.subpixel, wl.f, wl.baseline)
        valid = o["mask"] == 0
        assert np.array_equal(d > 0, valid)
        np.testing.assert_allclose(d[valid], o["depth"][valid], rtol=1e-5, atol=0)
        m.set_rectify()                                  # off again: the plain stage
        d2 = m.compute(torch.from_numpy(p["left"]).cuda(), torch.from_numpy(p["right"]).cuda()).cpu().numpy()
        o2 = oracle.compute(p["left"], p["right"], wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq,
                            wl.lr_max_diff, wl.subpixel, wl.f, wl.baseline)
        assert np.array_equal(d2 > 0, o2["mask"] == 0)


def test_table2_pipeline_960x540_to_1920x1080(lib):
    # the paper's Table 2 workload shape: a 960 x 540 pair rectified, SGM with
    # 4 paths at D = 128, the depth registered to a 1920 x 1080 RGB camera
    import dataclasses
    import torch
    wl = dataclasses.replace(configs.HD_720, name="table2_960x540", W=960, H=540, D=128, paths=4, census_cs=True,
                             median=3)
    p = scenes.make_pair(wl)
    cl, cr = _cam(wl.W, wl.H, 21), _cam(wl.W, wl.H, 22)
    reg_args = (cl[18], cl[19], cl[20], cl[21], 2 * cl[18], 2 * cl[19], 2 * cl[20] + 0.5, 2 * cl[21] + 0.5,
                _rot(0.002, 0.001, 0.0), [0.015, 0.0, 0.0], 1920, 1080)
    with lib.SimSense.from_workload(wl) as m:
        m.set_rectify(cl, cr)
        d = m.compute(torch.from_numpy(p["left"]).cuda(), torch.from_numpy(p["right"]).cuda())
        reg = lib.register_depth(d, lib.registration_t(*reg_args)).cpu().numpy()
        d = d.cpu().numpy()
    rl, rr = oracle.rectify(p["left"], cl), oracle.rectify(p["right"], cr)
    o = oracle.compute(rl, rr, wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq, wl.lr_max_diff,
                       wl.subpixel, wl.f, wl.baseline, census_cs=True, median=3)
    valid = o["depth"] > 0
    assert np.array_equal(d > 0, valid)
    np.testing.assert_allclose(d[valid], o["depth"][valid], rtol=1e-5, atol=0)
    # registration of the GPU's own depth map: bit for bit
    assert np.array_equal(reg, oracle.register(d, *reg_args))
