"""Parity of the CUDA stage's variants (centre-symmetric census, SGBM block
cost, median filter; arxiv 2201.11924 Sec. VI-D) with the CPU oracle,
through the C ABI.

Bar: census codes, aggregated costs S, integer disparities and masks
bit-exact; fp32 disparity within 1e-4 px and depth within 1e-5 relative of
the oracle's fp64 values.  With the median filter the compared outputs are
the filtered disparity and depth (the median of fp32 and fp64 copies of the
same disparities picks the same pixel's value).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2201_11924_gb300 import configs, scenes

pytestmark = pytest.mark.gpu

DISP_TOL = 1e-4
DEPTH_RTOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    from paper_2201_11924_gb300 import _build, simsense
    _build.build()
    return simsense


def _wl(name, W, H, D, ww, wh, paths, uniq, lr, sub, seed, **variant):
    wl = configs.Workload(name=name, W=W, H=H, D=D, win_w=ww, win_h=wh, P1=7, P2=86, paths=paths, uniq=uniq,
                          lr_max_diff=lr, subpixel=sub, f=300.0, baseline=0.055, seed=seed,
                          scene=configs.SMALL_320.scene)
    return dataclasses.replace(wl, **variant)


CASES = [
    _wl("csct_7x7_8p", 150, 70, 96, 7, 7, 8, 15, 1, True, 21, census_cs=True),
    _wl("csct_9x7_4p_D160", 300, 33, 160, 9, 7, 4, 10, 1, True, 22, census_cs=True),
    _wl("csct_5x5_D48", 97, 45, 48, 5, 5, 8, 0, 1, False, 23, census_cs=True),
    _wl("csct_3x3_runtime_window", 80, 40, 64, 3, 3, 4, 0, 1, True, 24, census_cs=True),
    _wl("sgbm_3x3", 130, 50, 64, 7, 7, 8, 5, 1, True, 25, block=(3, 3)),
    _wl("sgbm_5x3_D192", 260, 40, 192, 9, 7, 8, 10, 0, True, 26, block=(5, 3)),
    _wl("sgbm_7x7_ragged", 97, 45, 48, 5, 5, 4, 0, 1, False, 27, block=(7, 7)),
    _wl("median_3", 150, 70, 96, 7, 7, 8, 15, 1, True, 28, median=3),
    _wl("median_5_D256", 260, 40, 256, 9, 7, 8, 10, 1, True, 29, median=5),
    _wl("all_three", 200, 60, 128, 7, 7, 4, 15, 1, True, 30, census_cs=True, block=(3, 3), median=3),
]


def _run(lib, wl, left, right):
    import torch
    dev = torch.device("cuda:0")
    with lib.SimSense.from_workload(wl) as m:
        lt = torch.from_numpy(left).to(dev)
        rt = torch.from_numpy(right).to(dev)
        out = m.compute_debug(lt, rt, aggregated=True)
        plain = m.compute(lt, rt)
        torch.cuda.synchronize()
        assert m.device_status() == 0
        res = {k: v.cpu().numpy() for k, v in out.items()}
        res["depth_plain"] = plain.cpu().numpy()
    return res


def _oracle(wl, left, right):
    return oracle.compute(left, right, wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq, wl.lr_max_diff,
                          wl.subpixel, wl.f, wl.baseline, want_codes=True, want_S=True, census_cs=wl.census_cs,
                          block=wl.block, median=wl.median)


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_variant_matches_oracle(lib, wl):
    p = scenes.make_pair(wl)
    g = _run(lib, wl, p["left"], p["right"])
    o = _oracle(wl, p["left"], p["right"])
    np.testing.assert_array_equal(g["census_left"].view(np.uint64), o["codes_left"])
    np.testing.assert_array_equal(g["census_right"].view(np.uint64), o["codes_right"])
    np.testing.assert_array_equal(g["aggregated"].view(np.uint16).astype(np.int32), o["S"])
    np.testing.assert_array_equal(g["disparity_int"].astype(np.int32), o["dstar"])
    np.testing.assert_array_equal(g["mask"], o["mask"])
    valid = o["depth"] > 0
    assert np.array_equal(g["depth"] > 0, valid)
    assert (g["disparity"][~valid] == -1.0).all()
    np.testing.assert_allclose(g["disparity"][valid], o["disp"][valid], rtol=0, atol=DISP_TOL)
    np.testing.assert_allclose(g["depth"][valid], o["depth"][valid], rtol=DEPTH_RTOL, atol=0)
    np.testing.assert_array_equal(g["depth_plain"], g["depth"])


def test_variant_plane_recovery(lib):
    # noise-free plane at d0: every variant returns d0 away from the borders
    W, H, D, d0 = 160, 48, 64, 21
    p = scenes.make_plane_pair(W, H, d0, seed=3)
    wl = _wl("plane", W, H, D, 7, 7, 8, 0, 1, False, 0, census_cs=True, block=(3, 3), median=3)
    g = _run(lib, wl, p["left"], p["right"])
    # (left of x = d0 + 10 the right-view argmin of the left-right check can
    # also pick pixels with no true match, as the oracle does too)
    inner = np.zeros((H, W), dtype=bool)
    inner[2:H - 2, d0 + 10:W - 6] = True
    assert (g["disparity"][inner] == d0).all()


def test_variant_option_ranges(lib):
    import torch
    m = lib.SimSense(64, 32, 16, 7, 7, 7, 86, 4, 0, 1, 300.0, 0.055)
    try:
        for opt, bad in [(lib.OPT_CENSUS_CS, 2), (lib.OPT_BLOCK, 2 | (3 << 8)), (lib.OPT_BLOCK, 9 | (1 << 8)),
                         (lib.OPT_BLOCK, 3 | (3 << 8) | (1 << 16)), (lib.OPT_MEDIAN, 4), (lib.OPT_MEDIAN, 7)]:
            with pytest.raises(Exception):
                m.set_option(opt, bad)
        # a rejected value changes nothing: the stage still equals the plain oracle
        wl = _wl("after_bad", 64, 32, 16, 7, 7, 4, 0, 1, True, 31)
        p = scenes.make_pair(wl)
        d = m.compute(torch.from_numpy(p["left"]).cuda(), torch.from_numpy(p["right"]).cuda())
        o = oracle.compute(p["left"], p["right"], 16, 7, 7, 7, 86, 4, 0, 1, True, 300.0, 0.055)
        valid = o["mask"] == 0
        got = d.cpu().numpy()
        assert np.array_equal(got > 0, valid)
        np.testing.assert_allclose(got[valid], o["depth"][valid], rtol=DEPTH_RTOL)
    finally:
        m.close()


def test_full_size_variant_matches_oracle(lib):
    # 1280 x 720, D = 128, the paper's census type with SGBM 3x3 and a 3x3
    # median: sampled rows of S, all of disparity and depth
    wl = dataclasses.replace(configs.HD_720, census_cs=True, block=(3, 3), median=3)
    p = scenes.make_pair(wl)
    g = _run(lib, wl, p["left"], p["right"])
    o = oracle.compute(p["left"], p["right"], wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq,
                       wl.lr_max_diff, wl.subpixel, wl.f, wl.baseline, census_cs=True, block=(3, 3), median=3)
    np.testing.assert_array_equal(g["disparity_int"].astype(np.int32), o["dstar"])
    valid = o["depth"] > 0
    assert np.array_equal(g["depth"] > 0, valid)
    np.testing.assert_allclose(g["depth"][valid], o["depth"][valid], rtol=DEPTH_RTOL, atol=0)
