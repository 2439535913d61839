"""The seeded input generator (scenes.py) against the recipe it states: the
projector's random-dot pattern (dot probability 0.15, dots uniform 180-255,
background uniform 20-60), rectified stereo geometry (a point at depth Z
appears f b / Z pixels further left in the right view), noise-free
fronto-parallel planes reproduced exactly, and seed determinism.  The
generator holds none of the depth stage's arithmetic; these tests pin that the
inputs both the CUDA path and the oracle see are the ones described."""
import numpy as np
import pytest

from paper_2201_11924_gb300 import configs, scenes


def test_pattern_recipe():
    sc = configs.Scene()
    p = scenes.make_pattern(np.random.default_rng(7), 1000, 1000, sc)
    dots = p >= sc.dot_lo
    # 10^6 Bernoulli(0.15) draws: standard deviation 3.6e-4
    assert abs(dots.mean() - sc.dot_density) < 0.002
    assert p[dots].min() == sc.dot_lo and p[dots].max() == sc.dot_hi
    assert p[~dots].min() == sc.bg_lo and p[~dots].max() == sc.bg_hi
    # uniform integers: every value occurs, means at the range centres
    assert np.array_equal(np.unique(p[dots]), np.arange(sc.dot_lo, sc.dot_hi + 1))
    assert np.array_equal(np.unique(p[~dots]), np.arange(sc.bg_lo, sc.bg_hi + 1))
    assert abs(p[dots].mean() - (sc.dot_lo + sc.dot_hi) / 2) < 0.5
    assert abs(p[~dots].mean() - (sc.bg_lo + sc.bg_hi) / 2) < 0.1


@pytest.mark.parametrize("d0", [0, 5, 31])
def test_noise_free_plane_is_an_exact_shift(d0):
    p = scenes.make_plane_pair(96, 40, d0, seed=3)
    l, r = p["left"].astype(int), p["right"].astype(int)
    assert np.array_equal(r[:, :96 - d0], l[:, d0:])
    assert ((r[:, 96 - d0:] >= 20) & (r[:, 96 - d0:] <= 60)).all()      # unseen strip: background only


def test_pairs_are_seeded_and_shaped():
    wl = configs.SMALL_320
    a, b, c = scenes.make_pair(wl), scenes.make_pair(wl), scenes.make_pair(wl, seed=wl.seed + 1)
    for k in ("left", "right", "depth_gt", "disp_gt"):
        assert np.array_equal(a[k], b[k])
    assert not np.array_equal(a["left"], c["left"])
    assert a["left"].dtype == np.uint8 and a["left"].shape == (wl.H, wl.W)
    assert a["right"].dtype == np.uint8 and a["right"].shape == (wl.H, wl.W)


@pytest.mark.parametrize("wl", [configs.SMALL_320, configs.HD_720], ids=lambda w: w.name)
def test_ground_truth_follows_the_rectified_geometry(wl):
    p = scenes.make_pair(wl)
    z, d = p["depth_gt"], p["disp_gt"]
    np.testing.assert_allclose(d, wl.f * wl.baseline / z, rtol=1e-12)
    sc = wl.scene
    assert z.min() >= sc.z_min * (1 - 1e-9) and np.isfinite(z).all()
    # the views differ by the disparity, not by a constant: most pixels whose
    # right-view partner lies inside the image agree within the sensor noise
    H, W = z.shape
    ys, xs = np.mgrid[0:H, 0:W]
    xr = np.rint(xs - d).astype(int)
    inside = (xr >= 0) & (np.abs(xs - d - xr) < 0.05)
    diff = np.abs(p["left"][inside].astype(int) - p["right"][ys[inside], xr[inside]].astype(int))
    assert np.median(diff) <= 3 * sc.noise_sigma


def test_workloads_match_their_stated_sizes_and_seeds():
    s, h, f = configs.SMALL_320, configs.HD_720, configs.FHD_1080
    assert (s.W, s.H, s.D, s.win_w, s.win_h, s.paths, s.seed) == (320, 240, 64, 5, 5, 4, 1001)
    assert (h.W, h.H, h.D, h.win_w, h.win_h, h.paths, h.seed) == (1280, 720, 128, 7, 7, 8, 1002)
    assert (f.W, f.H, f.D, f.win_w, f.win_h, f.paths, f.seed) == (1920, 1080, 256, 9, 7, 8, 1004)
    # every path cost fits a byte (nbits + P2 <= 255) and P1 <= P2
    for w in (s, h, f):
        assert w.win_w * w.win_h - 1 + w.P2 <= 255 and w.P1 <= w.P2
