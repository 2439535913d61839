"""End-to-end pins of the oracle's depth stage (arxiv 2201.11924 Sec. VI-D).

A noise-free fronto-parallel plane at integer disparity d0 makes the census
windows of matching pixels identical, so the matching cost at d0 is exactly 0
there; the stage must then return d0 and the closed-form depth f*b/d0 on
every such pixel.  The multi-plane scene does the same band by band away
from the depth edges.
"""
import numpy as np
import pytest

import oracle
from paper_2201_11924_gb300 import configs, scenes


@pytest.mark.parametrize("ww,wh", [(5, 5), (7, 7), (9, 7)])
@pytest.mark.parametrize("paths", [4, 8])
@pytest.mark.parametrize("d0", [5, 13, 30])
def test_plane_exact_recovery(ww, wh, paths, d0):
    W, H, D = 96, 40, 48
    f, b = 300.0, 0.055
    p = scenes.make_plane_pair(W, H, d0, seed=d0 + ww)
    o = oracle.compute(p["left"], p["right"], D, ww, wh, 7, 86, paths, 0, -1, False, f, b)
    xs = np.arange(W)
    inner = (xs >= d0 + ww // 2) & (xs <= W - 1 - ww // 2)
    assert (o["dstar"][:, inner] == d0).all()
    assert (o["mask"][:, inner] == 0).all()
    fb = float(np.float32(f)) * float(np.float32(b))
    np.testing.assert_allclose(o["depth"][:, inner], fb / d0, rtol=1e-12)


@pytest.mark.parametrize("paths", [4, 8])
def test_multiplane_exact_away_from_edges(paths):
    W, H, D = 120, 32, 40
    disps = [8, 20, 12, 30]
    ww = wh = 7
    p = scenes.make_multiplane_pair(W, H, disps, seed=17)
    o = oracle.compute(p["left"], p["right"], D, ww, wh, 7, 86, paths, 0, -1, False, 300.0, 0.055)
    gt = p["disp_gt"][0]
    xs = np.arange(W)
    margin = ww // 2 + 2
    ok = np.ones(W, dtype=bool)
    # stay a census radius (+2) away from every depth edge; where the disparity
    # steps up (a nearer band to the right), the jump's width of left pixels
    # just left of the edge is occluded in the right view and is excluded too
    for e in np.flatnonzero(np.diff(gt) != 0):
        jump = int(gt[e + 1] - gt[e])
        lo = e - margin + 1 - max(jump, 0)
        ok[max(0, lo): e + margin + 1] = False
    ok &= (xs >= gt + margin) & (xs <= W - 1 - margin)
    assert ok.sum() > 10
    assert (o["dstar"][:, ok] == gt[None, ok]).all()


def test_small_workload_matches_ground_truth_mostly():
    # a statistical sanity check on the synthetic scene, not a parity pin:
    # valid pixels land within one pixel of the rendered disparity
    wl = configs.SMALL_320
    p = scenes.make_pair(wl)
    o = oracle.compute(p["left"], p["right"], wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths,
                       wl.uniq, wl.lr_max_diff, wl.subpixel, wl.f, wl.baseline)
    valid = o["mask"] == 0
    assert valid.mean() > 0.8
    err = np.abs(o["dstar"] - p["disp_gt"])
    assert (err[valid] <= 1.0).mean() > 0.95
