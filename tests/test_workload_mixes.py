"""The batched and serving workloads against their stated recipes (no GPU):
64 pairs with sizes drawn uniformly from four classes, seeds 3000 + i; 1024
cameras with sizes in 50/40/10 proportion, seeds 5000 + cam; Poisson request
arrivals at the stated rate.  The mean cells per request and the offered cell
rate follow from them."""
import numpy as np
from scipy import stats

from paper_2201_11924_gb300 import configs, serve


def test_batch_mix_is_seeded_and_uniform_over_its_classes():
    ws = configs.batch_workloads()
    assert len(ws) == 64 and [w.seed for w in ws] == list(range(3000, 3064))
    assert ws == configs.batch_workloads()                         # deterministic
    counts = np.array([sum((w.W, w.H, w.D) == s for w in ws) for s in configs.BATCH_SIZES])
    assert counts.sum() == 64 and (counts > 0).all()
    assert stats.chisquare(counts).pvalue > 0.001                  # uniform over the four classes
    for w in ws:
        assert (w.win_w, w.win_h, w.paths, w.uniq, w.lr_max_diff, w.subpixel) == (7, 7, 8, 0, 1, False)


def test_serving_cameras_follow_the_50_40_10_split():
    cams = [configs.serve_camera(c) for c in range(1024)]
    assert [c.seed for c in cams] == list(range(5000, 6024))
    sizes = [s for s, _ in configs.SERVE_SIZES]
    counts = np.array([sum((c.W, c.H, c.D) == s for c in cams) for s in sizes])
    assert counts.sum() == 1024
    expect = 1024 * np.array([p for _, p in configs.SERVE_SIZES])
    assert stats.chisquare(counts, expect).pvalue > 0.001
    for c in cams:
        assert (c.win_w, c.win_h, c.paths, c.uniq, c.lr_max_diff, c.subpixel) == (7, 7, 8, 15, 1, True)


def test_request_arrivals_are_poisson():
    rate, dur = 4000.0, 10.0
    tr = serve.poisson_trace(1024, rate, dur, seed=5999)
    n = len(tr)
    assert abs(n - rate * dur) < 5 * np.sqrt(rate * dur)          # Poisson count
    t = np.array([r.arrival for r in tr])
    assert (np.diff(t) >= 0).all() and t.min() >= 0 and t.max() <= dur
    assert stats.kstest(t / dur, "uniform").pvalue > 0.001        # uniform times given the count
    gaps = np.diff(t)
    assert stats.kstest(gaps * rate, "expon").pvalue > 0.001       # exponential gaps
    cams = np.array([r.camera for r in tr])
    assert cams.min() >= 0 and cams.max() < 1024
    assert stats.chisquare(np.bincount(cams, minlength=1024)).pvalue > 0.001


def test_offered_load_of_the_serving_mix():
    # mean cells per request from the split: 0.5 * 848*480*96 (19,537,920)
    # + 0.4 * 1280*720*128 (47,185,920) + 0.1 * 1920*1080*256 (53,084,160)
    # = 119,808,000; at 4000 requests/s, 4.79e11 cells/s
    mean = sum(p * W * H * D for (W, H, D), p in configs.SERVE_SIZES)
    assert abs(mean - 119_808_000) < 1e-3
    assert abs(4000 * mean - 4.79232e11) < 1.0
