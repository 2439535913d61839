"""Pins of the oracle's optional variants of the depth stage (arxiv
2201.11924 Sec. VI-D names a centre-symmetric census, SGBM's block cost and
a median filter among SimSense's steps).

Each pin comes from outside the oracle: a hand-worked fixture, an invariant
of the definition (180-degree rotation complements a centre-symmetric code),
a library routine the step reduces to (a box convolution, a median filter),
or exact depth recovery on a noise-free plane.
"""
import os

import numpy as np
import pytest
import scipy.ndimage
import scipy.signal

import oracle
from paper_2201_11924_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(name):
    lines = [l.split("#")[0].strip() for l in open(os.path.join(GOLDEN, name))]
    lines = [l for l in lines if l]
    i = lines.index("image")
    j = lines.index("codes")
    img = np.array([[int(v) for v in l.split()] for l in lines[i + 1:j]], dtype=np.uint8)
    codes = [(int(a), int(b), int(c, 2)) for a, b, c in (l.split() for l in lines[j + 1:])]
    return img, codes


def test_csct_hand_worked_codes():
    img, codes = _read_fixture("csct_3x3_hand.txt")
    got = oracle.census_cs(img, 3, 3)
    for x, y, c in codes:
        assert int(got[y, x]) == c, (x, y)


@pytest.mark.parametrize("ww,wh", [(3, 3), (5, 5), (7, 7), (9, 7)])
def test_csct_rotation_complements_interior_codes(ww, wh):
    # with distinct intensities, rotating the image by 180 degrees swaps the
    # two pixels of every centre-symmetric pair, so each interior code turns
    # into its complement (a wrong pair, offset or bit order breaks this)
    rng = np.random.default_rng(ww * 10 + wh)
    H, W = 12, 15                                   # 180 distinct values < 256
    img = rng.permutation(256)[:H * W].reshape(H, W).astype(np.uint8)
    nb = (ww * wh - 1) // 2
    full = (1 << nb) - 1
    a = oracle.census_cs(img, ww, wh)
    b = oracle.census_cs(img[::-1, ::-1].copy(), ww, wh)[::-1, ::-1]
    rx, ry = ww // 2, wh // 2
    inner = (slice(ry, H - ry), slice(rx, W - rx))
    assert np.array_equal(a[inner] ^ b[inner], np.full_like(a[inner], full))


def test_csct_constant_image_and_bit_width():
    img = np.full((9, 11), 77, dtype=np.uint8)
    assert not oracle.census_cs(img, 7, 7).any()
    ramp = np.tile(np.arange(11, dtype=np.uint8), (9, 1))
    assert int(oracle.census_cs(ramp, 7, 7).max()) < (1 << 24)


@pytest.mark.parametrize("bw,bh", [(3, 3), (5, 3), (1, 5)])
def test_block_cost_is_a_rounded_box_mean(bw, bh):
    # the block sum is a box convolution with zero padding, the pixel count
    # the same convolution of ones; the mean is rounded half up
    rng = np.random.default_rng(bw * 7 + bh)
    C = rng.integers(0, 49, size=(10, 13, 6), dtype=np.uint8)
    got = oracle.cost_block(C, bw, bh)
    k = np.ones((bh, bw), dtype=np.int64)
    n = scipy.signal.convolve2d(np.ones(C.shape[:2], dtype=np.int64), k, mode="same")
    for d in range(C.shape[2]):
        s = scipy.signal.convolve2d(C[:, :, d].astype(np.int64), k, mode="same")
        assert np.array_equal(got[:, :, d], (s + n // 2) // n)


def test_block_cost_one_by_one_and_constant():
    rng = np.random.default_rng(5)
    C = rng.integers(0, 49, size=(7, 9, 4), dtype=np.uint8)
    assert np.array_equal(oracle.cost_block(C, 1, 1), C)
    K = np.full((7, 9, 4), 31, dtype=np.uint8)
    assert np.array_equal(oracle.cost_block(K, 5, 5), K)


@pytest.mark.parametrize("k", [3, 5])
def test_median_matches_library_filter(k):
    rng = np.random.default_rng(k)
    m = rng.normal(20.0, 5.0, size=(11, 14))
    m[rng.random(m.shape) < 0.2] = 0.0
    assert np.array_equal(oracle.median(m, k), scipy.ndimage.median_filter(m, size=k, mode="nearest"))


@pytest.mark.parametrize("variant", ["csct", "sgbm", "median"])
@pytest.mark.parametrize("d0", [6, 17])
def test_variants_recover_a_plane_exactly(variant, d0):
    # on a noise-free fronto-parallel plane the matching cost at d0 is 0 for
    # every census code (full or centre-symmetric), so is its block mean, and
    # the median of a constant disparity is that disparity
    W, H, D, ww, wh = 96, 40, 40, 7, 7
    f, b = 300.0, 0.055
    p = scenes.make_plane_pair(W, H, d0, seed=d0 + 3)
    kw = {"csct": dict(census_cs=True), "sgbm": dict(block=(3, 3)), "median": dict(median=3)}[variant]
    o = oracle.compute(p["left"], p["right"], D, ww, wh, 7, 86, 8, 0, -1, False, f, b, **kw)
    xs = np.arange(W)
    m = ww // 2 + (1 if variant == "sgbm" else 0) + (1 if variant == "median" else 0)
    inner = (xs >= d0 + m) & (xs <= W - 1 - m)
    rows = slice(1, H - 1) if variant != "csct" else slice(0, H)
    assert (o["disp"][rows][:, inner] == d0).all()
    fb = float(np.float32(f)) * float(np.float32(b))
    np.testing.assert_allclose(o["depth"][rows][:, inner], fb / d0, rtol=1e-12)


def test_variants_off_equal_the_plain_stage():
    rng = np.random.default_rng(9)
    L = rng.integers(0, 256, (24, 40), dtype=np.uint8)
    R = np.roll(L, -4, axis=1)
    a = oracle.compute(L, R, 16, 5, 5, 7, 60, 4, 10, 1, True, 300.0, 0.055)
    b = oracle.compute(L, R, 16, 5, 5, 7, 60, 4, 10, 1, True, 300.0, 0.055, census_cs=False, block=(1, 1), median=0)
    for k in ("depth", "disp", "dstar", "mask"):
        assert np.array_equal(a[k], b[k])


def _pair(seed, H=20, W=36, shift=3):
    rng = np.random.default_rng(seed)
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = np.roll(L, -shift, axis=1)
    R[:, W - shift:] = rng.integers(0, 256, (H, shift), dtype=np.uint8)
    return L, R


@pytest.mark.parametrize("census_cs,block", [(True, (1, 1)), (False, (1, 5)), (False, (5, 1)),
                                             (False, (3, 3)), (True, (3, 1))])
def test_stage_composes_its_variant_steps(census_cs, block):
    # with P1 = P2 = 0 every path reproduces the cost, so S = paths * C for the
    # variant's own cost volume: the (centre-symmetric) census codes, their
    # Hamming cost with nbits for x - d < 0 (nbits = (w h - 1) / 2 for the
    # centre-symmetric census), then the block mean -- each step pinned on its own
    L, R = _pair(21 + 3 * block[0] + block[1] + census_cs)
    D, ww, wh, paths = 12, 5, 5, 4
    codes = oracle.census_cs if census_cs else oracle.census
    nbits = (ww * wh - 1) // 2 if census_cs else ww * wh - 1
    C = oracle.cost(codes(L, ww, wh), codes(R, ww, wh), D, nbits)
    assert (C[:, 0, 1:] == nbits).all()                     # x = 0, every d >= 1: x - d < 0
    if block != (1, 1):
        C = oracle.cost_block(C, *block)
    o = oracle.compute(L, R, D, ww, wh, 0, 0, paths, 0, -1, False, 300.0, 0.055, want_S=True,
                       census_cs=census_cs, block=block)
    assert np.array_equal(o["S"], paths * C.astype(np.int32))


def test_median_output_is_the_filtered_disparity_and_its_depth():
    # the filter takes the disparity map after the checks (invalid pixels as 0)
    # and the depth follows the filtered disparity: Z = f b / d, 0 where d <= 0
    L, R = _pair(5, H=28, W=48, shift=4)
    args = (L, R, 16, 5, 5, 7, 60, 4, 10, 1, True, 300.0, 0.055)
    pre = oracle.compute(*args)
    post = oracle.compute(*args, median=3)
    d0 = np.where(pre["mask"] == 0, pre["disp"], 0.0)
    want = scipy.ndimage.median_filter(d0, size=3, mode="nearest")
    assert not np.array_equal(want, d0)                       # the filter changes this map
    valid = want > 0
    np.testing.assert_array_equal(post["disp"][valid], want[valid])
    assert (post["disp"][~valid] == -1.0).all()
    fb = float(np.float32(300.0)) * float(np.float32(0.055))
    np.testing.assert_allclose(post["depth"][valid], fb / want[valid], rtol=1e-12)
    assert (post["depth"][~valid] == 0.0).all()
