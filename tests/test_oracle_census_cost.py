"""Pins for the oracle's census transform and Hamming cost (arxiv 2201.11924 Sec. VI-D).

None of these expected values comes from the oracle: they are hand-worked
codes (tests/golden), invariants of the census definition, numpy's own bit
count, and the exact zero cost of a pure horizontal shift.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_census_golden(name):
    img, codes, mode = [], [], None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line in ("image", "codes"):
                mode = line
                continue
            if mode == "image":
                img.append([int(v) for v in line.split()])
            else:
                x, y, bits = line.split()
                codes.append((int(x), int(y), int(bits, 2)))
    return np.array(img, dtype=np.uint8), codes


def test_census_hand_worked_5x5():
    img, codes = _read_census_golden("census_5x5_hand.txt")
    got = oracle.census(img, 5, 5)
    for x, y, want in codes:
        assert int(got[y, x]) == want, (x, y, bin(int(got[y, x])), bin(want))


def test_census_3x3_msb_order():
    # centre 5; only the first raster neighbour (top-left) is smaller -> MSB of 8 bits
    img = np.array([[1, 9, 9], [9, 5, 9], [9, 9, 9]], dtype=np.uint8)
    assert int(oracle.census(img, 3, 3)[1, 1]) == 0b10000000
    # only the last raster neighbour (bottom-right) is smaller -> LSB
    img = np.array([[9, 9, 9], [9, 5, 9], [9, 9, 1]], dtype=np.uint8)
    assert int(oracle.census(img, 3, 3)[1, 1]) == 0b00000001


@pytest.mark.parametrize("ww,wh", [(5, 5), (7, 7), (9, 7)])
def test_census_constant_image_is_zero(ww, wh):
    img = np.full((13, 17), 77, dtype=np.uint8)
    assert not oracle.census(img, ww, wh).any()


@pytest.mark.parametrize("ww,wh", [(5, 5), (7, 7), (9, 7)])
def test_census_invariant_under_increasing_map(ww, wh):
    rng = np.random.default_rng(7)
    img = rng.integers(0, 128, size=(21, 33)).astype(np.uint8)
    # any strictly increasing intensity map leaves every comparison unchanged
    lut = np.cumsum(rng.integers(1, 3, size=256))
    lut = (lut - lut[0]).astype(np.int64)
    mapped = lut[img]
    assert mapped.max() <= 255
    a = oracle.census(img, ww, wh)
    b = oracle.census(mapped.astype(np.uint8), ww, wh)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("ww,wh", [(5, 5), (7, 7), (9, 7)])
def test_census_code_width(ww, wh):
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, size=(19, 23)).astype(np.uint8)
    codes = oracle.census(img, ww, wh)
    nbits = ww * wh - 1
    assert int(codes.max()) < (1 << nbits)
    assert int(np.bitwise_count(codes).max()) <= nbits
    # an interior pixel that is a strict maximum of its window has every bit set
    img2 = img.copy()
    img2[9, 11] = 255
    img2[9 - wh // 2: 9 + wh // 2 + 1, 11 - ww // 2: 11 + ww // 2 + 1] = np.minimum(
        img2[9 - wh // 2: 9 + wh // 2 + 1, 11 - ww // 2: 11 + ww // 2 + 1], 254)
    img2[9, 11] = 255
    assert int(oracle.census(img2, ww, wh)[9, 11]) == (1 << nbits) - 1


def test_census_border_neighbours_are_zero_bits():
    # a corner pixel that is larger than everything: only in-image offsets set bits
    img = np.zeros((5, 5), dtype=np.uint8)
    img[0, 0] = 200
    code = int(oracle.census(img, 3, 3)[0, 0])
    # in-image neighbours of (0,0) in a 3x3 window: (1,0), (0,1), (1,1)
    # raster positions 4, 6, 7 of 8 -> bits 3, 1, 0
    assert code == (1 << 3) | (1 << 1) | (1 << 0)


def test_cost_matches_numpy_bitcount():
    rng = np.random.default_rng(3)
    H, W, D, nbits = 6, 29, 9, 48
    cl = rng.integers(0, 1 << nbits, size=(H, W), dtype=np.uint64)
    cr = rng.integers(0, 1 << nbits, size=(H, W), dtype=np.uint64)
    C = oracle.cost(cl, cr, D, nbits)
    for d in range(D):
        for x in range(W):
            if x - d >= 0:
                want = np.bitwise_count(cl[:, x] ^ cr[:, x - d])
            else:
                want = np.full(H, nbits)
            np.testing.assert_array_equal(C[:, x, d], want)


def test_cost_symmetry_identity_triangle():
    rng = np.random.default_rng(5)
    H, W, nbits = 5, 40, 62
    a, b, c = (rng.integers(0, 1 << nbits, size=(H, W), dtype=np.uint64) for _ in range(3))
    ab = oracle.cost(a, b, 1, nbits)[..., 0].astype(int)
    ba = oracle.cost(b, a, 1, nbits)[..., 0].astype(int)
    ac = oracle.cost(a, c, 1, nbits)[..., 0].astype(int)
    cb = oracle.cost(c, b, 1, nbits)[..., 0].astype(int)
    np.testing.assert_array_equal(ab, ba)
    assert (ab <= ac + cb).all()
    assert not oracle.cost(a, a, 1, nbits)[..., 0].any()


@pytest.mark.parametrize("ww,wh,d0", [(5, 5, 3), (7, 7, 6), (9, 7, 11)])
def test_cost_zero_at_true_shift(ww, wh, d0):
    rng = np.random.default_rng(d0)
    H, W, D = 15, 48, 16
    left = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    right = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    right[:, : W - d0] = left[:, d0:]           # right(x) = left(x + d0)
    nbits = ww * wh - 1
    C = oracle.cost(oracle.census(left, ww, wh), oracle.census(right, ww, wh), D, nbits)
    xs = np.arange(W)
    # both windows hold the same pixels wherever both stay inside the image
    inside = (xs >= d0 + ww // 2) & (xs <= W - 1 - ww // 2)
    assert not C[:, inside, d0].any()
    # cells whose right pixel x-d falls off the image carry the worst cost
    assert (C[:, :d0, d0] == nbits).all()
