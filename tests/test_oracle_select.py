"""Pins for the oracle's selection steps (arxiv 2201.11924 Sec. VI-D: best
disparity, uniqueness test, quadratic sub-pixel fit, left-right consistency
check, disparity to depth).  Every expected value is worked out by hand in the
comments or is a closed form.
"""
import numpy as np
import pytest

import oracle


def _vol(rows):
    """H=1 volume from a list of per-pixel cost lists."""
    return np.array([rows], dtype=np.int32)


def test_wta_smallest_index_on_ties_and_constant():
    S = _vol([[5, 3, 3, 7, 9], [4, 4, 4, 4, 4], [9, 8, 7, 6, 6]])
    dstar, _, _, _ = oracle.select(S, 0, -1, False, 1.0)
    assert dstar.tolist() == [[1, 0, 3]]


def test_uniqueness_ratio_threshold():
    # d* = 1 (cost 50); d = 0 and 2 are neighbours and never count.
    # u = 15: a far candidate fails the pixel iff 85 * S(d) < 100 * 50 = 5000.
    #   S(4) = 58 -> 85*58 = 4930 < 5000 -> fail;  S(4) = 59 -> 5015 -> pass
    S = _vol([[100, 50, 50, 200, 58], [100, 50, 50, 200, 59], [51, 50, 51, 200, 58]])
    _, mask, _, _ = oracle.select(S, 15, -1, False, 1.0)
    assert (mask[0] & 1).tolist() == [1, 0, 1]
    # u = 0 disables the test
    _, mask, _, _ = oracle.select(S, 0, -1, False, 1.0)
    assert (mask[0] & 1).tolist() == [0, 0, 0]
    # the boundary: (100 - u) S(d) = 100 S(d*) is unique (the test is >=)
    #   d* = 1 (S = 17), far S(4) = 20: 85 * 20 = 1700 = 100 * 17 -> pass;
    #   S(4) = 19: 1615 < 1700 -> fail
    S = _vol([[200, 17, 30, 200, 20], [200, 17, 30, 200, 19]])
    _, mask, _, _ = oracle.select(S, 15, -1, False, 1.0)
    assert (mask[0] & 1).tolist() == [0, 1]
    # u = 1, the smallest ratio that tests: a far candidate equal to S(d*)
    # fails (99 * 100 < 100 * 100), one 2% above passes (99 * 102 >= 10000)
    S = _vol([[300, 100, 300, 300, 100], [300, 100, 300, 300, 102]])
    _, mask, _, _ = oracle.select(S, 1, -1, False, 1.0)
    assert (mask[0] & 1).tolist() == [1, 0]


def test_left_right_check_hand_worked():
    # W = 4, D = 2.  Per pixel S = [S(d=0), S(d=1)]:
    #   x=0 [1, 9] -> d*=0;  x=1 [5, 2] -> d*=1;  x=2 [3, 8] -> d*=0;  x=3 [6, 1] -> d*=1
    # right-view winners D_R(xr) = argmin_d S(xr + d, d) over d <= min(D-1, W-1-xr):
    #   D_R(0): S(0,0)=1, S(1,1)=2 -> 0
    #   D_R(2): S(2,0)=3, S(3,1)=1 -> 1
    # x=0: xr=0, |0-0|=0;  x=1: xr=0, |1-0|=1;  x=2: xr=2, |0-1|=1;  x=3: xr=2, |1-1|=0
    S = _vol([[1, 9], [5, 2], [3, 8], [6, 1]])
    _, m1, _, _ = oracle.select(S, 0, 1, False, 1.0)
    _, m0, _, _ = oracle.select(S, 0, 0, False, 1.0)
    assert (m1[0] & 2).tolist() == [0, 0, 0, 0]
    assert (m0[0] & 2).tolist() == [0, 2, 2, 0]
    # d* = 0 means zero disparity, i.e. no finite depth: bit 4
    assert (m0[0] & 4).tolist() == [4, 0, 4, 0]
    # a winner that points outside the right image fails the check: x=0, d*=1
    S2 = _vol([[9, 1], [5, 2], [3, 8], [6, 1]])
    _, m, _, _ = oracle.select(S2, 0, 5, False, 1.0)
    assert int(m[0, 0]) & 2 == 2


def test_right_view_ties_take_the_smallest_disparity():
    # W = 3, D = 2.  x=0 [4, 9] -> d*=0;  x=1 [9, 4] -> d*=1;  x=2 [5, 6] -> d*=0
    # D_R(0): S(0, d=0) = 4 and S(1, d=1) = 4 tie -> the smaller d, 0
    # with lr = 0: x=0 (xr=0) |0 - 0| = 0 passes, x=1 (xr=0) |1 - 0| = 1 fails
    S = _vol([[4, 9], [9, 4], [5, 6]])
    dstar, m, _, _ = oracle.select(S, 0, 0, False, 1.0)
    assert dstar[0].tolist() == [0, 1, 0]
    assert (m[0, :2] & 2).tolist() == [0, 2]


def test_right_view_search_range_is_clipped_at_the_border():
    # W = 3, D = 3.  D_R(2) may only look at d = 0 (x = 2 + d must stay < 3),
    # so D_R(2) = 0 whatever S holds at other pixels.
    # Pixel x=2 has d* = 0 -> xr = 2 -> |0 - 0| = 0: passes with lr = 0.
    S = _vol([[40, 1, 1], [40, 40, 1], [0, 60, 60]])
    dstar, m, _, _ = oracle.select(S, 0, 0, False, 1.0)
    assert int(dstar[0, 2]) == 0 and int(m[0, 2]) & 2 == 0


@pytest.mark.parametrize("k", [3, 5, 10])
@pytest.mark.parametrize("frac", [0.0, 0.25, -0.25, 0.5, -0.5, 0.125])
def test_subpixel_recovers_parabola_vertex(k, frac):
    # S(d) = a (d - v)^2 + c with a = 64 keeps every sample an integer; the
    # three-point quadratic fit is exact for a parabola.
    D = 16
    v = k + frac
    a, c = 64, 10
    s = [a * (d - v) ** 2 + c for d in range(D)]
    assert all(float(x).is_integer() for x in s)
    S = _vol([[int(x) for x in s]])
    fb = 50.6
    dstar, mask, disp, depth = oracle.select(S, 0, -1, True, fb)
    assert int(mask[0, 0]) == 0
    assert abs(disp[0, 0] - v) < 1e-12
    assert abs(depth[0, 0] - fb / v) < 1e-12 * fb / v


@pytest.mark.parametrize("k,frac", [(1, 0.25), (1, -0.25), (1, 0.5), (1, 0.125), (14, 0.25), (14, -0.5),
                                    (14, 0.5)])
def test_subpixel_at_the_refinable_range_ends(k, frac):
    # d* = 1 and d* = D - 2 are the first and last refined disparities
    D, a, c = 16, 64, 10
    v = k + frac
    S = _vol([[int(a * (d - v) ** 2 + c) for d in range(D)]])
    _, mask, disp, _ = oracle.select(S, 0, -1, True, 50.6)
    assert int(mask[0, 0]) == 0 and abs(disp[0, 0] - v) < 1e-12


def test_subpixel_off_and_at_range_ends():
    # d* at 0 or D-1 is never refined; with sub-pixel off d_f = d*
    S = _vol([[10, 20, 30, 40], [40, 30, 20, 10], [30, 12, 10, 20]])
    _, _, disp, _ = oracle.select(S, 0, -1, True, 1.0)
    assert disp[0, 1] == 3.0
    # x=2: d*=2, S- = 12, S0 = 10, S+ = 20 -> (12-20) / (2 (12+20-20)) = -8/24
    assert abs(disp[0, 2] - (2.0 - 1.0 / 3.0)) < 1e-12
    _, _, disp_off, _ = oracle.select(S, 0, -1, False, 1.0)
    assert disp_off[0, 2] == 2.0
    assert disp[0, 0] == -1.0   # d* = 0 -> invalid, reported as -1


def test_depth_closed_form():
    S = _vol([[9, 9, 1, 9, 9, 9], [9, 9, 9, 9, 9, 1]])
    f, b = 920.0, 0.055
    _, mask, _, depth = oracle.select(S, 0, -1, False, f * b)
    assert mask.tolist() == [[0, 0]]
    assert abs(depth[0, 0] - f * b / 2) < 1e-12
    assert abs(depth[0, 1] - f * b / 5) < 1e-12
