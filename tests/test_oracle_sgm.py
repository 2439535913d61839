"""Pins for the oracle's SGM path aggregation (arxiv 2201.11924 Sec. VI-D, the
semi-global matching of Hirschmueller that the paper cites).

The main pin is independent of the recurrence: along any scanline, SGM's
L_r(p, d) plus the sum of the minima m' subtracted at the earlier pixels of
the path equals the minimum, over ALL label sequences of the path that end in
d, of the sum of the costs plus a penalty of 0 / P1 / P2 for a label change of
0 / 1 / more than 1.  The tests enumerate every label sequence by brute force.
"""
import itertools

import numpy as np
import pytest

import oracle

DIRS = oracle.PATH_DIRS


def _min_energy_ending(costs, P1, P2):
    """costs: n x D list; returns E[d] = min over sequences ending in d."""
    n, D = len(costs), len(costs[0])
    best = [None] * D
    for seq in itertools.product(range(D), repeat=n):
        e = sum(costs[i][seq[i]] for i in range(n))
        for i in range(1, n):
            j = abs(seq[i] - seq[i - 1])
            e += 0 if j == 0 else (P1 if j == 1 else P2)
        if best[seq[-1]] is None or e < best[seq[-1]]:
            best[seq[-1]] = e
    return best


@pytest.mark.parametrize("P1,P2", [(7, 86), (3, 3), (0, 5), (2, 40), (0, 0)])
@pytest.mark.parametrize("r", range(8))
def test_path_equals_brute_force_min_energy(r, P1, P2):
    rng = np.random.default_rng(100 + r + 10 * P1 + P2)
    H, W, D = 4, 5, 3
    C = rng.integers(0, 25, size=(H, W, D)).astype(np.uint8)
    rx, ry = DIRS[r]
    L = oracle.path(C, rx, ry, P1, P2)
    for y in range(H):
        for x in range(W):
            # the scanline that ends at (x, y), from its entry pixel onwards
            line = []
            qx, qy = x, y
            while 0 <= qx < W and 0 <= qy < H:
                line.append((qx, qy))
                qx, qy = qx - rx, qy - ry
            line.reverse()
            want = _min_energy_ending([C[qy, qx].astype(int).tolist() for qx, qy in line], P1, P2)
            offset = sum(int(L[qy, qx].min()) for qx, qy in line[:-1])
            got = [int(v) + offset for v in L[y, x]]
            assert got == want, (r, x, y, got, want)


@pytest.mark.parametrize("n,D", [(6, 4), (5, 4), (3, 2)])
def test_1d_line_brute_force_long(n, D):
    rng = np.random.default_rng(n * 10 + D)
    P1, P2 = 4, 11
    C = rng.integers(0, 30, size=(1, n, D)).astype(np.uint8)
    L = oracle.path(C, 1, 0, P1, P2)
    for x in range(n):
        want = _min_energy_ending(C[0, : x + 1].astype(int).tolist(), P1, P2)
        offset = sum(int(L[0, k].min()) for k in range(x))
        assert [int(v) + offset for v in L[0, x]] == want


def test_large_penalties_give_prefix_sums():
    # with every label change dearer than any cost sum, the best sequence ending
    # in d keeps d throughout: the energy is the prefix column sum of C(., d)
    rng = np.random.default_rng(9)
    n, D = 7, 5
    C = rng.integers(0, 20, size=(1, n, D)).astype(np.uint8)
    P = 20 * n + 1
    L = oracle.path(C, 1, 0, P, P)
    offset = 0
    for x in range(n):
        want = C[0, : x + 1].astype(int).sum(axis=0)
        np.testing.assert_array_equal(L[0, x].astype(int) + offset, want)
        offset += int(L[0, x].min())


@pytest.mark.parametrize("r", range(8))
def test_path_bounds(r):
    rng = np.random.default_rng(r)
    C = rng.integers(0, 49, size=(9, 11, 16)).astype(np.uint8)
    P1, P2 = 7, 86
    L = oracle.path(C, *DIRS[r], P1, P2)
    Ci = C.astype(np.int32)
    assert (L >= Ci).all() and (L <= Ci + P2).all()
    assert (L.min(axis=2) >= Ci.min(axis=2)).all()


def test_transpose_symmetry():
    rng = np.random.default_rng(4)
    C = rng.integers(0, 49, size=(7, 10, 6)).astype(np.uint8)
    Ct = np.ascontiguousarray(C.transpose(1, 0, 2))
    P1, P2 = 7, 86
    # transposing swaps x and y, so direction (rx, ry) becomes (ry, rx)
    for rx, ry in DIRS:
        a = oracle.path(C, rx, ry, P1, P2)
        b = oracle.path(Ct, ry, rx, P1, P2).transpose(1, 0, 2)
        np.testing.assert_array_equal(a, b)


def test_mirror_symmetry():
    rng = np.random.default_rng(6)
    C = rng.integers(0, 49, size=(6, 9, 5)).astype(np.uint8)
    Cm = np.ascontiguousarray(C[:, ::-1])
    for rx, ry in DIRS:
        a = oracle.path(C, rx, ry, 7, 86)
        b = oracle.path(Cm, -rx, ry, 7, 86)[:, ::-1]
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("paths", [4, 8])
def test_zero_penalties_sum_is_paths_times_cost(paths):
    rng = np.random.default_rng(paths)
    C = rng.integers(0, 49, size=(5, 8, 7)).astype(np.uint8)
    S = oracle.aggregate(C, paths, 0, 0)
    np.testing.assert_array_equal(S, paths * C.astype(np.int32))


def test_aggregate_is_sum_of_listed_directions():
    # 4 paths are the horizontal and vertical directions; 8 add the diagonals
    rng = np.random.default_rng(8)
    C = rng.integers(0, 49, size=(5, 6, 4)).astype(np.uint8)
    hv = [(1, 0), (-1, 0), (0, 1), (0, -1)]
    diag = [(1, 1), (-1, 1), (1, -1), (-1, -1)]
    s4 = sum(oracle.path(C, rx, ry, 7, 86).astype(np.int64) for rx, ry in hv)
    s8 = s4 + sum(oracle.path(C, rx, ry, 7, 86).astype(np.int64) for rx, ry in diag)
    np.testing.assert_array_equal(oracle.aggregate(C, 4, 7, 86), s4)
    np.testing.assert_array_equal(oracle.aggregate(C, 8, 7, 86), s8)
