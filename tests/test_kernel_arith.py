"""Exactness of the integer division shortcuts the CUDA kernels rely on,
checked exhaustively over the ranges the method's bounds allow (no GPU).

- Uniqueness threshold (selection kernel): (100 - u) S(d) < 100 S(d*) iff
  S(d) < T = ceil(100 S(d*) / (100 - u)); T is taken as the high 32 bits of
  (100 S(d*) + 99 - u) * (floor(2^32 / (100 - u)) + 1) for 1 <= u <= 98 (u = 99
  divides by one).  S(d*) <= paths * (nbits + P2) <= 8 * 255.
- SGBM block mean (block-cost kernel): floor((sum + floor(n / 2)) / n) as the
  high 32 bits of (sum + floor(n / 2)) * (floor(2^32 / n) + 1), for the
  in-image pixel counts 2 <= n <= 81 and every sum of n byte costs (a count
  of 1 never reaches the kernel).
"""
import numpy as np

S_MAX = 8 * 255


def _mulhi(x, m):
    return (x.astype(np.uint64) * np.uint64(m)) >> np.uint64(32)


def test_uniqueness_threshold_multiply_high_is_exact():
    s = np.arange(S_MAX + 1, dtype=np.uint64)
    for u in range(1, 100):
        num = np.uint64(100) * s + np.uint64(99 - u)
        assert int(num.max()) < 1 << 18
        want = (100 * s + (100 - u) - 1) // (100 - u)                 # ceil(100 s / (100 - u))
        got = num if u == 99 else _mulhi(num, (1 << 32) // (100 - u) + 1)
        assert np.array_equal(got, want), u
        # and the threshold decides the uniqueness inequality as written
        d = np.arange(0, 2 * S_MAX + 1, dtype=np.int64)
        for sstar in (0, 1, 17, 85, 1000, S_MAX):
            t = int(got[sstar])
            assert np.array_equal(d < t, (100 - u) * d < 100 * sstar), (u, sstar)


def test_block_mean_multiply_high_is_exact():
    for n in range(2, 82):
        m = (1 << 32) // n + 1
        assert m < 1 << 32
        x = np.arange(n * 255 + 1, dtype=np.uint64) + np.uint64(n // 2)
        assert int(x.max()) < 1 << 16
        assert np.array_equal(_mulhi(x, m), x // np.uint64(n)), n


def test_one_pixel_count_needs_a_33_bit_multiplier():
    # why a count of 1 is kept away from the kernel: its multiplier
    # floor(2^32 / 1) + 1 does not fit 32 bits, and truncated it gives 0
    assert (1 << 32) // 1 + 1 >= 1 << 32
    assert int(_mulhi(np.array([200], dtype=np.uint64), ((1 << 32) + 1) & 0xffffffff)[0]) == 0
