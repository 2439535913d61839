"""The selection kernel adds 16-bit path sums with add.f16x2: a half whose
bit pattern is an integer n < 2048 is the f16 value n * 2^-24 (subnormal for
n < 1024, exponent field 1 above), so IEEE addition of two such halves is
exact and its bit pattern is the integer sum as long as the sum stays below
2048 (eight path bytes sum to at most 8 * 255 = 2040).  Checked here
exhaustively with numpy's IEEE half-precision arithmetic; the GPU parity
tests check the kernel's sums themselves against the oracle."""
import numpy as np


def test_f16_bit_patterns_add_like_integers_below_2048():
    n = np.arange(2048, dtype=np.uint16)
    a = np.repeat(n[:, None], 2048, axis=1)
    b = np.repeat(n[None, :], 2048, axis=0)
    ok = (a.astype(np.int32) + b.astype(np.int32)) < 2048
    s = (a.view(np.float16) + b.view(np.float16)).view(np.uint16)
    assert np.array_equal(s[ok], (a + b)[ok])


def test_eight_path_bytes_stay_below_2048():
    rng = np.random.default_rng(7)
    paths = rng.integers(0, 256, size=(8, 4096), dtype=np.uint16)
    paths[:, 0] = 255                                  # the largest sum, 2040
    acc = paths[0].view(np.float16)
    for r in range(1, 8):
        acc = (acc + paths[r].view(np.float16)).astype(np.float16)
    assert np.array_equal(acc.view(np.uint16), paths.sum(axis=0))
    assert int(paths.sum(axis=0).max()) == 2040
