"""Both SGM kernels split a word of four cost or path bytes (b0, b1, b2, b3)
into 16-bit pairs (b0, b2) and (b1, b3) without a byte mask.  One permute
gives o = (b1, b3); the even pair is then w - 256 * o, folded into the adds
that follow, and every sum is taken modulo 2^32:
 - the selection adds the whole words of up to 8 paths (carries between bytes
   included) and the odd pairs separately, then takes 256 * sum(o) off:
   sum(w) - 256 * sum(o) = sum(b0) + 2^16 sum(b2), exact because it is below
   2^32 although the running word sum is not;
 - the path recurrence forms L = t + w - m' - 256 * o, which equals
   (t - m') + (b0, b2) with every half of t at least the matching half of m'.
Checked here in numpy's modular uint32 arithmetic, on random words and on
the extremes (all bytes 255, all 0); the GPU parity tests check the kernels'
sums and path costs themselves against the oracle."""
import numpy as np

MASK = np.uint32(0x00FF00FF)


def odd_pair(w):
    # the permute with selector 0x4341 and a zero second operand
    return (w >> np.uint32(8)) & MASK


def words(rng, n):
    w = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    w[:4] = [0xFFFFFFFF, 0, 0xFF00FF00, 0x00FF00FF]
    return w


def test_path_sums_without_mask_equal_masked_sums():
    rng = np.random.default_rng(11)
    for paths in (1, 2, 4, 8):
        a = np.stack([words(rng, 1 << 16) for _ in range(paths)])
        with np.errstate(over="ignore"):
            ev = a.sum(axis=0, dtype=np.uint32)
            od = odd_pair(a).sum(axis=0, dtype=np.uint32)
            ev = ev - od * np.uint32(256)
        want_even = (a & MASK).astype(np.uint64).sum(axis=0)
        want_odd = odd_pair(a).astype(np.uint64).sum(axis=0)
        assert np.array_equal(ev.astype(np.uint64), want_even)
        assert np.array_equal(od.astype(np.uint64), want_odd)
        # every half holds the plain sum of its bytes
        assert int((ev & np.uint32(0xFFFF)).max()) <= 255 * paths
        assert int((ev >> np.uint32(16)).max()) <= 255 * paths
    # the largest sums: eight paths of 255 in every byte
    a = np.full((8, 1), 0xFFFFFFFF, dtype=np.uint32)
    with np.errstate(over="ignore"):
        ev = a.sum(axis=0, dtype=np.uint32) - odd_pair(a).sum(axis=0, dtype=np.uint32) * np.uint32(256)
    assert int(ev[0]) == 2040 + (2040 << 16)


def test_recurrence_step_without_mask():
    rng = np.random.default_rng(12)
    n = 1 << 18
    m = rng.integers(0, 1 << 14, size=n, dtype=np.uint32)
    m = m | (m << np.uint32(16))                       # m' in both halves
    lo = rng.integers(0, 1 << 14, size=n, dtype=np.uint32)
    hi = rng.integers(0, 1 << 14, size=n, dtype=np.uint32)
    t = (m & np.uint32(0xFFFF)) + lo + ((hi + (m >> np.uint32(16))) << np.uint32(16))
    t[:2] = m[:2]                                      # t equal to m' in both halves
    w = words(rng, n)
    with np.errstate(over="ignore"):
        got = t + w - m - odd_pair(w) * np.uint32(256)
    assert np.array_equal(got, (t - m) + (w & MASK))
