"""Pins of the oracle's sensor-noise step (arxiv 2201.11924 Sec. VI-C:
I_noisy = gamma * I_clean + n, gamma ~ Gamma(k, theta), n ~ N(mu, sigma^2);
the D415 parameters of Sec. VII).

The generator is pinned bit for bit to numpy's own Philox4x64-10 (which
advances its counter before producing a block); the samples are pinned to the
closed-form distributions (Kolmogorov-Smirnov and moments on fixed seeds),
the independence of the two terms through the variance of their sum, and the
noise-free limit."""
import numpy as np
import pytest
import scipy.stats

import oracle

P = oracle.D415_NOISE


@pytest.mark.parametrize("ctr,key", [([0, 0, 0, 0], [0, 0]), ([5, 7, 9, 11], [123, 456]),
                                     ([2**64 - 2, 3, 2**63, 1], [2**64 - 1, 77])])
def test_philox_matches_numpy(ctr, key):
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    want = bg.random_raw(4)
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64           # numpy increments the 256-bit counter first
    if c[0] == 0:
        c[1] += 1
    got = oracle.philox4x64(c, key)
    assert np.array_equal(got, want)


def test_gamma_term_follows_its_distribution():
    # I_clean = 100, no thermal term: value / 100 is the speckle factor gamma
    img = np.full((300, 400), 100, dtype=np.uint8)
    _, v, _ = oracle.noise(img, 0.0, 0.0, P["k"], P["theta"], seed=11)
    g = (v / 100.0).ravel()
    ks = scipy.stats.kstest(g, scipy.stats.gamma(a=P["k"], scale=P["theta"]).cdf)
    assert ks.pvalue > 1e-3
    se = np.sqrt(P["k"] * P["theta"] ** 2 / g.size)
    assert abs(g.mean() - P["k"] * P["theta"]) < 4 * se


def test_thermal_term_follows_its_distribution():
    img = np.zeros((300, 400), dtype=np.uint8)
    _, v, _ = oracle.noise(img, P["mu"], P["sigma"], P["k"], P["theta"], seed=12)
    ks = scipy.stats.kstest(v.ravel(), scipy.stats.norm(loc=P["mu"], scale=P["sigma"]).cdf)
    assert ks.pvalue > 1e-3


def test_terms_are_independent():
    # Var(gamma I + n) = I^2 Var(gamma) + sigma^2 only if the terms are uncorrelated
    I = 60
    img = np.full((400, 500), I, dtype=np.uint8)
    _, v, _ = oracle.noise(img, 0.0, 3.0, P["k"], P["theta"], seed=13)
    want = I * I * P["k"] * P["theta"] ** 2 + 9.0
    assert abs(v.var() / want - 1.0) < 0.02


def test_noise_free_limit_returns_the_clean_image():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (64, 80), dtype=np.uint8)
    # gamma ~ Gamma(1e8, 1e-8) has mean 1 and spread 1e-4: far below half a level
    n, _, _ = oracle.noise(img, 0.0, 0.0, 1e8, 1e-8, seed=4)
    assert np.array_equal(n, img)


def test_quantisation_and_streams():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (40, 50), dtype=np.uint8)
    a, va, _ = oracle.noise(img, **P, seed=9, frame=2, view=0)
    b, _, _ = oracle.noise(img, **P, seed=9, frame=2, view=0)
    c, _, _ = oracle.noise(img, **P, seed=9, frame=2, view=1)
    d, _, _ = oracle.noise(img, **P, seed=9, frame=3, view=0)
    assert np.array_equal(a, b)                               # deterministic
    assert (a != c).mean() > 0.5 and (a != d).mean() > 0.5    # other streams
    assert np.array_equal(a, np.clip(np.rint(va), 0, 255).astype(np.uint8))
