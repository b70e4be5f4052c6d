"""Pins for the oracle's disorder generator (SplitMix64 + box distribution)."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_splitmix():
    vals = []
    for line in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            vals.append(int(line, 16))
    return vals


def test_splitmix64_published_vector():
    want = _golden_splitmix()
    got = [int(v) for v in rng.splitmix64(0, len(want))]
    assert got == want


def test_splitmix64_is_counter_based():
    full = rng.splitmix64(987654321, 100)
    part = rng.splitmix64(987654321, 10, offset=90)
    assert np.array_equal(full[90:], part)


def test_uniform_uses_top_53_bits():
    z = rng.splitmix64(5, 1000)
    u = rng.uniform01(5, 1000)
    assert np.all(u >= 0.0) and np.all(u < 1.0)
    # exact reconstruction of the top 53 bits
    assert np.array_equal((u * 2.0 ** 53).astype(np.uint64), z >> np.uint64(11))


@pytest.mark.parametrize("W", [1.0, 16.5, 21.0])
def test_potential_box_distribution(W):
    n = 200_000
    eps = rng.potential(round(n ** (1 / 3)) + 1, W, 3)
    assert eps.min() >= -W / 2 and eps.max() < W / 2
    # covers the box: extremes within 1e-3 relative of the edges
    assert eps.min() < -W / 2 * (1 - 1e-3) and eps.max() > W / 2 * (1 - 1e-3)
    ks = stats.kstest((eps + W / 2) / W, "uniform")
    assert ks.pvalue > 1e-4
    assert abs(eps.mean()) < 5 * W / np.sqrt(12 * len(eps))


def test_potential_zero_disorder_and_seeds_differ():
    assert np.all(rng.potential(4, 0.0, 1) == 0.0)
    a = rng.potential(6, 16.5, 1)
    b = rng.potential(6, 16.5, 2)
    assert not np.array_equal(a, b)
    assert np.array_equal(a, rng.potential(6, 16.5, 1))
