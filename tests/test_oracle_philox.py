"""Pins of the oracle's counter-based generator (Philox4x32-10, Salmon et al. SC'11)."""
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_known_answers(ctr, key, expect):
    assert list(O.philox(ctr, key)) == expect


def test_uniform_lanes_and_counter_layout():
    # pixel g uses counter (g/4, image, stream, 0) and output lane g%4
    seed = 0x0123456789ABCDEF
    out = O.philox([5, 3, 1, 0], [seed & 0xFFFFFFFF, seed >> 32])
    for lane in range(4):
        u = O.uniform(seed, 3, 1, 20 + lane)
        assert u == (int(out[lane]) >> 8) / 2.0 ** 24


def test_uniform_statistics():
    u = O.uniform_map(7, 0, 0, 256, 256).ravel()
    assert u.min() >= 0.0 and u.max() < 1.0
    # mean and variance of U[0,1): 1/2, 1/12 (65536 samples: 5-sigma bounds)
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / u.size)
    # chi-square over 64 equal bins, 63 dof: 99.99% quantile ~ 116
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    e = u.size / 64
    assert ((hist - e) ** 2 / e).sum() < 116
    # independent streams / images differ
    assert not np.array_equal(O.uniform_map(7, 0, 1, 8, 8), O.uniform_map(7, 0, 0, 8, 8))
    assert not np.array_equal(O.uniform_map(7, 1, 0, 8, 8), O.uniform_map(7, 0, 0, 8, 8))
