"""Pins of the oracle's reward (Eq. reward, Eq. final_reward, Eq. cssim, contrast map)."""
import numpy as np
import pytest
from scipy.signal import correlate2d

import oracle as O
from paper_2304_12152_gb300 import synth


def test_gaussian_window_normalised_and_separable():
    for s in (1.5, 2.0):
        g = O.gauss2d(s, 5)
        assert abs(g.sum() - 1.0) < 1e-14
        k = np.exp(-np.arange(-5, 6) ** 2 / (2 * s * s)); k /= k.sum()
        np.testing.assert_allclose(g, np.outer(k, k), rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(g, g.T, rtol=0, atol=0)


def test_identical_images():
    """SSIM(x, x) = 1 and CSSIM(x, x) = 1, MSE = 0 for a binary 'contone'."""
    rng = np.random.default_rng(0)
    hb = (rng.random((30, 27)) < 0.4).astype(np.uint8)
    r = O.reward(hb.astype(np.float32), hb)
    assert abs(r["ssim"] - 1) < 1e-12 and abs(r["cssim"] - 1) < 1e-12 and r["mse"] < 1e-28
    assert abs(r["R"] - 0.06) < 1e-12


@pytest.mark.parametrize("g", [0.1, 0.25, 0.5, 0.75])
def test_constant_contone(g):
    """Constant contone: zero contrast -> CSSIM = 1 for any halftone; MSE closed form."""
    c = np.full((21, 25), g, np.float32)
    ones = np.ones_like(c, dtype=np.uint8)
    r = O.reward(c, ones)
    gg = float(np.float32(g))
    assert abs(r["mse"] - (1 - gg) ** 2) < 1e-12
    assert abs(r["cssim"] - 1) < 1e-12
    rng = np.random.default_rng(1)
    r2 = O.reward(c, (rng.random(c.shape) < g).astype(np.uint8))
    assert abs(r2["cssim"] - 1) < 1e-12


def test_maps_against_library_filtering():
    c = synth.contone_image(40, 33, seed=3)
    rng = np.random.default_rng(2)
    hb = (rng.random(c.shape) < c).astype(np.uint8)
    r = O.reward(c, hb, maps=True)
    cd, hd = c.astype(np.float64), hb.astype(np.float64)
    ghvs, gw = O.gauss2d(2.0), O.gauss2d(1.5)
    e = correlate2d(hd, ghvs, "valid") - correlate2d(cd, ghvs, "valid")
    np.testing.assert_allclose(r["e"], e, atol=1e-13)
    assert abs(r["mse"] - np.mean(e * e)) < 1e-14
    mu = correlate2d(cd, gw, "valid")
    var = correlate2d(cd * cd, gw, "valid") - mu * mu
    np.testing.assert_allclose(r["sigma"], 2 * np.sqrt(np.maximum(var, 0)), atol=1e-7)
    assert r["sigma"].max() <= 1.0 + 1e-12                 # std of [0,1] data <= 1/2
    # valid region size M = (H-10)(W-10)
    assert r["e"].shape == (30, 23)
    np.testing.assert_allclose(r["cssim"], np.mean(r["sigma"] * r["ssim_map"] + 1 - r["sigma"]), rtol=1e-13)
    assert abs(r["R"] - (-r["mse"] + 0.06 * r["cssim"])) < 1e-15


def test_ssim_symmetry_and_bounds():
    c = synth.contone_image(24, 24, seed=5)
    rng = np.random.default_rng(4)
    hb = (rng.random(c.shape) < c).astype(np.uint8)
    r = O.reward(c, hb, maps=True)
    assert np.all(r["ssim_map"] <= 1 + 1e-12) and np.all(r["ssim_map"] >= -1 - 1e-12)
    # SSIM is symmetric in its two arguments: swap roles through a binary/binary pair
    hb2 = (rng.random(c.shape) < 0.5).astype(np.uint8)
    a = O.reward(hb2.astype(np.float32), hb, maps=True)["ssim_map"]
    b = O.reward(hb.astype(np.float32), hb2, maps=True)["ssim_map"]
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_rejects_too_small():
    with pytest.raises(ValueError):
        O.reward(np.zeros((10, 30), np.float32), np.zeros((10, 30), np.uint8))
