"""The seeded synthetic inputs (no halftoning arithmetic): each array is a pure function of
its seed tuple and follows its stated recipe -- gradient background spanning 0.1 .. 0.9,
ellipses painted with uniform grays, Gaussian noise, clamping to [0, 1]; He-normal weights;
log-uniform uneven sizes within their clamps."""
import math

import numpy as np
import pytest

from paper_2304_12152_gb300 import synth


def test_contone_is_a_pure_function_of_its_seed_tuple():
    a = synth.contone_image(64, 80, seed=3, index=2)
    assert a.dtype == np.float32 and a.shape == (64, 80)
    assert np.array_equal(a, synth.contone_image(64, 80, seed=3, index=2))
    assert not np.array_equal(a, synth.contone_image(64, 80, seed=3, index=1))
    assert not np.array_equal(a, synth.contone_image(64, 80, seed=4, index=2))
    assert a.min() >= 0.0 and a.max() <= 1.0
    with pytest.raises(ValueError):
        synth.contone_image(0, 5, seed=0)


def test_gradient_background_spans_point_one_to_point_nine():
    for seed in range(5):
        g = synth.contone_image(50, 70, seed=seed, n_ellipses=0, noise_sigma=0.0).astype(np.float64)
        assert abs(g.min() - 0.1) < 1e-6 and abs(g.max() - 0.9) < 1e-6
        # linear in (x, y): every second difference along a row or column vanishes
        assert np.abs(np.diff(g, 2, axis=1)).max() < 1e-5 and np.abs(np.diff(g, 2, axis=0)).max() < 1e-5


def test_ellipses_paint_flat_regions_and_noise_has_the_stated_sigma():
    clean = synth.contone_image(256, 256, seed=7, noise_sigma=0.0).astype(np.float64)
    bg = synth.contone_image(256, 256, seed=7, n_ellipses=0, noise_sigma=0.0).astype(np.float64)
    painted = np.abs(clean - bg) > 1e-6
    assert 0.05 < painted.mean() < 0.99
    # painted pixels take at most 20 distinct grays
    assert len(np.unique(np.round(clean[painted], 6))) <= 20
    noisy = synth.contone_image(256, 256, seed=7).astype(np.float64)
    inner = (clean > 0.1) & (clean < 0.9)                # away from the clamp
    d = (noisy - clean)[inner]
    assert abs(d.std() - 0.02) < 0.001 and abs(d.mean()) < 0.001


def test_he_normal_weights():
    chs = synth.NET_WIDE
    ws, bs = synth.he_normal_policy(chs, seed=5)
    assert [w.shape for w in ws] == [(chs[l + 1], chs[l], 3, 3) for l in range(len(chs) - 1)]
    for l, w in enumerate(ws[:-1]):
        std = math.sqrt(2.0 / (9 * chs[l]))
        n = w.size
        assert abs(w.std() / std - 1) < 5 / math.sqrt(2 * n) + 1e-3, l
        assert abs(w.mean()) < 5 * std / math.sqrt(n)
    assert all(not b.any() for b in bs)
    w2, _ = synth.he_normal_policy(chs, seed=5)
    assert all(np.array_equal(a, b) for a, b in zip(ws, w2))


def test_uneven_shapes_recipe():
    shapes = synth.uneven_shapes(4000, seed=4)
    assert shapes == synth.uneven_shapes(4000, seed=4) and len(shapes) == 4000
    h = np.array([s[0] for s in shapes], float)
    w = np.array([s[1] for s in shapes], float)
    assert h.min() >= 200 and w.min() >= 200 and h.max() <= 4096 and w.max() <= 4096
    # log-area uniform between log(200 * 300) and log(4096 * 3072) away from the clamps
    la = np.log(h * w)
    lo, hi = math.log(200 * 300), math.log(4096 * 3072)
    unclamped = (h > 200) & (w > 200) & (h < 4096) & (w < 4096)
    mid = (la > lo + 1) & (la < hi - 1) & unclamped
    frac = mid.mean()
    assert abs(frac - (hi - lo - 2) / (hi - lo)) < 0.08
    # aspect w / h within [1/2, 2] wherever no side was clamped (rounding aside)
    r = (w / h)[unclamped]
    assert r.min() > 0.49 and r.max() < 2.02
    # the benchmark's 64-image draw is the first 64 of the same stream
    assert synth.uneven_shapes(64, seed=4) == shapes[:64]
