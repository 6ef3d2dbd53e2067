"""Pins of the oracle's multitoning prototype (Sec. VI-E): the action between the two
levels around the sigmoid output, the reward of a multi-level halftone, the toggle deltas
between those two levels and the local-expectation surrogate built on them."""
import numpy as np
import pytest
from scipy.signal import correlate2d

import oracle as O
from paper_2304_12152_gb300 import synth


@pytest.mark.parametrize("L", [2, 3, 4])
def test_action_pair_and_rule(L):
    rng = np.random.default_rng(L)
    v = rng.random(20000)
    k, frac = O.multitone_pair(v, L)
    d = 1.0 / (L - 1)
    assert np.all((k >= 0) & (k <= L - 2)) and np.all((frac >= 0) & (frac < 1))
    np.testing.assert_allclose(k * d + frac * d, v, atol=1e-15)          # v = floor + frac * Delta
    # v = 1 belongs to the top pair (L - 2, L - 1) with the upper level certain, so its toggle
    # is between two valid levels
    k1, f1 = O.multitone_pair(np.array([1.0, 0.0]), L)
    assert (k1[0], f1[0]) == (L - 2, 1.0) and (k1[1], f1[1]) == (0, 0.0)
    # exact levels map to themselves (threshold and any u); 0 and 1 included
    lv = np.arange(L) / (L - 1)
    assert np.array_equal(O.sample_multitone(lv, L), np.arange(L))
    assert np.array_equal(O.sample_multitone(lv, L, u=np.full(L, 0.999)), np.arange(L))
    # threshold = nearest level
    near = np.rint(v * (L - 1)).astype(np.int64)
    off = np.abs(frac - 0.5) > 1e-9
    assert np.array_equal(O.sample_multitone(v, L)[off], near[off])
    # a tie (frac exactly 1/2: v (L - 1) = 0.5 or 1.5, exact in binary) goes to the lower
    # level, as p = 1/2 does in the binary threshold rule
    vt = np.array([{2: 0.5, 3: 0.25, 4: 0.5}[L]])
    kt, ft = O.multitone_pair(vt, L)
    assert ft[0] == 0.5 and O.sample_multitone(vt, L)[0] == kt[0]
    # Bernoulli: only the two levels around v, upper one with probability frac
    u = rng.random(v.shape)
    h = O.sample_multitone(v, L, u).astype(np.int64)
    assert np.all((h == k) | (h == k + 1))
    vs = np.full(400000, 0.37)
    ks, fs = O.multitone_pair(vs, L)
    hs = O.sample_multitone(vs, L, rng.random(vs.shape)).astype(np.int64)
    assert abs(np.mean(hs == ks + 1) - fs[0]) < 4 * np.sqrt(fs[0] * (1 - fs[0]) / vs.size)
    # L = 2 is the binary rule h = [u < v]
    if L == 2:
        assert np.array_equal(h, (u < v).astype(np.int64))


@pytest.mark.parametrize("L", [3, 4])
def test_multilevel_reward_against_direct_filtering(L):
    """MSE, SSIM with E[h^2] != E[h] and CSSIM of a multi-level halftone against scipy."""
    c = synth.contone_image(37, 41, seed=5)
    rng = np.random.default_rng(9)
    idx = rng.integers(0, L, c.shape).astype(np.uint8)
    r = O.reward(c, idx, maps=True, levels=L)
    hd, cd = idx.astype(np.float64) / (L - 1), c.astype(np.float64)
    ghvs, gw = O.gauss2d(2.0), O.gauss2d(1.5)
    e = correlate2d(hd, ghvs, "valid") - correlate2d(cd, ghvs, "valid")
    assert abs(r["mse"] - np.mean(e * e)) < 1e-14
    mh, mc = correlate2d(hd, gw, "valid"), correlate2d(cd, gw, "valid")
    vh = correlate2d(hd * hd, gw, "valid") - mh * mh
    vc = correlate2d(cd * cd, gw, "valid") - mc * mc
    cov = correlate2d(hd * cd, gw, "valid") - mh * mc
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    ssim = (2 * mh * mc + c1) * (2 * cov + c2) / ((mh * mh + mc * mc + c1) * (vh + vc + c2))
    np.testing.assert_allclose(r["ssim_map"], ssim, rtol=1e-9, atol=1e-12)
    sig = 2 * np.sqrt(np.maximum(vc, 0))
    assert abs(r["cssim"] - np.mean(sig * ssim + 1 - sig)) < 1e-11
    # L = 2 with 0/1 indices is the binary reward
    hb = (rng.random(c.shape) < c).astype(np.uint8)
    assert O.reward(c, hb, levels=2)["R"] == O.reward(c, hb)["R"]


@pytest.mark.parametrize("L", [3, 4])
def test_multilevel_toggle_against_brute_force(L):
    c = synth.contone_image(24, 26, seed=6)
    rng = np.random.default_rng(11)
    v = rng.random(c.shape)
    k, frac = O.multitone_pair(v, L)
    h = O.sample_multitone(v, L, rng.random(c.shape))
    idx = np.array([0, 5, 25, 26 * 12 + 13, 26 * 23 + 25, 300, 401], np.int64)
    d = O.toggle_delta(c, h, idx, levels=L, lo=k.astype(np.uint8))
    for t, a in enumerate(idx):
        y, x = divmod(int(a), 26)
        hi_img, lo_img = h.copy(), h.copy()
        hi_img[y, x] = k[y, x] + 1
        lo_img[y, x] = k[y, x]
        ref = O.reward(c, hi_img, levels=L)["R"] - O.reward(c, lo_img, levels=L)["R"]
        assert abs(d[t] - ref) < 1e-12 * max(1.0, abs(ref)) + 1e-15, (t, d[t], ref)


def test_multitone_le_estimator_is_unbiased_by_enumeration():
    """E_{h~pi}[dR_a / Delta] = dJ/dv_a with J(v) = sum_h prod_a pi_a(h_a) R(h), enumerated
    over all 2^16 pairs-of-levels halftones of a 4x4 image (L = 4, 3x3 reward window)."""
    L, N = 4, 16
    opts = O.reward_opts(radius=1, sigma_hvs=1.0, sigma_ssim=1.0)
    c = synth.contone_image(4, 4, seed=12)
    rng = np.random.default_rng(13)
    k = rng.integers(0, L - 1, N)
    frac = rng.uniform(0.1, 0.9, N)
    v = (k + frac) / (L - 1)
    kk, ff = O.multitone_pair(v, L)
    assert np.array_equal(kk, k)
    bits = ((np.arange(1 << N)[:, None] >> np.arange(N)[None]) & 1)
    Rs = np.zeros(1 << N)
    dRs = np.zeros((1 << N, N))
    for q in range(1 << N):
        h = (k + bits[q]).astype(np.uint8).reshape(4, 4)
        Rs[q] = O.reward(c, h, opts, levels=L)["R"]
        dRs[q] = O.toggle_delta(c, h, opts=opts, levels=L, lo=k.astype(np.uint8))

    def J(ff_):
        pi = np.prod(np.where(bits > 0, ff_[None], 1 - ff_[None]), axis=1)
        return pi, float(pi @ Rs)

    pi, _ = J(ff)
    est = (pi @ dRs) * (L - 1)                                   # E[dR_a / Delta]
    eps = 1e-3                                                   # dv = eps keeps v inside its level pair
    fd = np.array([(J(ff + eps * (L - 1) * np.eye(N)[a])[1] - J(ff - eps * (L - 1) * np.eye(N)[a])[1]) / (2 * eps)
                   for a in range(N)])
    np.testing.assert_allclose(est, fd, rtol=1e-8, atol=1e-12)


def test_multitone_surrogate_value_by_brute_force():
    L = 3
    c = synth.contone_image(14, 13, seed=21)
    rng = np.random.default_rng(22)
    v = rng.random(c.shape)
    k, frac = O.multitone_pair(v, L)
    h = O.sample_multitone(v, L, rng.random(c.shape))
    R = O.reward(c, h, levels=L)["R"]
    dR = O.toggle_delta(c, h, levels=L, lo=k.astype(np.uint8)).reshape(c.shape)
    val, grad = O.le_surrogate_multitone(v, h, dR, R, L)
    ref = 0.0
    for y in range(c.shape[0]):
        for x in range(c.shape[1]):
            hi, lo = h.copy(), h.copy()
            hi[y, x], lo[y, x] = k[y, x] + 1, k[y, x]
            ref -= frac[y, x] * O.reward(c, hi, levels=L)["R"] + (1 - frac[y, x]) * O.reward(c, lo, levels=L)["R"]
    assert abs(val - ref) < 1e-10 * abs(ref)
    np.testing.assert_array_equal(grad, -dR * (L - 1))
