"""Pins of the oracle's toggle deltas and of the local-expectation estimator (Eq. le, Eq. marl)."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2304_12152_gb300 import synth


def test_toggle_delta_brute_force():
    """dR_a from the windowed recompute equals R(flip to 1) - R(flip to 0) from two full rewards."""
    c = synth.contone_image(24, 24, seed=7)
    rng = np.random.default_rng(5)
    hb = (rng.random(c.shape) < c).astype(np.uint8)
    d = O.toggle_delta(c, hb)
    ref = np.zeros(24 * 24)
    for a in range(24 * 24):
        y, x = divmod(a, 24)
        h1 = hb.copy(); h1[y, x] = 1
        h0 = hb.copy(); h0[y, x] = 0
        ref[a] = O.reward(c, h1)["R"] - O.reward(c, h0)["R"]
    np.testing.assert_allclose(d, ref, rtol=1e-9, atol=1e-15)
    # corner pixels outside every valid window of radius 5 still touch some (24 >= 11)
    assert np.all(np.abs(d) > 0)


def test_le_estimator_is_unbiased_by_enumeration():
    """E_{h~pi}[sum_{h'} d pi_a(h') R(h'_a, h_-a)] = dJ/dp_a exactly (J multilinear in p),
    enumerated over all 2^16 halftones of a 4x4 image with a 3x3 reward window."""
    opts = O.reward_opts(radius=1, sigma_hvs=1.0, sigma_ssim=1.0)
    c = synth.contone_image(4, 4, seed=8)
    rng = np.random.default_rng(6)
    p = rng.uniform(0.1, 0.9, 16)
    N = 16
    Rs = np.zeros(1 << N)
    dRs = np.zeros((1 << N, N))
    for k in range(1 << N):
        hb = np.array([(k >> i) & 1 for i in range(N)], np.uint8).reshape(4, 4)
        Rs[k] = O.reward(c, hb, opts)["R"]
        dRs[k] = O.toggle_delta(c, hb, opts=opts)
    bits = ((np.arange(1 << N)[:, None] >> np.arange(N)[None]) & 1).astype(np.float64)

    def J(pp):
        pi = np.prod(np.where(bits > 0, pp[None], 1 - pp[None]), axis=1)
        return pi, float(pi @ Rs)

    pi, _ = J(p)
    est = pi @ dRs                                    # E[g_LE] per pixel
    eps = 1e-3
    fd = np.array([(J(p + eps * np.eye(N)[a])[1] - J(p - eps * np.eye(N)[a])[1]) / (2 * eps) for a in range(N)])
    np.testing.assert_allclose(est, fd, rtol=1e-8, atol=1e-13)


def test_le_surrogate_value_and_gradient():
    """Algorithm 1: L_MARL = -sum_a sum_{h'} R({h'_a, h_-a}) pi_a(h'_a), checked term by term."""
    c = synth.contone_image(16, 16, seed=9)
    rng = np.random.default_rng(7)
    p = rng.uniform(0.05, 0.95, (16, 16))
    hb = (rng.random(c.shape) < p).astype(np.uint8)
    R = O.reward(c, hb)["R"]
    dR = O.toggle_delta(c, hb).reshape(16, 16)
    val, grad = O.le_surrogate(p, hb, dR, R)
    ref = 0.0
    for y in range(16):
        for x in range(16):
            h1 = hb.copy(); h1[y, x] = 1
            h0 = hb.copy(); h0[y, x] = 0
            ref -= p[y, x] * O.reward(c, h1)["R"] + (1 - p[y, x]) * O.reward(c, h0)["R"]
    assert abs(val - ref) < 1e-10 * abs(ref)
    np.testing.assert_array_equal(grad, -dR)


def test_coma_estimator_is_unbiased_by_enumeration():
    """Eq. (coma): E_{h~pi}[d log pi_a(h_a)/dp_a (R(h) - b_a(h_-a))] = dJ/dp_a exactly,
    enumerated over all 2^16 halftones of a 4x4 image with a 3x3 reward window; the
    baseline b_a is formed from brute-force rewards of both actions of agent a."""
    opts = O.reward_opts(radius=1, sigma_hvs=1.0, sigma_ssim=1.0)
    c = synth.contone_image(4, 4, seed=8)
    rng = np.random.default_rng(16)
    p = rng.uniform(0.1, 0.9, 16)
    N = 16
    Rs = np.array([O.reward(c, np.array([(k >> i) & 1 for i in range(N)], np.uint8).reshape(4, 4), opts)["R"]
                   for k in range(1 << N)])
    bits = ((np.arange(1 << N)[:, None] >> np.arange(N)[None]) & 1)
    pi = np.prod(np.where(bits > 0, p[None], 1 - p[None]), axis=1)
    est = np.zeros(N)
    for a in range(N):
        k1 = np.arange(1 << N) | (1 << a)
        k0 = np.arange(1 << N) & ~(1 << a)
        b = p[a] * Rs[k1] + (1 - p[a]) * Rs[k0]                      # Eq. (baseline)
        dlog = np.where(bits[:, a] > 0, 1.0 / p[a], -1.0 / (1.0 - p[a]))
        est[a] = pi @ (dlog * (Rs - b))
    eps = 1e-3

    def J(pp):
        return float(np.prod(np.where(bits > 0, pp[None], 1 - pp[None]), axis=1) @ Rs)

    fd = np.array([(J(p + eps * np.eye(N)[a]) - J(p - eps * np.eye(N)[a])) / (2 * eps) for a in range(N)])
    np.testing.assert_allclose(est, fd, rtol=1e-8, atol=1e-13)
    # the oracle's closed form (from the toggle deltas) gives the same per-sample gradient
    for k in (0, 12345, (1 << N) - 1):
        hb = bits[k].astype(np.uint8).reshape(4, 4)
        dR = O.toggle_delta(c, hb, opts=opts).reshape(4, 4)
        _, g = O.coma_surrogate(p.reshape(4, 4), hb, dR, Rs[k])
        for a in range(N):
            b = p[a] * Rs[k | (1 << a)] + (1 - p[a]) * Rs[k & ~(1 << a)]
            dlog = 1.0 / p[a] if bits[k, a] else -1.0 / (1.0 - p[a])
            assert abs(-g.ravel()[a] - dlog * (Rs[k] - b)) < 1e-12


def test_coma_surrogate_value_by_brute_force():
    """L_COMA = -sum_a log pi_a(h_a) (R(h) - b_a) with b_a from brute-force flipped rewards."""
    c = synth.contone_image(12, 12, seed=19)
    rng = np.random.default_rng(17)
    p = rng.uniform(0.05, 0.95, (12, 12))
    hb = (rng.random(c.shape) < p).astype(np.uint8)
    R = O.reward(c, hb)["R"]
    dR = O.toggle_delta(c, hb).reshape(12, 12)
    val, grad = O.coma_surrogate(p, hb, dR, R)
    ref = 0.0
    for y in range(12):
        for x in range(12):
            h1 = hb.copy(); h1[y, x] = 1
            h0 = hb.copy(); h0[y, x] = 0
            b = p[y, x] * O.reward(c, h1)["R"] + (1 - p[y, x]) * O.reward(c, h0)["R"]
            lp = np.log(p[y, x]) if hb[y, x] else np.log(1 - p[y, x])
            ref -= lp * (R - b)
    assert abs(val - ref) < 1e-9 * abs(ref)
