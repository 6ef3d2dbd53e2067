"""GPU parity of the FP8 E4M3 tensor-core form and of the 4-level softmax head.

FP8 form: inner-layer weights quantised per output channel (scale amax/448), each
inner layer's input activations stored as e4m3 with a static per-layer scale
(calibrated here with the oracle on a separate generator image and rounded up to a
power of two, so that the division is exact on both sides), FP32 accumulation.  Against
the oracle emulating those rounding points (quant 2): the e4m3 rows of the tight rule
(tests/_cases.TIGHT; median |dp| at float32 rounding, the tail set by rare e4m3 flips) for
the sigmoid head, and actions equal on decided pixels (|p - u| > 1e-4) but at most 1e-3 of
them; the 4-logit head: median |dq| <= 1e-6 and at most 3e-3 mismatches (three decision
boundaries per pixel).  Probability error against the pure FP64 oracle is stated (printed):
e4m3's unit roundoff 2^-4 at six quantisation stages moves a logit of magnitude ~2 by up to
~0.3, i.e. p by up to ~0.08; bounded at 0.15 max and 0.1 at the 99.9th percentile, median
below 0.03.

Softmax head, BF16 form: a decision flips where |cdf_k - u| is below the probability
error (~1e-3 in BF16), so the residual-mismatch allowance scales with the K - 1 = 3
decision boundaries per pixel: 3e-3 of the decided pixels."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

from _cases import compare_levels, decided_mask, tight_rule, unexplained

pytestmark = pytest.mark.gpu


def calibrate(ws, bs, chs):
    """Per-layer input scales for the FP8 form from an FP64 oracle pass (seed 99 image)."""
    c = synth.contone_image(64, 64, seed=99)
    _, _, acts = O.forward(c, ws, bs, noise_seed=99, save_acts=True)
    L = len(chs) - 1
    sc = [1.0] * L
    for l in range(1, L - 1):
        amax = float(np.abs(acts[l - 1]).max())
        sc[l] = 2.0 ** math.ceil(math.log2(max(amax, 1e-6) / 448.0))
    return sc


def _run(pol, imgs, mode, seed):
    cs = [torch.from_numpy(c).cuda() for c in imgs]
    bits, probs = pol.halftone(cs, mode=mode, seed=seed, want_prob=True)
    api.sync()
    lev = [api.unpack_bits(b, c.shape[0], c.shape[1], pol.head) for b, c in zip(bits, imgs)]
    return lev, [p.cpu().numpy().astype(np.float64) for p in probs]


@pytest.mark.parametrize("head,chs", [(N.HT_HEAD_SIGMOID, synth.NET_WIDE), (N.HT_HEAD_SOFTMAX, synth.NET_WIDE_K4)])
def test_fp8_form(head, chs):
    ws, _ = synth.he_normal_policy(chs, 2)
    bs = synth.random_biases(chs, 5)
    sc = calibrate(ws, bs, chs)
    pol = api.Policy(chs, ws, bs, head=head, precision=N.HT_FP8_E4M3)
    pol.set_act_scales(sc)
    shapes = [(70, 200), (33, 129)]
    imgs = [synth.contone_image(h, w, seed=2, index=i) for i, (h, w) in enumerate(shapes)]
    lev, probs = _run(pol, imgs, 1, seed=2)
    tot_n = tot_bad = 0
    errs, dq = [], []
    for i, c in enumerate(imgs):
        h, w = c.shape
        _, p8, _ = O.forward(c, ws, bs, noise_seed=2, image=i, quant=2, act_scale=sc)
        _, px, _ = O.forward(c, ws, bs, noise_seed=2, image=i)
        ref, u = O.sample(p8, h, w, (0, 0, h, w), 1, 2, i)
        dec = decided_mask(p8, u, 1)
        n, bad = compare_levels(lev[i], ref, dec)
        if head == N.HT_HEAD_SIGMOID:
            assert unexplained(lev[i], ref, probs[i][0], p8[0], u, dec) == 0
        tot_n += n
        tot_bad += bad
        errs.append(np.abs(probs[i] - px).ravel())
        dq.append((probs[i] - p8).ravel())
    e = np.concatenate(errs)
    dq = np.concatenate(dq)
    print(f"FP8 head={head}: |dp| vs FP64 max {e.max():.3e} p99.9 {np.quantile(e, 0.999):.3e}; "
          f"vs quant 2 median {np.median(np.abs(dq)):.2e} p99.9 {np.quantile(np.abs(dq), 0.999):.2e}; "
          f"bit mismatches {tot_bad}/{tot_n}")
    if head == N.HT_HEAD_SIGMOID:
        fails = tight_rule(dq, "e4m3", 7)
        assert fails == [], fails
        assert tot_bad <= max(2, 1e-3 * tot_n), (tot_bad, tot_n)
    else:
        assert np.median(np.abs(dq)) <= 1e-6
        assert tot_bad <= max(3, 3e-3 * tot_n), (tot_bad, tot_n)
    assert e.max() < 0.15 and np.quantile(e, 0.999) < 0.1 and np.median(e) < 0.03
    if head == N.HT_HEAD_SOFTMAX:
        assert all(set(np.unique(l)) <= {0, 1, 2, 3} for l in lev)


@pytest.mark.parametrize("mode", [0, 1])
def test_bf16_softmax_head(mode):
    chs = synth.NET_WIDE_K4
    ws, bs = synth.he_normal_policy(chs, 3)
    pol = api.Policy(chs, ws, bs, head=N.HT_HEAD_SOFTMAX, precision=N.HT_BF16)
    imgs = [synth.contone_image(50, 140, seed=4)]
    lev, probs = _run(pol, imgs, mode, seed=4)
    _, pq, _ = O.forward(imgs[0], ws, bs, noise_seed=4, quant=1)
    _, px, _ = O.forward(imgs[0], ws, bs, noise_seed=4)
    ref, u = O.sample(pq, 50, 140, (0, 0, 50, 140), mode, 4, 0)
    n, bad = compare_levels(lev[0], ref, decided_mask(pq, u, mode))
    assert bad <= max(1, 3e-3 * n)
    assert np.abs(probs[0] - px).max() < 6e-3


def test_library_calibration_matches_oracle_scales():
    """ht_policy_calibrate (FP32 forward + per-layer abs-max, power-of-two scales) gives the
    same halftone as scales derived with the oracle on the same calibration image."""
    chs = synth.NET_WIDE
    ws, _ = synth.he_normal_policy(chs, 2)
    bs = synth.random_biases(chs, 5)
    sc = calibrate(ws, bs, chs)
    a = api.Policy(chs, ws, bs, precision=N.HT_FP8_E4M3)
    a.set_act_scales(sc)
    b = api.Policy(chs, ws, bs, precision=N.HT_FP8_E4M3)
    b.calibrate(torch.from_numpy(synth.contone_image(64, 64, seed=99)).cuda(), seed=99)
    imgs = [synth.contone_image(40, 140, seed=6)]
    la, _ = _run(a, imgs, 1, seed=3)
    lb, _ = _run(b, imgs, 1, seed=3)
    np.testing.assert_array_equal(la[0], lb[0])
