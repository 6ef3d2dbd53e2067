"""Full-size parity in the benchmark's launch configurations, on sampled outputs.

The FP8 4-level multitone workload (4 x 4096^2, 8-layer 64-wide policy with the 4-logit
softmax head, e4m3 weights and activations, Bernoulli seed 2) and the uneven batch (64
generator images of log-uniform sizes between 200 x 300 and 4096 x 3072, BF16, Bernoulli
seed 4) run in one call each, as the benchmark runs them; corners and interior crops of
the images are compared with the FP64 oracle evaluated on the crop with its halo (the
policy is fully convolutional and the noise is keyed by the global pixel index, so a
crop's outputs are exact functions of the crop plus an L-pixel halo).  Rules as in the
small-size tests: e4m3 form (4-logit head) against the e4m3-emulating oracle, median |dq|
at float32 rounding (<= 1e-6) and mismatched actions at most 3e-3 of the decided pixels;
BF16 form against the BF16-emulating oracle, the 7-layer bf16 row of the tight rule
(tests/_cases.TIGHT) and mismatches at most 2e-4 of the decided pixels.  The training
step's losses, which the oracle computes whole, are checked at the benchmark's size too."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

from _cases import compare_levels, decided_mask, tight_rule

pytestmark = pytest.mark.gpu

CROP = 24


def _regions(h, w, rng, interior=1):
    regs = [(0, 0, min(CROP, h), min(CROP, w)), (max(h - CROP, 0), max(w - 40, 0), min(CROP, h), min(40, w))]
    for _ in range(interior):
        if h > 3 * CROP and w > 3 * CROP:
            y, x = rng.integers(CROP, h - 2 * CROP), rng.integers(CROP, w - 2 * CROP)
            regs.append((int(y), int(x), CROP, CROP))
    return regs


def _oracle_scales(ws, bs, chs, calib):
    """Per-layer e4m3 input scales from an FP64 oracle pass over the calibration image
    (abs-max, rounded up to a power of two): what ht_policy_calibrate derives."""
    _, _, acts = O.forward(calib, ws, bs, noise_seed=99, save_acts=True)
    L = len(chs) - 1
    sc = [1.0] * L
    for l in range(1, L - 1):
        amax = float(np.abs(acts[l - 1]).max())
        sc[l] = 2.0 ** math.ceil(math.log2(max(amax, 1e-6) / 448.0))
    return sc


def test_multitone_fp8_full_size_sampled():
    chs = synth.NET_WIDE_K4
    ws, bs = synth.he_normal_policy(chs, 1)
    calib = synth.contone_image(256, 256, seed=99)
    sc = _oracle_scales(ws, bs, chs, calib)
    pol = api.Policy(chs, ws, bs, head=N.HT_HEAD_SOFTMAX, precision=N.HT_FP8_E4M3, levels=4)
    pol.set_act_scales(sc)
    imgs = [synth.contone_image(4096, 4096, seed=2, index=i) for i in range(4)]
    cs = [torch.from_numpy(c).cuda() for c in imgs]
    bits, probs = pol.halftone(cs, mode=N.HT_MODE_BERNOULLI, seed=2, want_prob=True)
    # the benchmark calibrates inside the library on the same image: same halftone
    pol_b = api.Policy(chs, ws, bs, head=N.HT_HEAD_SOFTMAX, precision=N.HT_FP8_E4M3, levels=4)
    pol_b.calibrate(torch.from_numpy(calib).cuda(), seed=99)
    bits_b, _ = pol_b.halftone(cs, mode=N.HT_MODE_BERNOULLI, seed=2)
    api.sync()
    rng = np.random.default_rng(1)
    tot_n = tot_bad = 0
    dq = []
    for i in range(4):
        assert torch.equal(bits[i], bits_b[i]), i
        lev = api.unpack_bits(bits[i], 4096, 4096, N.HT_HEAD_SOFTMAX)
        for reg in _regions(4096, 4096, rng):
            y0, x0, rh, rw = reg
            _, p8, _ = O.forward(imgs[i], ws, bs, noise_seed=2, image=i, quant=2, act_scale=sc, region=reg)
            ref, u = O.sample(p8, 4096, 4096, reg, N.HT_MODE_BERNOULLI, 2, i)
            pg = probs[i][:, y0:y0 + rh, x0:x0 + rw].cpu().numpy().astype(np.float64)
            assert pg.shape == p8.shape
            dq.append(np.abs(pg - p8).ravel())
            n, bad = compare_levels(lev[y0:y0 + rh, x0:x0 + rw], ref, decided_mask(p8, u, N.HT_MODE_BERNOULLI))
            tot_n += n
            tot_bad += bad
            assert set(np.unique(lev[y0:y0 + rh, x0:x0 + rw])) <= {0, 1, 2, 3}
    assert tot_n > 0.9 * 4 * 3 * CROP * CROP
    assert np.median(np.concatenate(dq)) <= 1e-6
    assert tot_bad <= max(3, 3e-3 * tot_n), (tot_bad, tot_n)


def test_uneven_batch_full_size_sampled():
    chs = synth.NET_WIDE
    ws, bs = synth.he_normal_policy(chs, 1)
    pol = api.Policy(chs, ws, bs, precision=N.HT_BF16)
    shapes = synth.uneven_shapes(64, seed=4)
    imgs = [synth.contone_image(h, w, seed=4, index=i) for i, (h, w) in enumerate(shapes)]
    cs = [torch.from_numpy(c).cuda() for c in imgs]
    bits = [pol.alloc_bits(h, w) for h, w in shapes]
    probs = [torch.empty((1, h, w), dtype=torch.float32, device="cuda") for h, w in shapes]
    pol.autotune(cs, bits, N.HT_MODE_BERNOULLI, 4, probs, reps=1)     # the benchmark's schedule choice
    pol.halftone_into(cs, bits, N.HT_MODE_BERNOULLI, 4, probs)
    api.sync()
    rng = np.random.default_rng(2)
    tot_n = tot_bad = 0
    diffs = []
    for i in range(0, 64, 7):
        h, w = shapes[i]
        lev = api.unpack_bits(bits[i], h, w)
        for reg in _regions(h, w, rng):
            y0, x0, rh, rw = reg
            _, pq, _ = O.forward(imgs[i], ws, bs, noise_seed=4, image=i, quant=1, region=reg)
            ref, u = O.sample(pq, h, w, reg, N.HT_MODE_BERNOULLI, 4, i)
            pg = probs[i][:, y0:y0 + rh, x0:x0 + rw].cpu().numpy().astype(np.float64)
            diffs.append((pg - pq).ravel())
            n, bad = compare_levels(lev[y0:y0 + rh, x0:x0 + rw], ref, decided_mask(pq, u, N.HT_MODE_BERNOULLI))
            tot_n += n
            tot_bad += bad
    fails = tight_rule(np.concatenate(diffs), "bf16", 7)
    assert fails == [], fails
    assert tot_bad <= max(2, 2e-4 * tot_n), (tot_bad, tot_n)


def test_training_step_full_size_losses():
    """The benchmark's training step (16 generator crops of 256^2, 4 constant-gray patches
    {0.1, 0.25, 0.5, 0.75} of 256^2, S = 4 Bernoulli samples, LE estimator, 32 x 16-bin
    anisotropy loss, w_a = 0.002, BF16 form): its losses against the BF16-emulating oracle
    computed whole (forward, samples, rewards and toggle deltas of all 64 crop-samples,
    anisotropy loss of the gray patches).  As in the small BF16 step test the two sides'
    samples differ wherever |p - u| is below the forward's BF16 error, so the losses are held
    to 1e-3 relative."""
    chs = synth.NET_WIDE
    ws, bs = synth.he_normal_policy(chs, 3)
    crops = [synth.contone_image(256, 256, seed=3, index=i) for i in range(16)]
    levels = [0.1, 0.25, 0.5, 0.75]
    S, seed, w_a = 4, 1, 0.002
    pol = api.Policy(chs, ws, bs, precision=N.HT_BF16)
    tr = api.Trainer(pol, (256, 256), max_crops=16, n_samples=S, n_gray=4, gray_n=256, las_mode=1, n_rad=32,
                     n_ang=16, w_a=w_a)
    losses = tr.forward([torch.from_numpy(c).cuda() for c in crops], levels, seed)
    api.sync()
    n = len(crops)
    l_marl, rs = 0.0, []
    for i, c in enumerate(crops):
        _, p, _ = O.forward(c, ws, bs, noise_seed=seed, image=i, quant=1)
        for s in range(S):
            u = O.uniform_map(seed, i, 1 + s, 256, 256)
            hb = (u < p[0]).astype(np.uint8)
            r = O.reward(c, hb)
            dR = O.toggle_delta(c, hb).reshape(256, 256)
            val, _ = O.le_surrogate(p[0], hb, dR, r["R"])
            l_marl += val / (n * S)
            rs.append(r["R"])
    l_as = 0.0
    for g, lev in enumerate(levels):
        c = np.full((256, 256), lev, np.float32)
        _, p, _ = O.forward(c, ws, bs, noise_seed=seed, image=n + g, quant=1)
        l_as += O.anisotropy_loss(p[0], mode=1, n_rad=32, n_ang=16)["loss"] / len(levels)
    ref = (l_marl + w_a * l_as, l_marl, l_as, float(np.mean(rs)))
    print("losses", losses, "oracle", ref)
    for k in range(4):
        assert abs(losses[k] - ref[k]) <= 1e-3 * abs(ref[k]) + 1e-7, (k, losses, ref)
