"""GPU parity of the FP16 tensor-core form (IEEE binary16 inner-layer weights and hidden
activations, FP32 accumulation, layer 1 to float32 accuracy, float32 head weights).

Against the oracle emulating those rounding points (quant 3): the tight rule of
tests/_cases.TIGHT for the policy's depth (7 rounded layers: 99.9% within 5e-4, all within
8e-4 -- binary16 flips near rounding boundaries are 8 times more frequent than bf16 ones and
8 times smaller, so over seven layers they reach most pixels but stay small); actions equal
on every decided pixel (|p - u| > 1e-4) but at most 2e-4 of them.  Against the pure FP64
oracle: max |dp| <= 2e-3, the precision target of the reduced-precision forms (binary16
storage of this policy moves p by up to ~7e-4; bfloat16 storage by up to ~4e-3, which is
why the BF16 form cannot meet it)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

from _cases import compare_levels, decided_mask, tight_rule, unexplained

pytestmark = pytest.mark.gpu

FP64_MAX = 2e-3


def _run(pol, imgs, mode, seed):
    cs = [torch.from_numpy(c).cuda() for c in imgs]
    bits, probs = pol.halftone(cs, mode=mode, seed=seed, want_prob=True)
    api.sync()
    lev = [api.unpack_bits(b, c.shape[0], c.shape[1], pol.head) for b, c in zip(bits, imgs)]
    return lev, [p.cpu().numpy().astype(np.float64) for p in probs]


@pytest.mark.parametrize("mode", [0, 1])
def test_fp16_wide_net_tiles_and_tails(mode):
    chs = synth.NET_WIDE
    ws, _ = synth.he_normal_policy(chs, 1)
    bs = synth.random_biases(chs, 2)
    pol = api.Policy(chs, ws, bs, precision=N.HT_FP16)
    shapes = [(96, 200), (67, 261), (5, 129), (1, 1)]
    imgs = [synth.contone_image(h, w, seed=1, index=i) for i, (h, w) in enumerate(shapes)]
    lev, probs = _run(pol, imgs, mode, seed=1)
    dq, dx, tot_n, tot_bad = [], [], 0, 0
    for i, c in enumerate(imgs):
        h, w = c.shape
        _, p_q, _ = O.forward(c, ws, bs, noise_seed=1, image=i, quant=3)
        _, p_x, _ = O.forward(c, ws, bs, noise_seed=1, image=i)
        ref, u = O.sample(p_q, h, w, (0, 0, h, w), mode, 1, i)
        dq.append((probs[i] - p_q).ravel())
        dx.append(np.abs(probs[i] - p_x).ravel())
        dec = decided_mask(p_q, u, mode)
        n, bad = compare_levels(lev[i], ref, dec)
        assert unexplained(lev[i], ref, probs[i][0], p_q[0], u, dec) == 0
        tot_n += n
        tot_bad += bad
    fails = tight_rule(np.concatenate(dq), "fp16", 7)
    assert fails == [], fails
    ex = np.concatenate(dx)
    print(f"FP16 vs FP64: max {ex.max():.3e} p99.9 {np.quantile(ex, 0.999):.3e}; mismatches {tot_bad}/{tot_n}")
    assert ex.max() <= FP64_MAX
    assert tot_bad <= max(2, 2e-4 * tot_n), (tot_bad, tot_n)


def test_fp16_full_size_sampled():
    """8 x 2048x2048 in one call (the printer workload's launch configuration, Bernoulli
    seed 1); corners and an interior crop of every image against the oracle evaluated on the
    crop with its halo, both the binary16-emulating and the pure FP64 one; a CUDA-graph plan
    of the same call gives the same bits."""
    chs = synth.NET_WIDE
    ws, bs = synth.he_normal_policy(chs, 1)
    pol = api.Policy(chs, ws, bs, precision=N.HT_FP16)
    imgs = [synth.contone_image(2048, 2048, seed=1, index=i) for i in range(8)]
    lev, probs = _run(pol, imgs, 1, seed=1)
    rng = np.random.default_rng(0)
    dq, dx, tot_n, tot_bad = [], [], 0, 0
    for i in range(8):
        y, x = rng.integers(32, 2048 - 64, size=2)
        regions = [(0, 0, 24, 24), (2048 - 24, 2048 - 40, 24, 40), (int(y), int(x), 24, 24)]
        for reg in regions:
            y0, x0, rh, rw = reg
            _, p_q, _ = O.forward(imgs[i], ws, bs, noise_seed=1, image=i, quant=3, region=reg)
            _, p_x, _ = O.forward(imgs[i], ws, bs, noise_seed=1, image=i, region=reg)
            lev_q, u = O.sample(p_q, 2048, 2048, reg, 1, 1, i)
            pg = probs[i][:, y0:y0 + rh, x0:x0 + rw]
            dq.append((pg - p_q).ravel())
            dx.append(np.abs(pg - p_x).ravel())
            n, bad = compare_levels(lev[i][y0:y0 + rh, x0:x0 + rw], lev_q, decided_mask(p_q, u, 1))
            tot_n += n
            tot_bad += bad
    fails = tight_rule(np.concatenate(dq), "fp16", 7)
    assert fails == [], fails
    assert np.concatenate(dx).max() <= FP64_MAX
    assert tot_bad <= max(2, 2e-4 * tot_n), (tot_bad, tot_n)
    cs = [torch.from_numpy(c).cuda() for c in imgs]
    bits = [pol.alloc_bits(2048, 2048) for _ in imgs]
    plan = api.Plan(pol, cs, bits, 1, 1)
    plan.launch()
    api.sync()
    for i in range(8):
        assert np.array_equal(api.unpack_bits(bits[i], 2048, 2048), lev[i]), i


@pytest.mark.parametrize("mode", [0, 1])
def test_fp16_softmax_head(mode):
    """4-logit softmax head in the FP16 form (weights as binary16 hi + lo parts of w x 2^k):
    three decision boundaries per pixel, residual mismatches at most 3e-3 of the decided
    pixels against quant 3; probabilities within the FP64 target."""
    chs = synth.NET_WIDE_K4
    ws, _ = synth.he_normal_policy(chs, 3)
    bs = synth.random_biases(chs, 4)
    pol = api.Policy(chs, ws, bs, head=N.HT_HEAD_SOFTMAX, precision=N.HT_FP16)
    imgs = [synth.contone_image(50, 140, seed=4)]
    lev, probs = _run(pol, imgs, mode, seed=4)
    _, pq, _ = O.forward(imgs[0], ws, bs, noise_seed=4, quant=3)
    _, px, _ = O.forward(imgs[0], ws, bs, noise_seed=4)
    ref, u = O.sample(pq, 50, 140, (0, 0, 50, 140), mode, 4, 0)
    n, bad = compare_levels(lev[0], ref, decided_mask(pq, u, mode))
    assert bad <= max(1, 3e-3 * n)
    assert np.abs(probs[0] - px).max() <= FP64_MAX
    assert set(np.unique(lev[0])) <= {0, 1, 2, 3}


def test_fp16_is_an_inference_form():
    chs = (2, 64, 64, 1)
    ws, bs = synth.he_normal_policy(chs, 5)
    pol = api.Policy(chs, ws, bs, precision=N.HT_FP16)
    with pytest.raises(N.HTError) as e:
        api.Trainer(pol, (32, 32), max_crops=1, n_samples=1)
    assert e.value.status == N.HT_ERR_UNSUPPORTED
