"""Tight parity of the tensor-core kernels on shallow 64-wide policies (BF16, FP16, FP8).

2 -> 64 -> 64 -> 1 runs layer 1 and the last hidden layer with the fused head partials;
2 -> 64 -> 64 -> 64 -> 1 adds a plain hidden 64 -> 64 layer.  Against the oracle emulating
the form's rounding points (bf16: quant 1) the rule is tests/_cases.TIGHT: the typical
pixel agrees to float32 rounding (median |dp| <= 1e-6), only a small fraction differs by
more than 1e-6, and the tail stays within what float32 accumulation produces on the same
policy (the bounds of the float32 model, tests/test_parity_model.py).  Actions: equal on
every pixel the oracle decides by more than 1e-4, none excepted.  Shapes span ragged
128-pixel column tiles, partial 8-row units and a single pixel; biases are non-zero."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

from _cases import compare_levels, decided_mask, tight_rule
from _rounding_model import fp8_scales

pytestmark = pytest.mark.gpu

SHAPES = [(67, 261), (24, 130), (9, 128), (1, 1)]
SHALLOW = [(2, 64, 64, 1), (2, 64, 64, 64, 1)]


def _check(chs, prec, quant, fmt, mode, seed):
    ws, bs = synth.he_normal_policy(chs, seed)
    bs = synth.random_biases(chs, seed + 1)
    pol = api.Policy(chs, ws, bs, precision=prec)
    sc = None
    if prec == N.HT_FP8_E4M3:
        sc = fp8_scales(ws, bs, chs)
        pol.set_act_scales(sc)
    imgs = [synth.contone_image(h, w, seed=seed, index=i) for i, (h, w) in enumerate(SHAPES)]
    cs = [torch.from_numpy(c).cuda() for c in imgs]
    bits, probs = pol.halftone(cs, mode=mode, seed=seed, want_prob=True)
    api.sync()
    diffs, tot_n, tot_bad = [], 0, 0
    for i, c in enumerate(imgs):
        h, w = c.shape
        _, p_q, _ = O.forward(c, ws, bs, noise_seed=seed, image=i, quant=quant, act_scale=sc)
        lev_q, u = O.sample(p_q, h, w, (0, 0, h, w), mode, seed, i)
        diffs.append((probs[i].cpu().numpy().astype(np.float64) - p_q).ravel())
        n, bad = compare_levels(api.unpack_bits(bits[i], h, w), lev_q, decided_mask(p_q, u, mode))
        tot_n += n
        tot_bad += bad
    fails = tight_rule(np.concatenate(diffs), fmt, len(chs) - 2)
    assert fails == [], fails
    assert tot_bad == 0, (tot_bad, tot_n)


@pytest.mark.parametrize("chs", SHALLOW)
@pytest.mark.parametrize("mode", [0, 1])
def test_bf16_shallow_tight(chs, mode):
    _check(chs, N.HT_BF16, 1, "bf16", mode, seed=21)


@pytest.mark.parametrize("chs", SHALLOW)
@pytest.mark.parametrize("mode", [0, 1])
def test_fp16_shallow_tight(chs, mode):
    """FP16 form (binary16 weights and activations) against the binary16-emulating oracle
    (quant 3): the same rule, whose FP16 rows bound the 99.9th percentile of |dp| at 1e-4
    (two rounded layers) and 2e-4 (three)."""
    _check(chs, N.HT_FP16, 3, "fp16", mode, seed=23)


@pytest.mark.parametrize("chs", SHALLOW)
@pytest.mark.parametrize("mode", [0, 1])
def test_fp8_shallow_tight(chs, mode):
    """FP8 E4M3 form (per-output-channel weight scales, power-of-two input scales from the
    calibration image) against the e4m3-emulating oracle (quant 2): the e4m3 rows."""
    _check(chs, N.HT_FP8_E4M3, 2, "e4m3", mode, seed=25)
