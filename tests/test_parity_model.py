"""The tight parity rule (tests/_cases.py TIGHT) against the float32 models of the reduced-
precision forms (tests/_rounding_model.py): a policy evaluated with float32 accumulation and
the oracle's rounding points satisfies the rule at every tabulated depth, with sums rounded
to nearest and (shallow policies) with the truncating tensor-core model the rows follow;
the same policy with layer 1 computed from two-part bf16 splits (products hi*hi + hi*lo +
lo*hi, relative error ~2^-16) breaks the shallow rows.  So the rule is one any
float32-accumulating kernel can meet, and it detects a layer-1 error of that size."""
import numpy as np
import pytest

import oracle as O
from paper_2304_12152_gb300 import synth

import _rounding_model as M
from _cases import tight_rule

CASES = [("bf16", (2, 64, 64, 1), True), ("bf16", (2, 64, 64, 64, 1), True), ("bf16", synth.NET_WIDE, True),
         ("fp16", (2, 64, 64, 1), True), ("fp16", (2, 64, 64, 64, 1), False), ("fp16", synth.NET_WIDE, False)]


@pytest.mark.parametrize("fmt,chs,split_fails", CASES)
def test_float32_model_meets_the_rule_and_a_split_layer_one_does_not(fmt, chs, split_fails):
    seed = 7
    ws, bs = synth.he_normal_policy(chs, seed)
    bs = synth.random_biases(chs, seed + 1)
    h, w = (112, 144) if len(chs) > 5 else (144, 176)
    img = synth.contone_image(h, w, seed=seed)
    _, p_or, _ = O.forward(img, ws, bs, noise_seed=seed, quant=1 if fmt == "bf16" else 3)
    stages = len(chs) - 2
    p32 = M.forward_p(img, ws, bs, seed, fmt=fmt, first="fp32")
    assert tight_rule(p32 - p_or[0], fmt, stages) == []
    if split_fails:
        p2 = M.forward_p(img, ws, bs, seed, fmt=fmt, first="split2")
        fails = tight_rule(p2 - p_or[0], fmt, stages)
        assert any(f.startswith("median") or f.startswith("frac") for f in fails), fails


def test_rule_picks_the_next_tabulated_depth():
    d = np.full(10000, 5e-7)
    assert tight_rule(d, "bf16", 5) == []           # read against the 7-layer row
    d[0] = 1.0
    assert tight_rule(d, "bf16", 2) == ["max 1 > 0.0015"]


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_truncating_model_meets_the_shallow_row(fmt):
    """The conservative truncating model (22 kept bits) on a two-layer policy: inside the row."""
    chs = (2, 64, 64, 1)
    ws, bs = synth.he_normal_policy(chs, 9)
    bs = synth.random_biases(chs, 10)
    img = synth.contone_image(96, 128, seed=9)
    _, p_or, _ = O.forward(img, ws, bs, noise_seed=9, quant=1 if fmt == "bf16" else 3)
    pt = M.forward_p(img, ws, bs, 9, fmt=fmt, acc="trunc", kept=22)
    assert tight_rule(pt - p_or[0], fmt, 2) == []


@pytest.mark.parametrize("chs", [(2, 64, 64, 1), (2, 64, 64, 64, 1), synth.NET_WIDE])
def test_e4m3_model_meets_the_rule(chs):
    """The FP8 form's float32 model (e4m3 codes of weights and inputs, float32 sums of code
    products times the scales) against quant 2 of the oracle."""
    seed = 25
    ws, bs = synth.he_normal_policy(chs, seed)
    bs = synth.random_biases(chs, seed + 1)
    sc = M.fp8_scales(ws, bs, chs)
    h, w = (112, 144) if len(chs) > 5 else (144, 176)
    img = synth.contone_image(h, w, seed=seed)
    _, p_or, _ = O.forward(img, ws, bs, noise_seed=seed, quant=2, act_scale=sc)
    p8 = M.forward_p(img, ws, bs, seed, fmt="e4m3", act_scale=sc)
    assert tight_rule(p8 - p_or[0], "e4m3", len(chs) - 2) == []


@pytest.mark.parametrize("nb", [1, 2, 16])
def test_residual_model_meets_the_rule(nb):
    """The residual policy's float32 model (round-to-nearest sums) against the oracle's
    residual forward with the BF16 rounding points."""
    seed = 43
    ws, _ = synth.resnet_policy(nb, synth.RESNET_WIDTH, seed)
    bs = synth.random_biases(synth.resnet_channels(nb, synth.RESNET_WIDTH), seed + 1, scale=0.05)
    img = synth.contone_image(96, 160, seed=seed)
    _, p_or = O.forward_resnet(img, ws, bs, 3, 0, quant=1)
    pm = M.forward_resnet_p(img, ws, bs, 3, 0)
    assert tight_rule(pm - p_or, "bf16-res", nb) == []
