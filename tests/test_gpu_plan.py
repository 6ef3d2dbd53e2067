"""CUDA-graph plans and the conv-schedule autotuner (tensor-core forms).

A plan replays the exact launch sequence of ht_halftone, and every schedule the
autotuner tries keeps each output pixel's accumulation order, so the outputs are
compared bit for bit: plan vs direct call, every schedule vs the default one."""
import numpy as np
import pytest
import torch

from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

pytestmark = pytest.mark.gpu

SHAPES = [(300, 200), (37, 515), (129, 131), (8, 9)]     # ragged tiles, partial units, a tiny image


def _batch(seed):
    return [torch.from_numpy(synth.contone_image(h, w, seed=seed, index=i)).cuda() for i, (h, w) in enumerate(SHAPES)]


def _policy(prec, chs=synth.NET_WIDE, seed=5):
    ws, bs = synth.he_normal_policy(chs, seed)
    return api.Policy(chs, ws, bs, precision=prec), ws, bs


@pytest.mark.parametrize("prec", [N.HT_BF16, N.HT_FP8_E4M3])
def test_plan_matches_direct_call(prec):
    pol, _, _ = _policy(prec)
    imgs = _batch(3)
    if prec == N.HT_FP8_E4M3:
        pol.calibrate(imgs[0], seed=9)
    ref, pref = pol.halftone(imgs, mode=N.HT_MODE_BERNOULLI, seed=7, want_prob=True)
    bits = [torch.zeros_like(b) for b in ref]
    probs = [torch.zeros_like(p) for p in pref]
    plan = api.Plan(pol, imgs, bits, N.HT_MODE_BERNOULLI, 7, probs)
    for _ in range(2):
        plan.launch()
    api.sync()
    for a, b in zip(bits, ref):
        assert torch.equal(a, b)
    for a, b in zip(probs, pref):
        assert torch.equal(a, b)


def test_plan_recaptures_after_weight_change():
    pol, ws, bs = _policy(N.HT_BF16)
    imgs = _batch(4)
    bits = [pol.alloc_bits(c.shape[0], c.shape[1]) for c in imgs]
    plan = api.Plan(pol, imgs, bits, N.HT_MODE_THRESHOLD, 1)
    plan.launch()
    ws2, bs2 = synth.he_normal_policy(synth.NET_WIDE, 6)
    w = torch.from_numpy(np.concatenate([x.ravel() for x in ws2])).cuda()
    b = torch.from_numpy(np.concatenate([x.ravel() for x in bs2])).cuda()
    pol.set_weights(w, b)
    plan.launch()                                  # new weights -> captured again
    ref, _ = pol.halftone(imgs, mode=N.HT_MODE_THRESHOLD, seed=1)
    api.sync()
    for a, r in zip(bits, ref):
        assert torch.equal(a, r)


def test_plan_refuses_fp32():
    pol, _, _ = _policy(N.HT_FP32, chs=synth.NET_SMALL)
    imgs = _batch(5)[:1]
    bits = [pol.alloc_bits(c.shape[0], c.shape[1]) for c in imgs]
    with pytest.raises(N.HTError):
        api.Plan(pol, imgs, bits, N.HT_MODE_THRESHOLD, 0)


def test_autotune_schedules_are_bit_identical():
    pol, _, _ = _policy(N.HT_BF16)
    imgs = _batch(6)
    ref, pref = pol.halftone(imgs, mode=N.HT_MODE_BERNOULLI, seed=2, want_prob=True)
    bits = [torch.zeros_like(b) for b in ref]
    probs = [torch.zeros_like(p) for p in pref]
    res = pol.autotune(imgs, bits, N.HT_MODE_BERNOULLI, 2, probs, reps=2)
    api.sync()
    assert len(res) == N.HT_TUNE_CANDIDATES
    assert sorted((r, o, pr) for r, o, pr, _ in res) == sorted(
        [(r, o, pr) for pr in (0, 1) for r in (8, 6, 4) for o in (0, 1)]
        + [(r, o, 0) for r in (32, 64, 128) for o in (0, 1)])
    assert all(ms > 0 for *_, ms in res)
    # the last candidate's outputs, and the chosen schedule's later calls, equal the default schedule's
    for a, b in zip(bits, ref):
        assert torch.equal(a, b)
    for a, b in zip(probs, pref):
        assert torch.equal(a, b)
    again, pagain = pol.halftone(imgs, mode=N.HT_MODE_BERNOULLI, seed=2, want_prob=True)
    api.sync()
    for a, b in zip(again, ref):
        assert torch.equal(a, b)
    for a, b in zip(pagain, pref):
        assert torch.equal(a, b)


def test_many_short_units_every_schedule():
    """Stress of the conv pipeline's per-block barriers: 160 images of 13 x 300 give
    CTAs long runs of units whose last row band is short (5 of 8 rows, and for rows per
    unit 6 / 4 other remainders), i.e. TMEM blocks left unused unit after unit; as
    streaming strips (9 rows and a 4-row rest, or the whole 13-row image) the TMEM ring
    continues across strips of odd height.  Every schedule must finish without a wait
    expiring and give the same bits."""
    pol, _, _ = _policy(N.HT_BF16)
    imgs = [torch.from_numpy(synth.contone_image(13, 300, seed=8, index=i)).cuda() for i in range(160)]
    bits = [pol.alloc_bits(13, 300) for _ in imgs]
    ref = None
    for ru, order, pair in [(8, 0, 0), (8, 1, 0), (6, 0, 0), (6, 1, 0), (4, 0, 0), (4, 1, 0), (3, 0, 0), (7, 1, 0),
                            (8, 0, 1), (8, 1, 1), (6, 0, 1), (4, 1, 1), (3, 0, 1), (7, 1, 1),
                            (9, 0, 0), (9, 1, 0), (13, 0, 0), (13, 1, 0), (64, 1, 0)]:
        pol.set_schedule(ru, order, pair)
        for _ in range(3):
            pol.halftone_into(imgs, bits, N.HT_MODE_BERNOULLI, 3)
            api.sync()
        if ref is None:
            ref = [b.clone() for b in bits]
        else:
            for a, b in zip(bits, ref):
                assert torch.equal(a, b), (ru, order, pair)
    pol.set_schedule(8, 0)


PAIR_SHAPES = [(300, 200), (37, 515), (129, 131), (8, 9), (1, 1), (5, 700), (70, 256), (17, 257)]


@pytest.mark.parametrize("prec,head", [(N.HT_BF16, N.HT_HEAD_SIGMOID), (N.HT_FP8_E4M3, N.HT_HEAD_SIGMOID),
                                       (N.HT_FP8_E4M3, N.HT_HEAD_SOFTMAX), (N.HT_BF16, N.HT_HEAD_MULTITONE)])
def test_cta_pair_form_matches_single_cta_form(prec, head):
    """The CTA-pair form of the 64 -> 64 layers (M = 256 MMAs over a 256-pixel tile,
    weights split by N between the two CTAs) accumulates every output pixel in the same
    order as the single-CTA form, so bits and probabilities are equal bit for bit, under
    every head that follows those layers (1-logit sigmoid, 4-logit softmax, multitoning
    prototype).  Widths leave the second CTA of a pair partly or wholly outside the
    image; heights leave short row bands."""
    chs = synth.NET_WIDE_K4 if head == N.HT_HEAD_SOFTMAX else synth.NET_WIDE
    ws, bs = synth.he_normal_policy(chs, 11)
    bs = synth.random_biases(chs, 3)
    pol = api.Policy(chs, ws, bs, head=head, precision=prec, levels=4)
    imgs = [torch.from_numpy(synth.contone_image(h, w, seed=12, index=i)).cuda() for i, (h, w) in enumerate(PAIR_SHAPES)]
    if prec == N.HT_FP8_E4M3:
        pol.calibrate(imgs[0], seed=9)
    for mode in (N.HT_MODE_THRESHOLD, N.HT_MODE_BERNOULLI):
        pol.set_schedule(8, 0, 0)
        ref, pref = pol.halftone(imgs, mode=mode, seed=4, want_prob=True)
        for ru, order in [(8, 0), (8, 1), (6, 1), (3, 0)]:
            pol.set_schedule(ru, order, 1)
            got, pgot = pol.halftone(imgs, mode=mode, seed=4, want_prob=True)
            api.sync()                     # also raises a device-side wait expiry
            for i, (a, b) in enumerate(zip(got, ref)):
                assert torch.equal(a, b), (mode, ru, order, PAIR_SHAPES[i])
            for i, (a, b) in enumerate(zip(pgot, pref)):
                assert torch.equal(a, b), (mode, ru, order, PAIR_SHAPES[i])
    # a plan captured with the pair form replays it
    pol.set_schedule(8, 0, 1)
    bits = [torch.zeros_like(b) for b in ref]
    plan = api.Plan(pol, imgs, bits, N.HT_MODE_BERNOULLI, 4)
    plan.launch()
    api.sync()
    for a, b in zip(bits, ref):
        assert torch.equal(a, b)
    pol.set_schedule(8, 0, 0)


STREAM_SHAPES = [(300, 200), (37, 515), (129, 131), (1, 1), (517, 140), (64, 256), (33, 129)]


@pytest.mark.parametrize("prec,head", [(N.HT_BF16, N.HT_HEAD_SIGMOID), (N.HT_FP8_E4M3, N.HT_HEAD_SIGMOID),
                                       (N.HT_FP16, N.HT_HEAD_SIGMOID), (N.HT_BF16, N.HT_HEAD_SOFTMAX),
                                       (N.HT_FP16, N.HT_HEAD_SOFTMAX), (N.HT_BF16, N.HT_HEAD_MULTITONE)])
def test_streaming_strips_match_row_units(prec, head):
    """Streaming strips (units of more than 8 rows, the eight TMEM blocks used as a ring,
    windows that pass the last block issued as two MMAs) accumulate every output pixel in
    one TMEM column through the same chain of MMAs as 8-row units, so bits and
    probabilities are equal bit for bit: every layer kind (layer 1, hidden, fused head
    partials, 4-logit head), strip heights that leave odd remainders and strips taller than
    the image, both unit orders; a plan captured with strips replays them."""
    chs = synth.NET_WIDE_K4 if head == N.HT_HEAD_SOFTMAX else synth.NET_WIDE
    ws, bs = synth.he_normal_policy(chs, 13)
    bs = synth.random_biases(chs, 14)
    pol = api.Policy(chs, ws, bs, head=head, precision=prec, levels=4)
    imgs = [torch.from_numpy(synth.contone_image(h, w, seed=15, index=i)).cuda()
            for i, (h, w) in enumerate(STREAM_SHAPES)]
    if prec == N.HT_FP8_E4M3:
        pol.calibrate(imgs[0], seed=9)
    for mode in (N.HT_MODE_THRESHOLD, N.HT_MODE_BERNOULLI):
        pol.set_schedule(8, 0, 0)
        ref, pref = pol.halftone(imgs, mode=mode, seed=6, want_prob=True)
        for ru, order in [(9, 0), (16, 1), (33, 0), (64, 1), (128, 0), (4096, 1)]:
            pol.set_schedule(ru, order, 0)
            got, pgot = pol.halftone(imgs, mode=mode, seed=6, want_prob=True)
            api.sync()                     # also raises a device-side wait expiry
            for i, (a, b) in enumerate(zip(got, ref)):
                assert torch.equal(a, b), (mode, ru, order, STREAM_SHAPES[i])
            for i, (a, b) in enumerate(zip(pgot, pref)):
                assert torch.equal(a, b), (mode, ru, order, STREAM_SHAPES[i])
    pol.set_schedule(64, 0, 0)
    bits = [torch.zeros_like(b) for b in ref]
    plan = api.Plan(pol, imgs, bits, N.HT_MODE_BERNOULLI, 6)
    plan.launch()
    api.sync()
    for a, b in zip(bits, ref):
        assert torch.equal(a, b)
    pol.set_schedule(8, 0, 0)


def test_streaming_strips_refused_for_the_residual_policy():
    chs = synth.resnet_channels(2, 32)
    ws, bs = synth.resnet_policy(2, 32, 3)
    pol = api.Policy(chs, ws, bs, precision=N.HT_BF16, arch=N.HT_ARCH_RESNET)
    with pytest.raises(N.HTError):
        pol.set_schedule(9, 0, 0)
    with pytest.raises(N.HTError):
        pol.set_schedule(4097, 0, 0)
    pol.set_schedule(8, 1, 0)
