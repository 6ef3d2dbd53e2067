"""Pins of the oracle's policy forward, sampling and quantisation emulation."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle as O
from paper_2304_12152_gb300 import synth


def _torch_forward(c, z, ws, bs):
    """Independent FP64 forward with torch's conv2d (a library primitive)."""
    x = torch.from_numpy(np.stack([c.astype(np.float64), z]))[None]
    for l, (w, b) in enumerate(zip(ws, bs)):
        x = F.conv2d(x, torch.from_numpy(w.astype(np.float64)), torch.from_numpy(b.astype(np.float64)), padding=1)
        if l < len(ws) - 1:
            x = torch.relu(x)
    return x[0].numpy()


@pytest.mark.parametrize("chs,hw", [((2, 4, 3, 1), (5, 5)), ((2, 8, 8, 1), (17, 23)), ((2, 6, 6, 4), (9, 12))])
def test_forward_matches_torch_conv_chain(chs, hw):
    h, w = hw
    c = synth.contone_image(h, w, seed=1)
    ws, _ = synth.he_normal_policy(chs, seed=2)
    bs = synth.random_biases(chs, seed=3)
    logits, probs, _ = O.forward(c, ws, bs, noise_seed=11, image=2)
    z = O.uniform_map(11, 2, 0, h, w)
    ref = _torch_forward(c, z, ws, bs)
    np.testing.assert_allclose(logits, ref, rtol=1e-12, atol=1e-12)
    if chs[-1] == 1:
        np.testing.assert_allclose(probs[0], 1 / (1 + np.exp(-ref[0])), rtol=1e-12)
    else:
        e = np.exp(ref - ref.max(0))
        np.testing.assert_allclose(probs, e / e.sum(0), rtol=1e-12)


def test_forward_hand_unrolled_tiny():
    # 1 hidden channel, 2 layers on a 3x3 image written out by hand
    c = np.arange(9, dtype=np.float32).reshape(3, 3) / 10
    w1 = np.zeros((1, 2, 3, 3), np.float32); w1[0, 0, 1, 1] = 1.0; w1[0, 0, 0, 0] = -0.5
    w2 = np.zeros((1, 1, 3, 3), np.float32); w2[0, 0, 1, 2] = 2.0
    b1 = np.array([0.1], np.float32); b2 = np.array([-0.3], np.float32)
    logits, _, _ = O.forward(c, [w1, w2], [b1, b2], noise_seed=0)
    cd = c.astype(np.float64)
    a = np.zeros((3, 3))
    for y in range(3):
        for x in range(3):
            v = 0.1 + cd[y, x]
            if y >= 1 and x >= 1:
                v += -0.5 * cd[y - 1, x - 1]
            a[y, x] = max(float(np.float32(0.1)) - 0.1 + v, 0.0)
    expect = np.full((3, 3), float(np.float32(-0.3)))
    for y in range(3):
        for x in range(2):
            expect[y, x] += 2.0 * a[y, x + 1]
    np.testing.assert_allclose(logits[0], expect, atol=1e-7)


def test_crop_equals_full_image():
    """Fully convolutional: any crop (with the halo handled inside) equals the same pixels
    of the whole-image evaluation, including at the image borders."""
    chs = (2, 6, 6, 6, 1)
    c = synth.contone_image(40, 37, seed=4)
    ws, bs = synth.he_normal_policy(chs, seed=5)
    full, _, _ = O.forward(c, ws, bs, noise_seed=9, image=1)
    for (y0, x0, rh, rw) in [(0, 0, 7, 9), (10, 12, 8, 5), (33, 30, 7, 7), (0, 20, 40, 3)]:
        part, _, _ = O.forward(c, ws, bs, noise_seed=9, image=1, region=(y0, x0, rh, rw))
        np.testing.assert_allclose(part[0], full[0, y0:y0 + rh, x0:x0 + rw], rtol=1e-13, atol=1e-13)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    # float32 subnormals too (bf16 keeps fp32's exponent range: subnormal spacing 2^-133)
    sub = np.array([3e-39, 1.1e-39, -7e-40, 2.0 ** -130, 1.5 * 2.0 ** -133, 2.5 * 2.0 ** -133, -5.5 * 2.0 ** -133])
    xs = np.concatenate([rng.normal(0, 1, 2000), rng.normal(0, 1e-3, 500), [1.00390625, 1.01171875, -3.0, 0.0], sub])
    ref = torch.from_numpy(xs.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([O.round_bf16(float(np.float32(x))) for x in xs])
    np.testing.assert_array_equal(got, ref)


def test_e4m3_rounding_matches_torch():
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.normal(0, 30, 2000), rng.normal(0, 0.01, 500), [448.0, 500.0, -1e4, 2 ** -9, 3 * 2 ** -10]])
    xs32 = xs.astype(np.float32)
    # torch's float8_e4m3fn cast is round-to-nearest-even; saturate first (torch does not saturate)
    ref = torch.from_numpy(np.clip(xs32, -448, 448)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = np.array([O.round_e4m3(float(x)) for x in xs32])
    np.testing.assert_array_equal(got, ref)


def test_fp8_form_forward_matches_torch_rounding_model():
    """The E4M3 form's rounding points, rebuilt from torch's float8_e4m3fn cast and an FP64
    conv2d chain: inner-layer weights per output channel scaled by amax / 448 and rounded;
    each inner layer's input activations divided by that layer's scale, rounded (saturating
    at +-448) and scaled back; every hidden ReLU output rounded to bf16; layer 1 and the head
    exact.  Nonzero biases, and scales small enough that some activations saturate."""
    chs = (2, 16, 16, 16, 1)
    c = synth.contone_image(18, 21, seed=4)
    ws, bs = synth.he_normal_policy(chs, seed=5)
    rng = np.random.default_rng(6)
    bs = [rng.normal(0, 0.1, b.shape).astype(np.float32) for b in bs]
    sc = [1.0, 1.0 / 448, 2.0 / 448, 1.0]
    lg8, _, _ = O.forward(c, ws, bs, noise_seed=3, quant=2, act_scale=sc)

    def e4m3(t):
        return t.clamp(-448, 448).to(torch.float8_e4m3fn).to(torch.float64)

    z = torch.from_numpy(O.uniform_map(3, 0, 0, *c.shape))
    x = torch.stack([torch.from_numpy(c.astype(np.float64)), z])[None]
    L = len(ws)
    saturated = 0
    for l in range(L):
        w = torch.from_numpy(ws[l].astype(np.float64))
        inner = 0 < l < L - 1
        if inner:
            s_o = w.abs().amax(dim=(1, 2, 3), keepdim=True) / 448.0
            w = e4m3((w / s_o).float()) * s_o
            saturated += int((x.abs() > 448 * sc[l]).sum())
            x = e4m3((x / sc[l]).float()) * sc[l]
        x = F.conv2d(x, w, torch.from_numpy(bs[l].astype(np.float64)), padding=1)
        if l < L - 1:
            x = x.clamp_min(0).float().to(torch.bfloat16).to(torch.float64)
    assert saturated > 0
    np.testing.assert_allclose(lg8[0], x[0, 0].numpy(), rtol=0, atol=1e-11)


def test_fp16_rounding_matches_torch():
    rng = np.random.default_rng(2)
    edge = [65504.0, 65519.0, 65520.0, 1e5, -7e4, 2.0 ** -14, 2.0 ** -24, 3 * 2.0 ** -25, 2.0 ** -26,
            1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, -2049.0, 0.0]
    xs = np.concatenate([rng.normal(0, 1, 2000), rng.normal(0, 1e-5, 500), rng.normal(0, 3e4, 200), edge])
    xs32 = xs.astype(np.float32)
    ref = torch.from_numpy(xs32).to(torch.float16).to(torch.float64).numpy()
    got = np.array([O.round_fp16(float(x)) for x in xs32])
    np.testing.assert_array_equal(got, ref)


def test_fp16_form_forward_matches_torch_rounding_model():
    """quant 3 (FP16 form): inner-layer weights rounded to IEEE binary16, every hidden ReLU
    output rounded to binary16, layer 1 and the head weights exact -- rebuilt from torch's
    float16 cast and an FP64 conv2d chain."""
    chs = (2, 16, 16, 16, 1)
    c = synth.contone_image(17, 22, seed=8)
    ws, bs = synth.he_normal_policy(chs, seed=9)
    rng = np.random.default_rng(10)
    bs = [rng.normal(0, 0.1, b.shape).astype(np.float32) for b in bs]
    lg16, _, _ = O.forward(c, ws, bs, noise_seed=4, quant=3)

    def f16(t):
        # one rounding from float64 (numpy converts double to half directly); going through
        # float32 first would round twice and can land on a binary16 tie
        return torch.from_numpy(t.numpy().astype(np.float16).astype(np.float64))

    z = torch.from_numpy(O.uniform_map(4, 0, 0, *c.shape))
    x = torch.stack([torch.from_numpy(c.astype(np.float64)), z])[None]
    L = len(ws)
    for l in range(L):
        w = torch.from_numpy(ws[l].astype(np.float64))
        if 0 < l < L - 1:
            w = f16(w)
        x = F.conv2d(x, w, torch.from_numpy(bs[l].astype(np.float64)), padding=1)
        if l < L - 1:
            x = f16(x.clamp_min(0))
    np.testing.assert_allclose(lg16[0], x[0, 0].numpy(), rtol=0, atol=1e-11)
    lg1, _, _ = O.forward(c, ws, bs, noise_seed=4, quant=1)
    lg0, _, _ = O.forward(c, ws, bs, noise_seed=4)
    assert np.abs(lg16 - lg0).max() < np.abs(lg1 - lg0).max()        # fp16 is the finer format


def test_quantised_forms_stay_close():
    chs = (2, 16, 16, 16, 1)
    c = synth.contone_image(20, 20, seed=6)
    ws, bs = synth.he_normal_policy(chs, seed=7)
    _, p, _ = O.forward(c, ws, bs, noise_seed=1)
    _, pb, _ = O.forward(c, ws, bs, noise_seed=1, quant=1)
    assert 0 < np.abs(pb - p).max() < 2e-2
    _, p8, _ = O.forward(c, ws, bs, noise_seed=1, quant=2, act_scale=[1.0, 4 / 448, 4 / 448, 1.0])
    assert 0 < np.abs(p8 - p).max() < 1e-1


def test_sampling_rules():
    h, w = 16, 16
    p = np.linspace(0, 1, h * w).reshape(1, h, w)
    p[0, 3, 3] = 0.5
    bits, u = O.sample(p, h, w, (0, 0, h, w), mode=0, seed=0)
    assert np.all(u == 0.5)                                  # threshold = the Bernoulli rule at u = 1/2
    assert set(np.unique(bits)) <= {0, 1}
    np.testing.assert_array_equal(bits, (p[0] > 0.5).astype(np.uint8))
    assert bits[3, 3] == 0                                   # tie p = 0.5 -> 0
    bits, u = O.sample(p, h, w, (0, 0, h, w), mode=1, seed=5)
    np.testing.assert_array_equal(u, O.uniform_map(5, 0, 1, h, w))
    np.testing.assert_array_equal(bits, (u < p[0]).astype(np.uint8))
    # Bernoulli frequencies follow p
    pp = np.full((1, 128, 128), 0.3)
    b, _ = O.sample(pp, 128, 128, (0, 0, 128, 128), 1, 9)
    assert abs(b.mean() - 0.3) < 5 * np.sqrt(0.21 / b.size)


def test_sampling_over_a_region_and_image_index():
    """A region's actions are the matching slice of the whole image's (the uniforms are
    keyed by the global pixel index), and the image index selects the Philox counter."""
    h, w = 23, 37
    rng = np.random.default_rng(8)
    p = rng.random((1, h, w))
    q4 = rng.dirichlet(np.ones(4), size=(h, w)).transpose(2, 0, 1).copy()
    for probs in (p, q4):
        full, uf = O.sample(probs, h, w, (0, 0, h, w), 1, 9, image=3)
        y0, x0, rh, rw = 5, 11, 9, 17
        part, up = O.sample(np.ascontiguousarray(probs[:, y0:y0 + rh, x0:x0 + rw]), h, w, (y0, x0, rh, rw), 1, 9, image=3)
        np.testing.assert_array_equal(part, full[y0:y0 + rh, x0:x0 + rw])
        np.testing.assert_array_equal(up, uf[y0:y0 + rh, x0:x0 + rw])
    np.testing.assert_array_equal(uf, O.uniform_map(9, 3, 1, h, w))
    assert not np.array_equal(uf, O.uniform_map(9, 0, 1, h, w))


def test_sampled_level_frequencies_follow_the_probabilities():
    """Sampling (Algorithm 1, TEST with stochastic actions; the K-level head of Sec. VI-E):
    over a 512 x 512 map with the same per-pixel distribution, the drawn level counts match
    the probabilities by a chi-square test (3 degrees of freedom, 99.99% quantile 21.1), and a
    binary map's fraction of ones matches p within 4.5 standard errors.  Independent of the
    inverse-CDF rule as written: a level-index shift or a reversed comparison fails it."""
    h = w = 512
    n = h * w
    q4 = np.array([0.1, 0.2, 0.3, 0.4])
    probs = np.broadcast_to(q4[:, None, None], (4, h, w)).copy()
    lev, _ = O.sample(probs, h, w, (0, 0, h, w), 1, 7)
    cnt = np.bincount(lev.ravel(), minlength=4)
    assert cnt.sum() == n
    chi2 = float((((cnt - n * q4) ** 2) / (n * q4)).sum())
    assert chi2 < 21.1, (cnt, chi2)
    for p in (0.05, 0.5, 0.8):
        pm = np.full((1, h, w), p)
        hb, _ = O.sample(pm, h, w, (0, 0, h, w), 1, 11)
        frac = hb.mean()
        assert abs(frac - p) < 4.5 * np.sqrt(p * (1 - p) / n), (p, frac)


def test_softmax_levels_sampling():
    K, h, w = 4, 64, 64
    rng = np.random.default_rng(3)
    lg = rng.normal(size=(K, h, w))
    q = np.exp(lg) / np.exp(lg).sum(0)
    lev, u = O.sample(q, h, w, (0, 0, h, w), 1, 2)
    cdf = np.cumsum(q, 0)
    ref = np.argmax(u[None] < cdf, axis=0)
    np.testing.assert_array_equal(lev, ref)
    lev0, _ = O.sample(q, h, w, (0, 0, h, w), 0, 2)
    np.testing.assert_array_equal(lev0, np.argmax(q, 0))
    # threshold mode on exact ties takes the lowest level index
    qt = np.array([[0.3, 0.3, 0.2, 0.2], [0.1, 0.4, 0.4, 0.1], [0.25, 0.25, 0.25, 0.25]]).T.reshape(4, 1, 3)
    lt, _ = O.sample(np.ascontiguousarray(qt), 1, 3, (0, 0, 1, 3), 0, 2)
    np.testing.assert_array_equal(lt[0], [0, 1, 0])
