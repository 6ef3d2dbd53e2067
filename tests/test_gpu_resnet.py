"""GPU parity of the residual policy (Sec. VI-A: 16 blocks of 32 channels) in the BF16
tensor-core form against the oracle's residual forward with the same rounding points."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _policy(seed, nb=synth.RESNET_BLOCKS, head=N.HT_HEAD_SIGMOID, levels=4):
    ws, _ = synth.resnet_policy(nb, synth.RESNET_WIDTH, seed)
    bs = synth.random_biases(synth.resnet_channels(nb, synth.RESNET_WIDTH), seed + 1, scale=0.05)
    pol = api.Policy(synth.resnet_channels(nb, synth.RESNET_WIDTH), ws, bs, head=head, precision=N.HT_BF16,
                     levels=levels, arch=N.HT_ARCH_RESNET)
    return pol, ws, bs


@pytest.mark.parametrize("shape,mode", [((70, 200), N.HT_MODE_BERNOULLI), ((33, 129), N.HT_MODE_THRESHOLD)])
def test_resnet_bf16_matches_bf16_oracle(shape, mode):
    """34 layers (stem, 16 blocks, output).  Against the BF16-emulating oracle the GPU's p
    differs by about as much as BF16 rounding moves p at all: FP32-vs-FP64 accumulation
    flips early bf16 roundings, and through the undamped residual stream the two sides
    become independent BF16 realisations.  Bound, from the oracle alone: the p99.9 and max
    of |p_gpu - p_q1| within 1.5x those of |p_q1 - p_fp64|.  Actions: a decided pixel can
    only flip if the GPU's p moves across u, so the mismatches are bounded by the decided
    pixels whose margin |p - u| lies inside that band (1.5x the p99.9 BF16 effect)."""
    H, W = shape
    pol, ws, bs = _policy(41)
    img = synth.contone_image(H, W, seed=42)
    bits, probs = pol.halftone([torch.from_numpy(img).cuda()], mode=mode, seed=3, want_prob=True)
    torch.cuda.synchronize()
    lev = api.unpack_bits(bits[0], H, W)
    _, p = O.forward_resnet(img, ws, bs, 3, 0, quant=1)
    _, p64 = O.forward_resnet(img, ws, bs, 3, 0, quant=0)
    dp = np.abs(probs[0][0].cpu().numpy() - p)
    eff = np.abs(p - p64)
    print("resnet bf16 |dp| p99.9 %.2e max %.2e; bf16 effect p99.9 %.2e max %.2e"
          % (np.quantile(dp, 0.999), dp.max(), np.quantile(eff, 0.999), eff.max()))
    assert np.quantile(dp, 0.999) <= 1.5 * np.quantile(eff, 0.999) and dp.max() <= 1.5 * eff.max()
    u = O.uniform_map(3, 0, 1, H, W) if mode == N.HT_MODE_BERNOULLI else np.full((H, W), 0.5)
    ref = (u < p) if mode == N.HT_MODE_BERNOULLI else (p > 0.5)
    dec = np.abs(p - u) > 1e-4
    mism = int(((lev == 1) != ref)[dec].sum())
    band = int((dec & (np.abs(p - u) < 1.5 * np.quantile(eff, 0.999))).sum())
    print("resnet mismatches %d of %d decided, %d inside the BF16 band" % (mism, int(dec.sum()), band))
    assert mism <= max(2, band), (mism, band)


def test_resnet_batch_and_plan_match_single_calls():
    """Two images of different sizes in one call, and the same call as a CUDA-graph plan,
    give the bits of the single-image calls."""
    pol, _, _ = _policy(51, nb=3)
    imgs = [torch.from_numpy(synth.contone_image(h, w, seed=52, index=i)).cuda()
            for i, (h, w) in enumerate([(40, 300), (131, 77)])]
    both, _ = pol.halftone(imgs, mode=N.HT_MODE_BERNOULLI, seed=4)
    bits = [torch.zeros_like(b) for b in both]
    plan = api.Plan(pol, imgs, bits, N.HT_MODE_BERNOULLI, 4)
    plan.launch()
    torch.cuda.synchronize()
    for a, b in zip(bits, both):
        assert torch.equal(a, b)
    # single-image calls: image index 0 each, so compare image 0 only
    one, _ = pol.halftone(imgs[:1], mode=N.HT_MODE_BERNOULLI, seed=4)
    torch.cuda.synchronize()
    assert torch.equal(one[0], both[0])


def test_resnet_refuses_other_precisions():
    ws, bs = synth.resnet_policy(2, 32, 1)
    with pytest.raises(N.HTError):
        api.Policy(synth.resnet_channels(2, 32), ws, bs, precision=N.HT_FP32, arch=N.HT_ARCH_RESNET)
