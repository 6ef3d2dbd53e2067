"""GPU parity of the residual policy (Sec. VI-A: 16 blocks of 32 channels) in the BF16
tensor-core form against the oracle's residual forward with the same rounding points."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

from _cases import tight_rule, unexplained

pytestmark = pytest.mark.gpu


def _policy(seed, nb=synth.RESNET_BLOCKS, head=N.HT_HEAD_SIGMOID, levels=4):
    ws, _ = synth.resnet_policy(nb, synth.RESNET_WIDTH, seed)
    bs = synth.random_biases(synth.resnet_channels(nb, synth.RESNET_WIDTH), seed + 1, scale=0.05)
    pol = api.Policy(synth.resnet_channels(nb, synth.RESNET_WIDTH), ws, bs, head=head, precision=N.HT_BF16,
                     levels=levels, arch=N.HT_ARCH_RESNET)
    return pol, ws, bs


@pytest.mark.parametrize("nb", [1, 2])
@pytest.mark.parametrize("mode", [N.HT_MODE_BERNOULLI, N.HT_MODE_THRESHOLD])
def test_resnet_shallow_tight(nb, mode):
    """One and two residual blocks (the stem, the 32-wide block kernels with the in-place
    shortcut add, the last block's fused head partials) on ragged shapes against the
    BF16-emulating oracle: the bf16-res rows of the tight rule (tests/_cases.TIGHT), and no
    action mismatch on a decided pixel."""
    seed = 41 + nb
    pol, ws, bs = _policy(seed, nb=nb)
    shapes = [(67, 261), (24, 130), (9, 128)]
    imgs = [synth.contone_image(h, w, seed=seed, index=i) for i, (h, w) in enumerate(shapes)]
    bits, probs = pol.halftone([torch.from_numpy(c).cuda() for c in imgs], mode=mode, seed=3, want_prob=True)
    torch.cuda.synchronize()
    d, tot_bad = [], 0
    for i, c in enumerate(imgs):
        h, w = c.shape
        _, p = O.forward_resnet(c, ws, bs, 3, i, quant=1)
        pg = probs[i][0].cpu().numpy().astype(np.float64)
        d.append((pg - p).ravel())
        u = O.uniform_map(3, i, 1, h, w) if mode == N.HT_MODE_BERNOULLI else np.full((h, w), 0.5)
        ref = (u < p) if mode == N.HT_MODE_BERNOULLI else (p > 0.5)
        dec = np.abs(p - u) > 1e-4
        tot_bad += int(((api.unpack_bits(bits[i], h, w) == 1) != ref)[dec].sum())
    fails = tight_rule(np.concatenate(d), "bf16-res", nb)
    assert fails == [], fails
    assert tot_bad == 0


@pytest.mark.parametrize("shape,mode", [((70, 200), N.HT_MODE_BERNOULLI), ((33, 129), N.HT_MODE_THRESHOLD)])
def test_resnet_bf16_matches_bf16_oracle(shape, mode):
    """The paper's 34 layers (stem, 16 blocks, output).  Against the BF16-emulating oracle
    the bf16-res row for 16 blocks: FP32-vs-FP64 accumulation flips early bf16 roundings, and
    through the undamped residual stream the two sides become independent BF16
    realisations (the float32 models of the same policy differ from the oracle as much).
    Actions: every mismatch on a decided pixel lies within the measured |dp| of u (their
    number then depends only on how many decided pixels lie that close: the outputs of this
    policy crowd around p = 1/2)."""
    H, W = shape
    pol, ws, bs = _policy(41)
    img = synth.contone_image(H, W, seed=42)
    bits, probs = pol.halftone([torch.from_numpy(img).cuda()], mode=mode, seed=3, want_prob=True)
    torch.cuda.synchronize()
    lev = api.unpack_bits(bits[0], H, W)
    _, p = O.forward_resnet(img, ws, bs, 3, 0, quant=1)
    pg = probs[0][0].cpu().numpy().astype(np.float64)
    fails = tight_rule(pg - p, "bf16-res", 16)
    assert fails == [], fails
    u = O.uniform_map(3, 0, 1, H, W) if mode == N.HT_MODE_BERNOULLI else np.full((H, W), 0.5)
    ref = ((u < p) if mode == N.HT_MODE_BERNOULLI else (p > 0.5)).astype(np.uint8)
    dec = np.abs(p - u) > 1e-4
    assert unexplained(lev, ref, pg, p, u, dec) == 0
    mism = int((lev != ref)[dec].sum())
    band = int((dec & (np.abs(p - u) <= np.abs(pg - p) + 1e-6)).sum())
    print("resnet mismatches %d of %d decided, %d decided pixels within |dp| of u" % (mism, int(dec.sum()), band))


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
