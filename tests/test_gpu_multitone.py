"""GPU parity of the multitoning prototype head (Sec. VI-E) against the oracle.

The level decision uses k = floor(v (L - 1)) and the fraction above it; pixels are
compared where the oracle's decision is unambiguous (|frac - u| > 1e-4 and v (L - 1)
more than 1e-4 away from an integer), the rule of the binary head."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

from _cases import tight_rule

pytestmark = pytest.mark.gpu


def _decided(v, L, u):
    t = v * (L - 1)
    k, frac = O.multitone_pair(v, L)
    return (np.abs(frac - u) > 1e-4) & (np.abs(t - np.rint(t)) > 1e-4)


@pytest.mark.parametrize("L,mode", [(4, N.HT_MODE_BERNOULLI), (3, N.HT_MODE_BERNOULLI), (4, N.HT_MODE_THRESHOLD)])
def test_fp32_multitone_head_matches_oracle(L, mode):
    chs = synth.NET_SMALL
    ws, bs = synth.he_normal_policy(chs, 31)
    pol = api.Policy(chs, ws, bs, head=N.HT_HEAD_MULTITONE, precision=N.HT_FP32, levels=L)
    H, W = 45, 70
    img = synth.contone_image(H, W, seed=32)
    bits, probs = pol.halftone([torch.from_numpy(img).cuda()], mode=mode, seed=5, want_prob=True)
    torch.cuda.synchronize()
    lev = api.unpack_bits(bits[0], H, W, N.HT_HEAD_MULTITONE)
    _, p, _ = O.forward(img, ws, bs, noise_seed=5)
    v = p[0]
    u = O.uniform_map(5, 0, 1, H, W) if mode == N.HT_MODE_BERNOULLI else np.full((H, W), 0.5)
    ref = O.sample_multitone(v, L, u if mode == N.HT_MODE_BERNOULLI else None)
    dec = _decided(v, L, u)
    assert dec.mean() > 0.99
    assert np.array_equal(lev[dec], ref[dec])
    assert lev.max() <= L - 1
    assert np.abs(probs[0][0].cpu().numpy() - v).max() < 2e-5


@pytest.mark.parametrize("H,W", [(60, 150), (37, 200)])
def test_bf16_multitone_head_matches_bf16_oracle(H, W):
    """Tensor-core form, 8-layer 64-wide net, 4 levels, Bernoulli: vs the BF16-emulating
    oracle.  v is held to the 7-layer bf16 row of the tight rule (tests/_cases.TIGHT), as
    the binary head's p.  Residual mismatches come from activations at bf16 rounding
    boundaries; the level rule compares v (L - 1) - k with u, so a decision can move only
    where the oracle's margin (|frac - u|, or the distance of v (L - 1) from a level) is
    within (L - 1) |dv| of the measured dv at that pixel: every mismatch must be explained
    so, and there are at most (L - 1) x 1e-3 of the decided pixels.  Widths 150 (pixels
    read one by one) and 200 (a multiple of 4: four pixels per lane from one Philox call,
    and a ragged second 128-pixel tile)."""
    chs = synth.NET_WIDE
    ws, bs = synth.he_normal_policy(chs, 33)
    L = 4
    pol = api.Policy(chs, ws, bs, head=N.HT_HEAD_MULTITONE, precision=N.HT_BF16, levels=L)
    img = synth.contone_image(H, W, seed=34)
    bits, probs = pol.halftone([torch.from_numpy(img).cuda()], mode=N.HT_MODE_BERNOULLI, seed=6, want_prob=True)
    torch.cuda.synchronize()
    lev = api.unpack_bits(bits[0], H, W, N.HT_HEAD_MULTITONE)
    _, p, _ = O.forward(img, ws, bs, noise_seed=6, quant=1)
    v = p[0]
    u = O.uniform_map(6, 0, 1, H, W)
    ref = O.sample_multitone(v, L, u)
    dec = _decided(v, L, u)
    mism = int((lev[dec] != ref[dec]).sum())
    assert mism <= max(2, int((L - 1) * 1e-3 * dec.sum())), (mism, int(dec.sum()))
    dv = probs[0][0].cpu().numpy() - v
    t = v * (L - 1)
    _, frac = O.multitone_pair(v, L)
    band = (L - 1) * np.abs(dv) + 1e-6
    explained = (np.abs(frac - u) <= band) | (np.abs(t - np.rint(t)) <= band)
    assert not np.any(dec & (lev != ref) & ~explained)
    fails = tight_rule(dv, "bf16", 7)
    assert fails == [], fails
    # levels are the two around v
    v32 = probs[0][0].cpu().numpy()
    k = np.minimum(np.floor(v32 * np.float32(L - 1)), L - 2).astype(np.int64)   # the kernel's FP32 rule
    assert np.all((lev == k) | (lev == k + 1))
