"""Pins of the oracle's residual policy (Sec. VI-A: 16 residual blocks of 32 channels;
here smaller depths where the check is the same)."""
import numpy as np
import torch
import torch.nn.functional as F

import oracle as O
from paper_2304_12152_gb300 import synth


def _torch_resnet(c, z, ws, bs, bf16=False):
    r = (lambda t: t.to(torch.bfloat16).to(torch.float64)) if bf16 else (lambda t: t)
    x = torch.from_numpy(np.stack([c.astype(np.float64), z]))[None]
    tw = [torch.from_numpy(w.astype(np.float64)) for w in ws]
    tb = [torch.from_numpy(b.astype(np.float64)) for b in bs]
    nb = (len(ws) - 2) // 2
    x = r(torch.relu(F.conv2d(x, tw[0], tb[0], padding=1)))
    for b in range(nb):
        t = r(torch.relu(F.conv2d(x, r(tw[1 + 2 * b]), tb[1 + 2 * b], padding=1)))
        x = r(torch.relu(x + F.conv2d(t, r(tw[2 + 2 * b]), tb[2 + 2 * b], padding=1)))
    lg = F.conv2d(x, tw[-1], tb[-1], padding=1)[0, 0]
    return lg.numpy(), torch.sigmoid(lg).numpy()


def test_resnet_forward_matches_torch():
    ws, _ = synth.resnet_policy(3, 8, seed=1)
    bs = synth.random_biases(synth.resnet_channels(3, 8), seed=2, scale=0.1)
    c = synth.contone_image(13, 17, seed=3)
    z = O.uniform_map(4, 1, 0, 13, 17)
    lg, p = O.forward_resnet(c, ws, bs, 4, 1)
    tl, tp = _torch_resnet(c, z, ws, bs)
    np.testing.assert_allclose(lg, tl, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(p, tp, rtol=1e-11, atol=1e-14)


def test_resnet_bf16_rounding_points_match_torch():
    ws, _ = synth.resnet_policy(2, 8, seed=5)
    bs = synth.random_biases(synth.resnet_channels(2, 8), seed=6, scale=0.1)
    c = synth.contone_image(11, 12, seed=7)
    z = O.uniform_map(8, 0, 0, 11, 12)
    lg, _ = O.forward_resnet(c, ws, bs, 8, 0, quant=1)
    tl, _ = _torch_resnet(c, z, ws, bs, bf16=True)
    np.testing.assert_allclose(lg, tl, rtol=1e-9, atol=1e-12)
    lg0, _ = O.forward_resnet(c, ws, bs, 8, 0, quant=0)
    assert np.abs(lg - lg0).max() > 1e-6                  # the rounding points matter


def test_resnet_with_silent_branches_is_the_plain_two_layer_net():
    """conv2 of every block zero (weights and bias): y = ReLU(x + 0) = x for x >= 0, so the
    net reduces to stem + output layer, computed by the plain forward."""
    ws, bs = synth.resnet_policy(4, 8, seed=9)
    bs = synth.random_biases(synth.resnet_channels(4, 8), seed=10, scale=0.1)
    for b in range(4):
        ws[2 + 2 * b][:] = 0
        bs[2 + 2 * b][:] = 0
    c = synth.contone_image(15, 14, seed=11)
    lg, p = O.forward_resnet(c, ws, bs, 12, 3)
    lg2, p2, _ = O.forward(c, [ws[0], ws[-1]], [bs[0], bs[-1]], noise_seed=12, image=3)
    np.testing.assert_allclose(lg, lg2[0], rtol=1e-12, atol=1e-14)


def test_resnet_parameter_count_near_the_paper():
    """16 blocks of 32 channels + stem + output: 296 833 parameters (the paper states 299K)."""
    ws, bs = synth.resnet_policy(16, 32, seed=0)
    n = sum(w.size for w in ws) + sum(b.size for b in bs)
    assert n == 296833 and abs(n - 299e3) / 299e3 < 0.01


def test_resnet_region_equals_the_whole_image_slice():
    """A region is computed on the rectangle grown by the receptive field, with the noise
    at image coordinates: it equals the slice of the whole-image result."""
    ws, _ = synth.resnet_policy(2, 8, seed=13)
    bs = synth.random_biases(synth.resnet_channels(2, 8), seed=14, scale=0.1)
    c = synth.contone_image(40, 37, seed=15)
    lg, _ = O.forward_resnet(c, ws, bs, 16, 2)
    for reg in [(10, 9, 12, 15), (0, 0, 5, 37), (30, 20, 10, 17)]:
        y0, x0, rh, rw = reg
        lr, _ = O.forward_resnet(c, ws, bs, 16, 2, region=reg)
        np.testing.assert_allclose(lr, lg[y0:y0 + rh, x0:x0 + rw], rtol=1e-12, atol=1e-14)
