"""Pins of the oracle's hand-written backward: central finite differences and torch autograd."""
import numpy as np
import torch
import torch.nn.functional as F

import oracle as O
from paper_2304_12152_gb300 import synth


def _setup():
    chs = (2, 4, 4, 1)
    c = synth.contone_image(10, 9, seed=11)
    ws, _ = synth.he_normal_policy(chs, seed=12)
    bs = synth.random_biases(chs, seed=13, scale=0.2)
    rng = np.random.default_rng(8)
    dprob = rng.normal(size=(10, 9))
    return chs, c, ws, bs, dprob


def test_backward_matches_finite_differences():
    chs, c, ws, bs, dprob = _setup()
    lg, pr, acts = O.forward(c, ws, bs, noise_seed=3, image=1, save_acts=True)
    gw, gb = O.backward(c, ws, bs, 3, 1, acts, lg, dprob)

    def loss(wl, bl):
        _, p, _ = O.forward(c, wl, bl, noise_seed=3, image=1)
        return float(np.sum(p[0] * dprob))

    eps = 1e-4
    rng = np.random.default_rng(9)
    for l in range(3):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in ws[l].shape)
            wp = [w.astype(np.float64).copy() for w in ws]
            # perturb in float32 storage: use a representable step
            w32p = [w.copy() for w in ws]; w32m = [w.copy() for w in ws]
            w32p[l][idx] += np.float32(eps); w32m[l][idx] -= np.float32(eps)
            step = float(w32p[l][idx]) - float(w32m[l][idx])
            fd = (loss(w32p, bs) - loss(w32m, bs)) / step
            assert abs(fd - gw[l][idx]) < 2e-5 * max(1.0, abs(fd)), (l, idx, fd, gw[l][idx])
        b32p = [b.copy() for b in bs]; b32m = [b.copy() for b in bs]
        b32p[l][0] += np.float32(eps); b32m[l][0] -= np.float32(eps)
        step = float(b32p[l][0]) - float(b32m[l][0])
        fd = (loss(ws, b32p) - loss(ws, b32m)) / step
        assert abs(fd - gb[l][0]) < 2e-5 * max(1.0, abs(fd))


def test_backward_matches_torch_autograd():
    chs, c, ws, bs, dprob = _setup()
    lg, pr, acts = O.forward(c, ws, bs, noise_seed=3, image=1, save_acts=True)
    gw, gb = O.backward(c, ws, bs, 3, 1, acts, lg, dprob)
    z = O.uniform_map(3, 1, 0, 10, 9)
    x = torch.from_numpy(np.stack([c.astype(np.float64), z]))[None]
    tw = [torch.from_numpy(w.astype(np.float64)).requires_grad_() for w in ws]
    tb = [torch.from_numpy(b.astype(np.float64)).requires_grad_() for b in bs]
    for l in range(3):
        x = F.conv2d(x, tw[l], tb[l], padding=1)
        if l < 2:
            x = torch.relu(x)
    p = torch.sigmoid(x)[0, 0]
    (p * torch.from_numpy(dprob)).sum().backward()
    for l in range(3):
        np.testing.assert_allclose(gw[l], tw[l].grad.numpy(), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(gb[l], tb[l].grad.numpy(), rtol=1e-10, atol=1e-12)


def _bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


class _RoundAct(torch.autograd.Function):
    """Forward: round to bf16 (the stored activation); backward: identity."""

    @staticmethod
    def forward(ctx, x):
        return _bf16(x)

    @staticmethod
    def backward(ctx, g):
        return g


class _RoundGrad(torch.autograd.Function):
    """Forward: identity; backward: round the incoming gradient to bf16."""

    @staticmethod
    def forward(ctx, x):
        return x.clone()

    @staticmethod
    def backward(ctx, g):
        return _bf16(g)


def test_bf16_form_backward_matches_torch_rounding_model():
    """quant 1 backward vs torch autograd with the same rounding points written as
    autograd functions: bf16 weights for inner layers (forward and data gradient),
    bf16 activations, bf16 pre-activation gradients of every hidden layer."""
    chs = (2, 6, 5, 4, 1)
    c = synth.contone_image(11, 13, seed=41)
    ws, _ = synth.he_normal_policy(chs, seed=42)
    bs = synth.random_biases(chs, seed=43, scale=0.2)
    dprob = np.random.default_rng(44).normal(size=(11, 13))
    lg, pr, acts = O.forward(c, ws, bs, noise_seed=5, image=2, quant=1, save_acts=True)
    gw, gb = O.backward(c, ws, bs, 5, 2, acts, lg, dprob, quant=1)
    z = O.uniform_map(5, 2, 0, 11, 13)
    x = torch.from_numpy(np.stack([c.astype(np.float64), z]))[None]
    tw = [torch.from_numpy(w.astype(np.float64)).requires_grad_() for w in ws]
    tb = [torch.from_numpy(b.astype(np.float64)).requires_grad_() for b in bs]
    L = len(ws)
    for l in range(L):
        inner = 0 < l < L - 1
        # straight-through rounding of the weight: the gradient reaches the master weight
        wl = tw[l] + (_bf16(tw[l].detach()) - tw[l].detach()) if inner else tw[l]
        x = F.conv2d(x, wl, tb[l], padding=1)
        if l < L - 1:
            x = _RoundAct.apply(torch.relu(_RoundGrad.apply(x)))
    p = torch.sigmoid(x)[0, 0]
    np.testing.assert_allclose(p.detach().numpy(), pr[0], rtol=1e-12, atol=1e-14)
    (p * torch.from_numpy(dprob)).sum().backward()
    for l in range(L):
        np.testing.assert_allclose(gw[l], tw[l].grad.numpy(), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(gb[l], tb[l].grad.numpy(), rtol=1e-9, atol=1e-12)
    # the rounding points matter: the plain backward on the same activations differs
    gw0, _ = O.backward(c, ws, bs, 5, 2, acts, lg, dprob, quant=0)
    assert max(np.abs(gw0[l] - gw[l]).max() for l in range(L)) > 1e-6
