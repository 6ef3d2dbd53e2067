"""Finite-difference check of the library's own training step on the GPU (Algorithm 1,
TRAIN; Eq. marl with the local-expectation estimator Eq. le; Eq. as).

The library's forward reports its losses as FP64 sums; its backward returns dL/dW.  Here
single weights and biases of an FP32 policy are moved through ht_policy_set_weights, the
library's loss is evaluated again, and central differences of it are compared with the
library's gradient -- no oracle involved, the library against itself.

L_MARL depends on the weights through p and, where a Bernoulli sample changes, through the
rewards (a jump, not a slope: the estimator's gradient holds the samples fixed).  The step
eps = 1e-4 moves p by ~1e-5, so that a sample changes only where u lies within ~1e-5 of p;
the difference quotients at eps and 2 eps must agree, which also catches the rare case
where one did change (such a weight is skipped; most must remain).  Agreement: 5e-3 of
the larger of |dL/dw| and 5% of the largest gradient entry, beyond the quotients' own
spread |fd(eps) - fd(2 eps)|, which estimates their error.  L_AS alone (a gray patch, no
sampling) has no sample jumps, but its float32 spectrum leaves ~1e-6 of noise in the loss
and single hidden parameters move many pre-activations across ReLU kinks, so it is
checked along random directions and on the output layer's parameters."""
import numpy as np
import pytest
import torch

from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

pytestmark = pytest.mark.gpu

CHS = (2, 8, 8, 1)


def _flat(ws, bs):
    return (torch.from_numpy(np.concatenate([w.ravel() for w in ws]).astype(np.float32)).cuda(),
            torch.from_numpy(np.concatenate([b.ravel() for b in bs]).astype(np.float32)).cuda())


def _picks(n_w, n_b, rng):
    """A few weights of every layer and a few biases: (is_bias, flat index)."""
    offs = np.cumsum([0] + [CHS[i] * CHS[i + 1] * 9 for i in range(len(CHS) - 1)])
    out = [(False, int(rng.integers(offs[l], offs[l + 1]))) for l in range(len(CHS) - 1) for _ in range(3)]
    out += [(True, int(rng.integers(0, n_b))) for _ in range(3)]
    return out


def _loss(pol, tr, w, b, crops, levels, seed, k):
    pol.set_weights(w, b)
    return tr.forward(crops, levels, seed)[k]


def _fd_check(pol, tr, w0, b0, crops, levels, seed, k, eps, consistency):
    gw, gb = tr.backward()
    gw, gb = gw.clone().cpu().numpy(), gb.clone().cpu().numpy()
    rng = np.random.default_rng(5)
    checked, worst = 0, 0.0
    scale = max(np.abs(gw).max(), np.abs(gb).max())
    for is_b, i in _picks(w0.numel(), b0.numel(), rng):
        def at(d):
            w, b = w0.clone(), b0.clone()
            (b if is_b else w)[i] += d
            return _loss(pol, tr, w, b, crops, levels, seed, k)
        fd1 = (at(eps) - at(-eps)) / (2 * eps)
        fd2 = (at(2 * eps) - at(-2 * eps)) / (4 * eps)
        g = float((gb if is_b else gw)[i])
        if abs(fd1 - fd2) > consistency * max(abs(fd1), 5e-2 * scale):
            continue                                  # a sample changed inside the stencil
        checked += 1
        # the difference quotients' own spread |fd1 - fd2| estimates their error
        err = max(0.0, abs(fd1 - g) - abs(fd1 - fd2)) / max(abs(g), 5e-2 * scale)
        worst = max(worst, err)
        assert err <= 5e-3, (is_b, i, fd1, fd2, g)
    pol.set_weights(w0, b0)
    return checked, worst


def test_marl_gradient_matches_central_differences():
    ws, _ = synth.he_normal_policy(CHS, 61)
    bs = synth.random_biases(CHS, 62, scale=0.1)
    crops = [torch.from_numpy(synth.contone_image(32, 32, seed=63, index=i)).cuda() for i in range(2)]
    pol = api.Policy(CHS, ws, bs, precision=N.HT_FP32)
    tr = api.Trainer(pol, (32, 32), max_crops=2, n_samples=2, n_gray=0, las_mode=1, n_rad=4, n_ang=4, w_a=0.0)
    w0, b0 = _flat(ws, bs)
    tr.forward(crops, [], 11)
    checked, worst = _fd_check(pol, tr, w0, b0, crops, [], 11, 1, 1e-4, 2e-2)
    print(f"L_MARL: {checked} of 12 weights checked, worst relative error {worst:.2e}")
    assert checked >= 8


def test_anisotropy_gradient_matches_central_differences():
    """w_a L_AS alone on one 32 x 32 constant-gray patch (binned form, 4 x 4 bins).  A single
    hidden weight moved by eps shifts many pre-activations across a ReLU kink at once, so
    the gradient is checked along three random directions over all parameters (directional
    derivative, eps = 1e-3: 1e-2 relative beyond the quotients' spread) and on single
    output-layer parameters, where the loss is smooth (eps = 1e-2, the rule above)."""
    ws, _ = synth.he_normal_policy(CHS, 64)
    bs = synth.random_biases(CHS, 65, scale=0.1)
    pol = api.Policy(CHS, ws, bs, precision=N.HT_FP32)
    tr = api.Trainer(pol, (32, 32), max_crops=1, n_samples=1, n_gray=1, gray_n=32, las_mode=1, n_rad=4, n_ang=4,
                     w_a=1.0)
    w0, b0 = _flat(ws, bs)
    tr.forward([], [0.3], 12)
    gw, gb = tr.backward()
    g = np.concatenate([gw.clone().cpu().numpy(), gb.clone().cpu().numpy()]).astype(np.float64)
    nw = w0.numel()
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = rng.standard_normal(g.size)
        v /= np.linalg.norm(v)
        vw = torch.from_numpy(v[:nw].astype(np.float32)).cuda()
        vb = torch.from_numpy(v[nw:].astype(np.float32)).cuda()

        def at(d):
            return _loss(pol, tr, w0 + d * vw, b0 + d * vb, [], [0.3], 12, 2)
        eps = 1e-3
        fd1 = (at(eps) - at(-eps)) / (2 * eps)
        fd2 = (at(2 * eps) - at(-2 * eps)) / (4 * eps)
        gv = float(g @ v)
        print(f"L_AS direction: fd {fd1:.6e} / {fd2:.6e}, g.v {gv:.6e}")
        assert abs(fd1 - gv) <= 1e-2 * abs(gv) + abs(fd1 - fd2), (fd1, fd2, gv)
    pol.set_weights(w0, b0)
    # single parameters of the output layer (no ReLU after it)
    last_w = sum(CHS[i] * CHS[i + 1] * 9 for i in range(len(CHS) - 2))
    for is_b, i in [(False, last_w + 3), (False, last_w + 40), (False, nw - 1), (True, sum(CHS[1:]) - 1)]:
        def at1(d):
            w, b = w0.clone(), b0.clone()
            (b if is_b else w)[i] += d
            return _loss(pol, tr, w, b, [], [0.3], 12, 2)
        eps = 1e-2
        fd1 = (at1(eps) - at1(-eps)) / (2 * eps)
        fd2 = (at1(2 * eps) - at1(-2 * eps)) / (4 * eps)
        gi = float(g[nw + i] if is_b else g[i])
        scale = float(np.abs(g).max())
        err = max(0.0, abs(fd1 - gi) - abs(fd1 - fd2)) / max(abs(gi), 5e-2 * scale)
        print(f"L_AS output-layer {'bias' if is_b else 'weight'} {i}: fd {fd1:.6e} / {fd2:.6e}, g {gi:.6e}")
        assert err <= 5e-3, (is_b, i, fd1, fd2, gi)
    pol.set_weights(w0, b0)
