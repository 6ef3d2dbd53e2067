"""GPU parity of the reward, toggle deltas and anisotropy loss against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _halftone(c, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(c.shape) < c).astype(np.uint8)


SHAPES = [(11, 11), (64, 64), (100, 37), (256, 256), (300, 257)]


def test_reward_matches_oracle():
    imgs = [synth.contone_image(h, w, seed=3, index=i) for i, (h, w) in enumerate(SHAPES)]
    hts = [_halftone(c, i) for i, c in enumerate(imgs)]
    cs = [torch.from_numpy(c).cuda() for c in imgs]
    bits = [torch.from_numpy(api.pack_bits(h)).cuda() for h in hts]
    out = api.reward(cs, bits).cpu().numpy()
    for i in range(len(imgs)):
        r = O.reward(imgs[i], hts[i])
        assert abs(out[i, 0] - r["mse"]) <= 1e-5 * r["mse"] + 1e-9, (SHAPES[i], out[i, 0], r["mse"])
        assert abs(out[i, 1] - r["ssim"]) < 2e-5
        assert abs(out[i, 2] - r["cssim"]) < 2e-5
        assert abs(out[i, 3] - r["R"]) < 2e-6


def test_reward_invariants_on_gpu():
    c = np.full((40, 50), 0.3, np.float32)
    hb = _halftone(c, 1)
    out = api.reward([torch.from_numpy(c).cuda()], [torch.from_numpy(api.pack_bits(hb)).cuda()]).cpu().numpy()
    assert abs(out[0, 2] - 1.0) < 1e-5                 # zero contrast -> CSSIM = 1
    b = (np.random.default_rng(2).random((33, 47)) < 0.5).astype(np.uint8)
    out = api.reward([torch.from_numpy(b.astype(np.float32)).cuda()],
                     [torch.from_numpy(api.pack_bits(b)).cuda()]).cpu().numpy()
    assert abs(out[0, 1] - 1.0) < 1e-5 and out[0, 0] < 1e-12   # SSIM(x, x) = 1, MSE 0


@pytest.mark.parametrize("shape", [(24, 24), (64, 96), (256, 256)])
def test_toggle_delta_matches_oracle(shape):
    h, w = shape
    c = synth.contone_image(h, w, seed=9)
    hb = _halftone(c, 5)
    dR = api.toggle_delta([torch.from_numpy(c).cuda()], [torch.from_numpy(api.pack_bits(hb)).cuda()])[0]
    g = dR.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(1)
    if h * w <= 4096:
        idx = np.arange(h * w)
    else:   # all four borders' rows/cols plus a random interior sample
        border = np.concatenate([np.arange(w), (h - 1) * w + np.arange(w), np.arange(h) * w, np.arange(h) * w + w - 1])
        idx = np.unique(np.concatenate([border, rng.integers(0, h * w, 1500)]))
    ref = O.toggle_delta(c, hb, idx)
    scale = np.abs(ref).max()
    err = np.abs(g.ravel()[idx] - ref)
    assert err.max() < 2e-4 * scale, (err.max(), scale)


@pytest.mark.parametrize("L", [3, 4])
def test_multilevel_reward_matches_oracle(L):
    """Reward of multi-level halftones (multitoning prototype, Sec. VI-E): SSIM needs
    E[h^2] != E[h]."""
    imgs = [synth.contone_image(h, w, seed=13, index=i) for i, (h, w) in enumerate(SHAPES)]
    rng = np.random.default_rng(L)
    levs = [O.sample_multitone(c.astype(np.float64), L, rng.random(c.shape)) for c in imgs]
    cs = [torch.from_numpy(c).cuda() for c in imgs]
    bits = [torch.from_numpy(api.pack_bits(h, N.HT_HEAD_MULTITONE)).cuda() for h in levs]
    out = api.reward(cs, bits, api.reward_opts(levels=L)).cpu().numpy()
    for i in range(len(imgs)):
        r = O.reward(imgs[i], levs[i], levels=L)
        assert abs(out[i, 0] - r["mse"]) <= 1e-5 * r["mse"] + 1e-9, (SHAPES[i], out[i, 0], r["mse"])
        assert abs(out[i, 1] - r["ssim"]) < 2e-5
        assert abs(out[i, 2] - r["cssim"]) < 2e-5
        assert abs(out[i, 3] - r["R"]) < 2e-6


@pytest.mark.parametrize("L,shape", [(3, (24, 24)), (4, (64, 96)), (4, (256, 256))])
def test_multilevel_toggle_delta_matches_oracle(L, shape):
    """dR_a = R(lo + 1) - R(lo) for the level pair around v_a, against the oracle."""
    h, w = shape
    c = synth.contone_image(h, w, seed=19)
    rng = np.random.default_rng(7)
    v = np.clip(c + 0.1 * rng.normal(size=c.shape), 0, 1).astype(np.float32)
    k, _ = O.multitone_pair(v.astype(np.float64), L)
    lev = O.sample_multitone(v.astype(np.float64), L, rng.random(c.shape))
    vt = torch.from_numpy(v).cuda()
    dR = api.toggle_delta([torch.from_numpy(c).cuda()],
                          [torch.from_numpy(api.pack_bits(lev, N.HT_HEAD_MULTITONE)).cuda()],
                          api.reward_opts(levels=L), v=[vt])[0]
    g = dR.cpu().numpy().astype(np.float64)
    # the kernel takes the level pair from v in FP32: compare where both sides agree on it
    k32 = np.minimum(np.floor(v * np.float32(L - 1)), L - 2).astype(np.int64)
    if h * w <= 4096:
        idx = np.arange(h * w)
    else:
        idx = np.unique(rng.integers(0, h * w, 1500))
    idx = idx[k32.ravel()[idx] == k.ravel()[idx]]
    ref = O.toggle_delta(c, lev, idx, levels=L, lo=k.astype(np.uint8))
    scale = np.abs(ref).max()
    err = np.abs(g.ravel()[idx] - ref)
    assert err.max() < 2e-4 * scale, (err.max(), scale)


@pytest.mark.parametrize("mode,n", [(0, 16), (0, 64), (1, 64), (1, 256)])
def test_anisotropy_matches_oracle(mode, n):
    rng = np.random.default_rng(n + mode)
    q = np.stack([rng.random((n, n)), np.clip(0.3 + 0.1 * rng.normal(size=(n, n)), 0, 1)]).astype(np.float32)
    loss, g = api.anisotropy_loss(torch.from_numpy(q).cuda(), mode=mode, n_rad=32 if n >= 64 else 4,
                                  n_ang=16 if n >= 64 else 4, grad=True)
    loss, g = loss.cpu().numpy(), g.cpu().numpy()
    for k in range(2):
        r = O.anisotropy_loss(q[k].astype(np.float64), mode=mode, n_rad=32 if n >= 64 else 4,
                              n_ang=16 if n >= 64 else 4, grad=True)
        assert abs(loss[k] - r["loss"]) <= 1e-4 * abs(r["loss"]) + 1e-12, (loss[k], r["loss"])
        assert np.abs(g[k] - r["grad"]).max() <= 1e-3 * np.abs(r["grad"]).max() + 1e-12
