"""A float32 model of the reduced-precision policy forms, for the parity rules only.

The rounding-emulating oracle (oracle.forward with quant 1 or 3) rounds every hidden
activation at the points the tensor-core kernels do, but accumulates in FP64.  A kernel
that accumulates in float32 therefore rounds an activation the other way whenever its exact
value lies within the float32 accumulation error of a rounding boundary (a "flip").  A flip
changes the sums that read that activation by one ulp of it, which can flip some of them in
turn, so the disagreement spreads from rare seeds, layer by layer.  How far it spreads is a
property of the arithmetic, not of any kernel, so the bounds of the tight parity rule
(_cases.tight_rule) are taken from this model: the same policy as plain PyTorch CPU float32
operators (im2col + float32 matrix products), with the same rounding points, compared with
the oracle.  It holds none of the library's code and none of its layouts.

first="fp32": layer 1 as a float32 convolution (what a kernel with float32-exact products
accumulating in float32 gives).  first="split2": layer 1 with its inputs and weights split
into two bf16 parts, and only the products hi*hi + hi*lo + lo*hi kept (relative error about
2^-16 per product), the form the tests use to show that the rule detects such an error.

acc="rn": the inner layers' sums as float32 matrix products (round to nearest).
acc="trunc": the inner layers' sums as a tensor core forms them in the model of Fasi,
Higham, Mikaitis and Pranesh ("Numerical behavior of NVIDIA tensor cores", PeerJ Computer
Science 7:e330, 2021): per block of 16 products (one MMA's K), the exact products and the
running float32 sum are aligned to the largest exponent among them, the bits below
`kept` positions under it are dropped (truncation), the aligned terms are added exactly
and the result is truncated to float32.  `kept` = 22 (two bits fewer than float32's 24)
is a conservative setting: on the shallow policies it predicts more rounding flips than
the GB300 kernels show.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F

import oracle as O


def _round(t: torch.Tensor, fmt: str) -> torch.Tensor:
    dt = {"bf16": torch.bfloat16, "fp16": torch.float16}[fmt]
    return t.to(dt).to(torch.float32)


def _e4m3(t: torch.Tensor) -> torch.Tensor:
    """E4M3 rounding (nearest even) with saturation at +-448, as float32."""
    return t.clamp(-448.0, 448.0).to(torch.float8_e4m3fn).to(torch.float32)


def _conv_f32(x: torch.Tensor, w: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """3x3 convolution, zero padding 1, as one float32 matrix product over im2col columns."""
    _, c, h, wd = x.shape
    cols = F.unfold(x, 3, padding=1)[0]                          # [c * 9, h * w]
    out = w.reshape(w.shape[0], -1) @ cols + b[:, None]
    return out.reshape(1, w.shape[0], h, wd)


def _trunc_f32(x: np.ndarray) -> np.ndarray:
    """Truncation (toward zero) of float64 values to float32's 24 significant bits."""
    _, e = np.frexp(x)
    q = np.ldexp(1.0, e - 24)
    return np.trunc(x / q) * q


def _conv_trunc(x: torch.Tensor, w: torch.Tensor, b: torch.Tensor, kept: int) -> torch.Tensor:
    """3x3 convolution, zero padding 1, summed as in the truncating tensor-core model: K in
    blocks of 16 in the kernel's order (kernel row, kernel column, input channel)."""
    _, c, h, wd = x.shape
    xp = F.pad(x, (1, 1, 1, 1))[0].double().numpy()
    cols = np.stack([xp[:, dy:dy + h, dx:dx + wd] for dy in range(3) for dx in range(3)])
    cols = cols.reshape(9 * c, h * wd)
    wm = w.double().numpy().transpose(0, 2, 3, 1).reshape(w.shape[0], 9 * c)
    acc = np.zeros((w.shape[0], h * wd))
    for k0 in range(0, 9 * c, 16):
        terms = np.concatenate([acc[:, None, :], wm[:, k0:k0 + 16, None] * cols[None, k0:k0 + 16, :]], 1)
        amax = np.abs(terms).max(1)
        _, e = np.frexp(np.where(amax > 0, amax, 1.0))
        q = np.ldexp(1.0, e - kept)[:, None, :]
        s = (np.trunc(terms / q) * q).sum(1)
        acc = np.where(s != 0, _trunc_f32(s), 0.0)
    y = torch.from_numpy(acc).float() + b[:, None]                  # epilogue bias add (float32)
    return y.reshape(1, w.shape[0], h, wd)


def forward_p(contone: np.ndarray, ws, bs, noise_seed: int, image: int = 0, fmt: str = "bf16",
              first: str = "fp32", acc: str = "rn", kept: int = 22, act_scale=None) -> np.ndarray:
    """Sigmoid output [h][w] (float64) of the float32 model.  fmt "e4m3" (the FP8 form):
    inner layers' weights as e4m3 codes of w / s_o with s_o = amax_o / 448 per output
    channel, their inputs (bf16 activations) as e4m3 codes of a / act_scale[l]; the sum of
    code products in float32, then times act_scale[l] s_o."""
    if fmt == "e4m3":
        return _forward_p_e4m3(contone, ws, bs, noise_seed, image, act_scale)
    h, w = contone.shape
    z = O.uniform_map(noise_seed, image, 0, h, w).astype(np.float32)     # exact: 24-bit values
    x = torch.from_numpy(np.stack([contone.astype(np.float32), z]))[None]
    L = len(ws)
    for l in range(L):
        wt = torch.from_numpy(np.asarray(ws[l], np.float32))
        bt = torch.from_numpy(np.asarray(bs[l], np.float32))
        if 0 < l < L - 1:
            wt = _round(wt, fmt)
        if l == 0 and first == "split2":
            x_hi = _round(x, "bf16")
            x_lo = _round(x - x_hi, "bf16")
            w_hi = _round(wt, "bf16")
            w_lo = _round(wt - w_hi, "bf16")
            # hi * (hi + lo) and lo * hi: every product is exact in float32 (8 x 16 bits)
            y = _conv_f32(torch.cat([x_hi, x_lo], 1), torch.cat([w_hi + w_lo, w_hi], 1), bt)
        elif acc == "trunc" and 0 < l < L - 1:
            y = _conv_trunc(x, wt, bt, kept)
        else:
            y = _conv_f32(x, wt, bt)
        if l < L - 1:
            y = _round(torch.relu(y), fmt)
        x = y
    return 1.0 / (1.0 + np.exp(-x[0, 0].double().numpy()))


def fp8_scales(ws, bs, chs):
    """Per-layer power-of-two input scales of the FP8 form from an oracle pass on the
    calibration image (seed 99), the rule the library's calibration follows:
    2^ceil(log2(amax / 448)) of each hidden layer's output."""
    from paper_2304_12152_gb300 import synth
    c = synth.contone_image(64, 64, seed=99)
    _, _, acts = O.forward(c, ws, bs, noise_seed=99, save_acts=True)
    sc = [1.0] * (len(chs) - 1)
    for l in range(1, len(chs) - 2):
        sc[l] = 2.0 ** math.ceil(math.log2(max(float(np.abs(acts[l - 1]).max()), 1e-6) / 448.0))
    return sc


def _forward_p_e4m3(contone, ws, bs, noise_seed, image, act_scale):
    h, w = contone.shape
    z = O.uniform_map(noise_seed, image, 0, h, w).astype(np.float32)
    x = torch.from_numpy(np.stack([contone.astype(np.float32), z]))[None]
    L = len(ws)
    for l in range(L):
        wt = torch.from_numpy(np.asarray(ws[l], np.float32))
        bt = torch.from_numpy(np.asarray(bs[l], np.float32))
        if 0 < l < L - 1:
            w64 = np.asarray(ws[l], np.float64)
            amax = np.abs(w64.reshape(w64.shape[0], -1)).max(1)
            so = np.where(amax > 0, amax / 448.0, 1.0)
            wcode = _e4m3(torch.from_numpy(w64 / so[:, None, None, None]).float())
            acode = _e4m3(x / float(act_scale[l]))
            y = _conv_f32(acode, wcode, torch.zeros_like(bt))
            y = y * torch.from_numpy((float(act_scale[l]) * so).astype(np.float32))[None, :, None, None] + bt[None, :, None, None]
        else:
            y = _conv_f32(x, wt, bt)
        if l < L - 1:
            y = _round(torch.relu(y), "bf16")
        x = y
    return 1.0 / (1.0 + np.exp(-x[0, 0].double().numpy()))


def forward_resnet_p(contone: np.ndarray, ws, bs, noise_seed: int, image: int = 0, acc: str = "rn",
                     kept: int = 22) -> np.ndarray:
    """The residual policy (stem, blocks y = ReLU(x + conv2(ReLU(conv1(x)))), output layer) in
    the BF16 form's rounding points -- block weights bf16, every stored activation bf16 (the
    block output after the shortcut add and the ReLU) -- with float32 sums."""
    h, w = contone.shape
    z = O.uniform_map(noise_seed, image, 0, h, w).astype(np.float32)
    x = torch.from_numpy(np.stack([contone.astype(np.float32), z]))[None]
    L = len(ws)
    conv = (lambda a, wt, bt: _conv_trunc(a, wt, bt, kept)) if acc == "trunc" else _conv_f32
    t = lambda l: (torch.from_numpy(np.asarray(ws[l], np.float32)), torch.from_numpy(np.asarray(bs[l], np.float32)))
    w0, b0 = t(0)
    x = _round(torch.relu(_conv_f32(x, w0, b0)), "bf16")
    for blk in range((L - 2) // 2):
        w1, b1 = t(1 + 2 * blk)
        w2, b2 = t(2 + 2 * blk)
        tt = _round(torch.relu(conv(x, _round(w1, "bf16"), b1)), "bf16")
        x = _round(torch.relu(conv(tt, _round(w2, "bf16"), b2) + x), "bf16")
    wl, bl = t(L - 1)
    y = _conv_f32(x, wl, bl)
    return 1.0 / (1.0 + np.exp(-y[0, 0].double().numpy()))
