"""Seeded synthetic inputs for the halftoning path.

This module holds no arithmetic of the halftoning method. It only produces
the *inputs* that the method consumes, so that the CUDA library and the CPU
oracle are fed identical data:

* contone images in [0, 1] (float32): a linear gradient, 20 filled ellipses
  painted in order and additive Gaussian noise (sigma 0.02), clamped.  They
  stand in for the VOC2012 / DIV2K photographs the paper evaluates on (the
  datasets are not available here); the paper's test shapes are 512x512 and
  2040x2040 and its training crops 64x64 (Sec. VI-A).
* He-normal policy weights, w ~ N(0, 2 / (9 * C_in)), zero biases, in the
  canonical OIHW float32 layout.
* constant-gray patches (Sec. IV: the anisotropy loss is evaluated on
  constant-gray images).
* the uneven size draw of a mixed batch (areas log-uniform, aspect ratios
  log-uniform).

Every array is a pure function of its seed tuple (numpy PCG64 seeded through
SeedSequence).  The per-pixel noise channel z and the Bernoulli uniforms u are
NOT produced here: both sides generate them from the counter-based Philox4x32-10
generator keyed by (seed, image, pixel), each side with its own implementation.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) & 0xFFFFFFFF for k in key])))


def contone_image(h: int, w: int, seed: int, index: int = 0, n_ellipses: int = 20,
                  noise_sigma: float = 0.02) -> np.ndarray:
    """One synthetic contone image, float32 [h][w] in [0, 1]."""
    if h < 1 or w < 1:
        raise ValueError("image size must be positive")
    rng = _rng(0x5EED, seed, index)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    ys = np.arange(h, dtype=np.float64)[:, None] + 0.5
    xs = np.arange(w, dtype=np.float64)[None, :] + 0.5
    proj = xs * math.cos(phi) + ys * math.sin(phi)
    lo, hi = proj.min(), proj.max()
    t = (proj - lo) / (hi - lo) if hi > lo else np.zeros_like(proj)
    img = 0.1 + 0.8 * t
    m = min(h, w)
    for _ in range(n_ellipses):
        cy = rng.uniform(0.0, h)
        cx = rng.uniform(0.0, w)
        a = rng.uniform(0.03, 0.3) * m
        b = rng.uniform(0.03, 0.3) * m
        ang = rng.uniform(0.0, math.pi)
        gray = rng.uniform(0.0, 1.0)
        r = max(a, b)
        y0, y1 = max(0, int(cy - r) - 1), min(h, int(cy + r) + 2)
        x0, x1 = max(0, int(cx - r) - 1), min(w, int(cx + r) + 2)
        if y0 >= y1 or x0 >= x1:
            continue
        dy = ys[y0:y1, :] - cy
        dx = xs[:, x0:x1] - cx
        ca, sa = math.cos(ang), math.sin(ang)
        u = (dx * ca + dy * sa) / a
        v = (-dx * sa + dy * ca) / b
        inside = (u * u + v * v) <= 1.0
        sub = img[y0:y1, x0:x1]
        sub[inside] = gray
    img = img + rng.normal(0.0, noise_sigma, size=(h, w))
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def contone_batch(shapes: Sequence[Tuple[int, int]], seed: int) -> List[np.ndarray]:
    return [contone_image(h, w, seed, i) for i, (h, w) in enumerate(shapes)]


def gray_patch(n: int, level: float) -> np.ndarray:
    return np.full((n, n), level, dtype=np.float32)


def he_normal_policy(channels: Sequence[int], seed: int) -> Tuple[List[np.ndarray], List[np.ndarray]]:
    """He-normal 3x3 weights (OIHW float32) and zero biases for every layer."""
    ws, bs = [], []
    for l in range(len(channels) - 1):
        cin, cout = channels[l], channels[l + 1]
        rng = _rng(0x3E16, seed, l)
        std = math.sqrt(2.0 / (9.0 * cin))
        ws.append(rng.normal(0.0, std, size=(cout, cin, 3, 3)).astype(np.float32))
        bs.append(np.zeros(cout, dtype=np.float32))
    return ws, bs


def resnet_policy(n_blocks: int, width: int, seed: int, branch_scale: float = 0.0) -> Tuple[List[np.ndarray], List[np.ndarray]]:
    """Residual policy weights (layers: stem, (conv1, conv2) per block, out), He-normal
    with each block's second convolution scaled by branch_scale (default 1 / sqrt(n_blocks),
    so that the residual stream does not grow with depth); zero biases."""
    ch = resnet_channels(n_blocks, width)
    ws, bs = he_normal_policy(ch, seed)
    k = branch_scale or 1.0 / math.sqrt(max(1, n_blocks))
    for b in range(n_blocks):
        ws[2 + 2 * b] = (ws[2 + 2 * b] * k).astype(np.float32)
    return ws, bs


def resnet_channels(n_blocks: int, width: int) -> Tuple[int, ...]:
    """Channels per layer boundary of the residual policy (stem, 2 per block, out)."""
    return (2,) + (width,) * (1 + 2 * n_blocks) + (1,)


def random_biases(channels: Sequence[int], seed: int, scale: float = 0.05) -> List[np.ndarray]:
    """Small non-zero biases (tests use them so that the bias path is exercised)."""
    out = []
    for l in range(len(channels) - 1):
        rng = _rng(0xB1A5, seed, l)
        out.append(rng.uniform(-scale, scale, size=channels[l + 1]).astype(np.float32))
    return out


def uneven_shapes(n: int, seed: int, min_hw=(200, 300), max_hw=(4096, 3072),
                  aspect=(0.5, 2.0), clamp=(200, 4096)) -> List[Tuple[int, int]]:
    """Sizes of a mixed batch: area log-uniform between the two extremes, aspect
    ratio w/h log-uniform, both sides clamped."""
    rng = _rng(0x512E, seed)
    a_lo = math.log(min_hw[0] * min_hw[1])
    a_hi = math.log(max_hw[0] * max_hw[1])
    r_lo, r_hi = math.log(aspect[0]), math.log(aspect[1])
    out = []
    for _ in range(n):
        area = math.exp(rng.uniform(a_lo, a_hi))
        r = math.exp(rng.uniform(r_lo, r_hi))
        hh = int(round(math.sqrt(area / r)))
        ww = int(round(math.sqrt(area * r)))
        hh = min(max(hh, clamp[0]), clamp[1])
        ww = min(max(ww, clamp[0]), clamp[1])
        out.append((hh, ww))
    return out


# Network shapes of the workloads (channels per layer boundary).
NET_SMALL = (2, 32, 32, 32, 32, 32, 1)            # 6 conv layers, 32 wide
NET_WIDE = (2, 64, 64, 64, 64, 64, 64, 64, 1)     # 8 conv layers, 64 wide
NET_WIDE_K4 = (2, 64, 64, 64, 64, 64, 64, 64, 4)  # 4-logit softmax head
RESNET_BLOCKS, RESNET_WIDTH = 16, 32              # residual policy of Sec. VI-A


def net_flops_per_px(channels: Sequence[int]) -> int:
    """2 * MACs per output pixel of a 3x3 conv stack."""
    return int(sum(2 * 9 * channels[i] * channels[i + 1] for i in range(len(channels) - 1)))
