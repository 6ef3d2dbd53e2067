"""FP64 CPU oracle for the halftoning path -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the CPU-baseline leg of bench.py
may import this package.  The product (the CUDA library and its binding) never
does.  The arithmetic lives in ht_oracle.c (plain C, double precision, direct
loops); this module only builds it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ht_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libht_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ht_oracle.c into a shared library (gcc, OpenMP, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_GNU_SOURCE",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class RewardOpts(C.Structure):
    _fields_ = [("sigma_hvs", C.c_double), ("sigma_ssim", C.c_double), ("k_contrast", C.c_double),
                ("w_s", C.c_double), ("c1", C.c_double), ("c2", C.c_double), ("radius", C.c_int)]


def reward_opts(sigma_hvs=2.0, sigma_ssim=1.5, k_contrast=2.0, w_s=0.06, c1=0.01 ** 2, c2=0.03 ** 2, radius=5):
    return RewardOpts(sigma_hvs, sigma_ssim, k_contrast, w_s, c1, c2, radius)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp, fp, u8p, i64p = (np.ctypeslib.ndpointer(np.float64, flags="C"),
                                 np.ctypeslib.ndpointer(np.float32, flags="C"),
                                 np.ctypeslib.ndpointer(np.uint8, flags="C"),
                                 np.ctypeslib.ndpointer(np.int64, flags="C"))
            L.or_philox4x32_10.argtypes = [np.ctypeslib.ndpointer(np.uint32, flags="C")] * 3
            L.or_uniform.restype = C.c_double
            L.or_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64]
            L.or_uniform_map.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, dp]
            L.or_round_bf16.restype = C.c_double
            L.or_round_bf16.argtypes = [C.c_double]
            L.or_round_e4m3.restype = C.c_double
            L.or_round_e4m3.argtypes = [C.c_double]
            L.or_round_fp16.restype = C.c_double
            L.or_round_fp16.argtypes = [C.c_double]
            L.or_forward.restype = C.c_int
            L.or_forward.argtypes = [fp, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_uint64, C.c_uint32,
                                     C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_sample.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.c_uint64, C.c_uint32, u8p, C.c_void_p]
            L.or_gauss2d.argtypes = [C.c_double, C.c_int, dp]
            L.or_reward.restype = C.c_int
            L.or_reward.argtypes = [fp, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(RewardOpts),
                                    dp, C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_toggle_delta.restype = C.c_int
            L.or_toggle_delta.argtypes = [fp, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p,
                                          C.POINTER(RewardOpts), i64p, C.c_int64, dp]
            L.or_dft2.argtypes = [dp, C.c_void_p, C.c_int, C.c_int, dp, dp]
            L.or_anisotropy_loss.restype = C.c_int
            L.or_anisotropy_loss.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, dp, C.c_void_p, C.c_int,
                                             C.c_void_p, C.c_void_p]
            L.or_backward.restype = C.c_int
            L.or_backward.argtypes = [fp, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                      C.POINTER(C.c_void_p), C.c_uint64, C.c_uint32, C.c_int,
                                      C.POINTER(C.c_void_p), dp, dp, C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p)]
            L.or_forward_resnet.restype = C.c_int
            L.or_forward_resnet.argtypes = [fp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p),
                                            C.POINTER(C.c_void_p), C.c_uint64, C.c_uint32, C.c_int, C.c_int,
                                            C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
            L.or_num_threads.restype = C.c_int
            L.or_set_num_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(c, k, out)
    return out


def uniform(seed: int, image: int, stream: int, g: int) -> float:
    return lib().or_uniform(seed, image, stream, g)


def uniform_map(seed: int, image: int, stream: int, h: int, w: int) -> np.ndarray:
    out = np.zeros((h, w), dtype=np.float64)
    lib().or_uniform_map(seed, image, stream, h, w, out)
    return out


def round_bf16(x: float) -> float:
    return lib().or_round_bf16(float(x))


def round_e4m3(x: float) -> float:
    return lib().or_round_e4m3(float(x))


def round_fp16(x: float) -> float:
    return lib().or_round_fp16(float(x))


def _layers(weights: Sequence[np.ndarray], biases: Sequence[np.ndarray]):
    ws = [np.ascontiguousarray(w, dtype=np.float32) for w in weights]
    bs = [np.ascontiguousarray(b, dtype=np.float32) for b in biases]
    ch = [ws[0].shape[1]] + [w.shape[0] for w in ws]
    wp = (C.c_void_p * len(ws))(*[w.ctypes.data for w in ws])
    bp = (C.c_void_p * len(bs))(*[b.ctypes.data for b in bs])
    chp = (C.c_int * len(ch))(*ch)
    return ws, bs, ch, wp, bp, chp


def forward(contone: np.ndarray, weights, biases, noise_seed: int, image: int = 0, quant: int = 0,
            act_scale: Optional[Sequence[float]] = None, region: Optional[Tuple[int, int, int, int]] = None,
            save_acts: bool = False):
    """Policy forward.  Returns (logits [K][rh][rw], probs [K][rh][rw], acts or None)."""
    c = np.ascontiguousarray(contone, dtype=np.float32)
    h, w = c.shape
    ws, bs, ch, wp, bp, chp = _layers(weights, biases)
    L = len(ws)
    y0, x0, rh, rw = region if region is not None else (0, 0, h, w)
    K = ch[-1]
    logits = np.zeros((K, rh, rw), dtype=np.float64)
    probs = np.zeros((K, rh, rw), dtype=np.float64)
    acts = None
    accp = None
    if save_acts:
        acts = [np.zeros((ch[l + 1], h, w), dtype=np.float64) for l in range(L - 1)]
        accp = (C.c_void_p * max(1, L - 1))(*[a.ctypes.data for a in acts])
    sc = None
    if act_scale is not None:
        sc = np.ascontiguousarray(act_scale, dtype=np.float64)
    rc = lib().or_forward(c, h, w, w, L, chp, wp, bp, noise_seed, image, quant, _ptr(sc),
                          y0, x0, rh, rw, _ptr(logits), _ptr(probs), accp)
    if rc != 0:
        raise ValueError(f"or_forward failed ({rc})")
    return logits, probs, acts


def sample(probs: np.ndarray, h: int, w: int, region, mode: int, seed: int, image: int = 0):
    """Actions for the region; returns (levels uint8 [rh][rw], u [rh][rw])."""
    K, rh, rw = probs.shape
    y0, x0, _, _ = region
    out = np.zeros((rh, rw), dtype=np.uint8)
    u = np.zeros((rh, rw), dtype=np.float64)
    lib().or_sample(np.ascontiguousarray(probs), K, h, w, y0, x0, rh, rw, mode, seed, image, out, _ptr(u))
    return out, u


def gauss2d(sigma: float, radius: int = 5) -> np.ndarray:
    g = np.zeros((2 * radius + 1, 2 * radius + 1), dtype=np.float64)
    lib().or_gauss2d(sigma, radius, g)
    return g


def reward(contone: np.ndarray, h_bits: np.ndarray, opts: Optional[RewardOpts] = None, maps: bool = False,
           levels: int = 2):
    """Returns dict(mse, ssim, cssim, R[, e, ssim_map, sigma]).  h_bits: level indices
    0 .. levels-1 (halftone value index / (levels - 1); binary for levels = 2)."""
    o = opts or reward_opts()
    c = np.ascontiguousarray(contone, dtype=np.float32)
    hb = np.ascontiguousarray(h_bits, dtype=np.uint8)
    H, W = c.shape
    out = np.zeros(4, dtype=np.float64)
    r = o.radius
    e = s = sg = None
    if maps:
        e = np.zeros((H - 2 * r, W - 2 * r)); s = np.zeros_like(e); sg = np.zeros_like(e)
    rc = lib().or_reward(c, W, hb, W, H, W, 1.0 / (levels - 1), C.byref(o), out, _ptr(e), _ptr(s), _ptr(sg))
    if rc != 0:
        raise ValueError("or_reward: image smaller than the window")
    d = dict(mse=out[0], ssim=out[1], cssim=out[2], R=out[3])
    if maps:
        d.update(e=e, ssim_map=s, sigma=sg)
    return d


def toggle_delta(contone: np.ndarray, h_bits: np.ndarray, idx: Optional[np.ndarray] = None,
                 opts: Optional[RewardOpts] = None, levels: int = 2, lo: Optional[np.ndarray] = None) -> np.ndarray:
    """dR_a = R(h_a = hi) - R(h_a = lo) per requested pixel.  Binary: lo 0, hi 1.  Multitone
    prototype (levels > 2): lo = the lower level index of the pair around the output
    (multitone_pair), hi = lo + 1; h_bits holds level indices."""
    o = opts or reward_opts()
    c = np.ascontiguousarray(contone, dtype=np.float32)
    hb = np.ascontiguousarray(h_bits, dtype=np.uint8)
    H, W = c.shape
    if idx is None:
        idx = np.arange(H * W, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(idx.shape[0], dtype=np.float64)
    lo_a = None if lo is None else np.ascontiguousarray(lo, dtype=np.uint8).reshape(H, W)
    rc = lib().or_toggle_delta(c, W, hb, W, H, W, 1.0 / (levels - 1), _ptr(lo_a), C.byref(o), idx, idx.shape[0],
                               out)
    if rc != 0:
        raise ValueError("or_toggle_delta: image smaller than the window")
    return out


def dft2(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unnormalised 2-D DFT from the definition (sign -1 forward, +1 inverse)."""
    x = np.asarray(x)
    n = x.shape[0]
    re = np.ascontiguousarray(x.real, dtype=np.float64)
    im = np.ascontiguousarray(x.imag, dtype=np.float64) if np.iscomplexobj(x) else None
    ro = np.zeros((n, n)); io = np.zeros((n, n))
    lib().or_dft2(re, _ptr(im), n, 1 if inverse else -1, ro, io)
    return ro + 1j * io


def anisotropy_loss(q: np.ndarray, mode: int = 0, n_rad: int = 32, n_ang: int = 16, grad: bool = False):
    """Returns dict(loss, aniso (paper-form A per ring, NaN where undefined), psd, grad)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = q.shape[0]
    out = np.zeros(1)
    n_an = int(round(np.sqrt(2.0) * (n // 2))) + 1
    an = np.zeros(n_an)
    psd = np.zeros((n, n))
    g = np.zeros((n, n)) if grad else None
    rings = lib().or_anisotropy_loss(q, n, mode, n_rad, n_ang, out, _ptr(an), n_an, _ptr(psd), _ptr(g))
    if rings < 0:
        raise ValueError("anisotropy loss needs an even n >= 4")
    return dict(loss=out[0], aniso=an, psd=psd, grad=g)


def forward_resnet(contone: np.ndarray, weights, biases, noise_seed: int, image: int = 0, quant: int = 0,
                   region: Optional[Tuple[int, int, int, int]] = None):
    """Residual policy (Sec. VI-A): stem 2 -> C, len(weights) // 2 - 1 residual blocks
    y = ReLU(x + conv2(ReLU(conv1(x)))), output C -> 1, sigmoid.  Returns (logits, probs)
    as [rh][rw] arrays over region (y0, x0, rh, rw) (default: the whole image)."""
    c = np.ascontiguousarray(contone, dtype=np.float32)
    H, W = c.shape
    y0, x0, h, w = region if region is not None else (0, 0, H, W)
    ws = [np.ascontiguousarray(x, dtype=np.float32) for x in weights]
    bs = [np.ascontiguousarray(x, dtype=np.float32) for x in biases]
    L = len(ws)
    nb = (L - 2) // 2
    C_ = ws[0].shape[0]
    wp = (C.c_void_p * L)(*[x.ctypes.data for x in ws])
    bp = (C.c_void_p * L)(*[x.ctypes.data for x in bs])
    lg = np.zeros((h, w))
    pr = np.zeros((h, w))
    rc = lib().or_forward_resnet(c, H, W, W, nb, C_, wp, bp, noise_seed, image, quant, y0, x0, h, w, _ptr(lg),
                                 _ptr(pr))
    if rc != 0:
        raise ValueError("or_forward_resnet failed")
    return lg, pr


def backward(contone: np.ndarray, weights, biases, noise_seed: int, image: int, acts, logits: np.ndarray,
             dprob: np.ndarray, quant: int = 0):
    """dL/dW, dL/db (double) for a sigmoid-head policy on a whole image.  quant 1: the BF16
    form's rounding points (inner layers' data gradients with bf16 weights, hidden-layer
    pre-activation gradients rounded to bf16); pass acts and logits of the quant-1 forward."""
    c = np.ascontiguousarray(contone, dtype=np.float32)
    h, w = c.shape
    ws, bs, ch, wp, bp, chp = _layers(weights, biases)
    L = len(ws)
    gw = [np.zeros(x.shape, dtype=np.float64) for x in ws]
    gb = [np.zeros(x.shape, dtype=np.float64) for x in bs]
    gwp = (C.c_void_p * L)(*[a.ctypes.data for a in gw])
    gbp = (C.c_void_p * L)(*[a.ctypes.data for a in gb])
    accp = (C.c_void_p * max(1, L - 1))(*[a.ctypes.data for a in acts]) if acts else None
    lg = np.ascontiguousarray(logits.reshape(h, w), dtype=np.float64)
    dp = np.ascontiguousarray(dprob.reshape(h, w), dtype=np.float64)
    rc = lib().or_backward(c, h, w, w, L, chp, wp, noise_seed, image, quant, accp, lg, dp, gwp, gbp)
    if rc != 0:
        raise ValueError("or_backward failed")
    return gw, gb


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(n)


# ---------------------------------------------------------------------------
# Composite helpers written from the paper's formulas on top of the routines
# above (Algorithm 1).
# ---------------------------------------------------------------------------

def multitone_pair(v: np.ndarray, levels: int):
    """Sec. VI-E: the two levels around the output v in [0, 1] with L = levels ink levels,
    Delta = 1 / (L - 1): lower index k = floor(v (L - 1)) (at most L - 2) and the
    probability (v - k Delta) / Delta of the upper one.  Returns (k, frac)."""
    t = np.asarray(v, np.float64) * (levels - 1)
    k = np.minimum(np.floor(t), levels - 2).astype(np.int64)
    return k, t - k


def sample_multitone(v: np.ndarray, levels: int, u: Optional[np.ndarray] = None):
    """Action of the multitone prototype: level k + 1 with probability frac, else k
    (u given: Bernoulli with u < frac; u None: threshold, frac > 0.5)."""
    k, frac = multitone_pair(v, levels)
    up = (frac > 0.5) if u is None else (np.asarray(u) < frac)
    return (k + up).astype(np.uint8)


def le_surrogate_multitone(v: np.ndarray, h_levels: np.ndarray, dR: np.ndarray, R: float, levels: int):
    """L_MARL of the multitone prototype for one sample (Sec. VI-E: the same target with
    the binary action between the two levels around v):
      L = -sum_a [pi_a(hi) R(h_a = hi) + pi_a(lo) R(h_a = lo)],
      pi_a(hi) = (v_a - lo Delta) / Delta, dR_a = R(hi) - R(lo), so dL/dv_a = -dR_a / Delta.
    Returns (value, dL/dv)."""
    k, frac = multitone_pair(v.reshape(dR.shape), levels)
    hl = h_levels.reshape(dR.shape).astype(np.int64)
    at_hi = (hl == k + 1).astype(np.float64)
    r_hi = R + (1.0 - at_hi) * dR
    r_lo = R - at_hi * dR
    val = -np.sum(frac * r_hi + (1.0 - frac) * r_lo)
    return float(val), -dR * (levels - 1)


def coma_surrogate(prob: np.ndarray, h_bits: np.ndarray, dR: np.ndarray, R: float):
    """Eq. (coma) with the counterfactual baseline Eq. (baseline), one sample:
    b_a = sum_{h'} pi_a(h') R({h', h_-a}), so R(h) - b_a = (1 - p_a) dR_a if h_a = 1 and
    -p_a dR_a if h_a = 0, with dR_a = R(h_a = 1) - R(h_a = 0).  Surrogate loss
    L_COMA = -sum_a log pi_a(h_a) (R(h) - b_a) with R - b held constant.
    Returns (value, dL/dp) where d log pi_a(h_a) / dp_a = h_a / p_a - (1 - h_a) / (1 - p_a)."""
    p = prob.reshape(dR.shape).astype(np.float64)
    hb = h_bits.reshape(dR.shape).astype(np.float64)
    adv = np.where(hb > 0, (1.0 - p) * dR, -p * dR)
    logpi = np.where(hb > 0, np.log(np.where(hb > 0, p, 1.0)), np.log(np.where(hb > 0, 1.0, 1.0 - p)))
    dlogpi = np.where(hb > 0, 1.0 / np.where(hb > 0, p, 1.0), -1.0 / np.where(hb > 0, 1.0, 1.0 - p))
    return float(-np.sum(logpi * adv)), -dlogpi * adv


def le_surrogate(prob: np.ndarray, h_bits: np.ndarray, dR: np.ndarray, R: float):
    """Eq. (marl) / Algorithm 1: L_MARL = -sum_a sum_{h'} R({h'_a, h_-a}) pi_a(h'_a)
    for one sample, with R(h_a = h'_a) = R + (h'_a - h_a) dR_a.
    Returns (value, dL/dp = -dR)."""
    p = prob.reshape(dR.shape)
    hb = h_bits.reshape(dR.shape).astype(np.float64)
    r1 = R + (1.0 - hb) * dR
    r0 = R - hb * dR
    val = -np.sum(p * r1 + (1.0 - p) * r0)
    return float(val), -dR
