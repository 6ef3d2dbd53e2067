"""Python binding of the halftoning library: argument marshalling only.

Every step of the path runs in libht.so's CUDA kernels; torch provides device
memory and the current stream.  Function names follow include/ht.h.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import _native as N
from ._native import check


def _stream(stream: Optional[torch.cuda.Stream] = None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _images(contones: Sequence[torch.Tensor]):
    arr = (N.Image * len(contones))()
    for i, c in enumerate(contones):
        if not (c.is_cuda and c.dtype == torch.float32 and c.dim() == 2 and c.stride(1) == 1):
            raise ValueError("contone images must be 2-D float32 CUDA tensors with unit column stride")
        arr[i] = N.Image(c.data_ptr(), c.shape[0], c.shape[1], c.stride(0))
    return arr


def _ptrs(ts: Sequence[Optional[torch.Tensor]]):
    return (C.c_void_p * len(ts))(*[(t.data_ptr() if t is not None else None) for t in ts])


def bits_row_words(w: int, head: int = N.HT_HEAD_SIGMOID) -> int:
    return N.load().ht_bits_row_words(w, head)


def reward_opts(**kw) -> N.RewardOpts:
    o = N.RewardOpts()
    N.load().ht_reward_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Policy:
    """ht_policy: owns packed weights and the forward workspace."""

    def __init__(self, channels: Sequence[int], weights: Sequence[np.ndarray], biases: Sequence[np.ndarray],
                 head: int = N.HT_HEAD_SIGMOID, precision: int = N.HT_FP32, levels: int = 4,
                 arch: int = N.HT_ARCH_PLAIN):
        L = N.load()
        d = N.PolicyDesc()
        d.arch = arch
        d.n_layers = len(channels) - 1
        for i, c in enumerate(channels):
            d.channels[i] = int(c)
        d.head, d.precision = head, precision
        d.levels = levels if head == N.HT_HEAD_MULTITONE else 0
        w = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).ravel() for x in weights]))
        b = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).ravel() for x in biases]))
        h = C.c_void_p()
        check(L.ht_create_policy(C.byref(d), w.ctypes.data, b.ctypes.data, C.byref(h)))
        self._h = h
        self.channels = tuple(int(c) for c in channels)
        self.head, self.precision = head, precision
        self.levels = levels if head == N.HT_HEAD_MULTITONE else (4 if head == N.HT_HEAD_SOFTMAX else 2)
        self.K = self.channels[-1]

    def close(self):
        if getattr(self, "_h", None):
            N.load().ht_destroy_policy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def num_params(self) -> int:
        return N.load().ht_policy_num_params(self._h)

    def flops_per_px(self) -> int:
        return N.load().ht_policy_flops_per_px(self._h)

    def set_act_scales(self, scales: Sequence[float]) -> None:
        a = np.ascontiguousarray(scales, np.float32)
        check(N.load().ht_policy_set_act_scales(self._h, a.ctypes.data, a.size))

    def calibrate(self, contone: torch.Tensor, seed: int = 99, stream=None) -> None:
        """FP8 form: static activation scales from one calibration image (ht_policy_calibrate)."""
        check(N.load().ht_policy_calibrate(self._h, _images([contone]), seed, _stream(stream)))

    def set_weights(self, w_dev: torch.Tensor, b_dev: torch.Tensor, stream=None) -> None:
        check(N.load().ht_policy_set_weights(self._h, w_dev.data_ptr(), b_dev.data_ptr(), _stream(stream)))

    def alloc_bits(self, h: int, w: int, device="cuda") -> torch.Tensor:
        words = bits_row_words(w, self.head)
        return torch.empty((h, words), dtype=torch.int32, device=device)

    def halftone_into(self, contones: Sequence[torch.Tensor], bits: Sequence[torch.Tensor], mode: int, seed: int,
                      probs: Optional[Sequence[Optional[torch.Tensor]]] = None, stream=None) -> None:
        imgs = _images(contones)
        check(N.load().ht_halftone(self._h, imgs, len(contones), mode, seed, _ptrs(bits),
                                   _ptrs(probs) if probs is not None else None, _stream(stream)))

    def set_schedule(self, rows_per_unit: int, unit_order: int, cta_pair: int = 0) -> None:
        check(N.load().ht_policy_set_schedule(self._h, rows_per_unit, unit_order, cta_pair))

    def autotune(self, contones: Sequence[torch.Tensor], bits: Sequence[torch.Tensor], mode: int, seed: int,
                 probs: Optional[Sequence[Optional[torch.Tensor]]] = None, reps: int = 3, stream=None):
        """ht_policy_autotune: times every conv schedule on this call, keeps the fastest.
        Returns [(rows_per_unit, unit_order, cta_pair, ms)] in candidate order."""
        res = (N.TuneResult * N.HT_TUNE_CANDIDATES)()
        n = C.c_int(0)
        check(N.load().ht_policy_autotune(self._h, _images(contones), len(contones), mode, seed, _ptrs(bits),
                                          _ptrs(probs) if probs is not None else None, reps, res,
                                          N.HT_TUNE_CANDIDATES, C.byref(n), _stream(stream)))
        return [(res[k].rows_per_unit, res[k].unit_order, res[k].cta_pair, float(res[k].ms)) for k in range(n.value)]

    def halftone(self, contones: Sequence[torch.Tensor], mode: int = N.HT_MODE_THRESHOLD, seed: int = 0,
                 want_prob: bool = False, stream=None):
        bits = [self.alloc_bits(c.shape[0], c.shape[1], c.device) for c in contones]
        probs = None
        if want_prob:
            probs = [torch.empty((self.K, c.shape[0], c.shape[1]), dtype=torch.float32, device=c.device)
                     for c in contones]
        self.halftone_into(contones, bits, mode, seed, probs, stream)
        return bits, probs


class Plan:
    """ht_plan: one halftone call (fixed images, outputs, mode, seed) captured into a
    CUDA graph; launch() replays it.  Keeps references to the tensors it points at."""

    def __init__(self, policy: Policy, contones: Sequence[torch.Tensor], bits: Sequence[torch.Tensor], mode: int,
                 seed: int, probs: Optional[Sequence[Optional[torch.Tensor]]] = None):
        h = C.c_void_p()
        check(N.load().ht_plan_create(policy.handle, _images(contones), len(contones), mode, seed, _ptrs(bits),
                                      _ptrs(probs) if probs is not None else None, C.byref(h)))
        self._h, self.policy = h, policy
        self._keep = (list(contones), list(bits), list(probs) if probs is not None else None)

    def launch(self, stream=None) -> None:
        check(N.load().ht_plan_launch(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            N.load().ht_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reward(contones: Sequence[torch.Tensor], bits: Sequence[torch.Tensor], opts: Optional[N.RewardOpts] = None,
           out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    o = opts or reward_opts()
    if out is None:
        out = torch.empty((len(contones), 4), dtype=torch.float64, device=contones[0].device)
    check(N.load().ht_reward(_images(contones), _ptrs(bits), len(contones), C.byref(o), out.data_ptr(),
                             _stream(stream)))
    return out


def toggle_delta(contones: Sequence[torch.Tensor], bits: Sequence[torch.Tensor],
                 opts: Optional[N.RewardOpts] = None, stream=None,
                 v: Optional[Sequence[torch.Tensor]] = None) -> List[torch.Tensor]:
    """dR per pixel; multi-level halftones (opts.levels > 2) need the policy outputs v."""
    o = opts or reward_opts()
    dR = [torch.empty_like(c) for c in contones]
    check(N.load().ht_toggle_delta(_images(contones), _ptrs(bits), _ptrs(v) if v is not None else None,
                                   len(contones), C.byref(o), _ptrs(dR), _stream(stream)))
    return dR


def anisotropy_loss(q: torch.Tensor, mode: int = 0, n_rad: int = 32, n_ang: int = 16, grad: bool = False,
                    stream=None) -> Tuple[torch.Tensor, Optional[torch.Tensor]]:
    if q.dim() == 2:
        q = q[None]
    q = q.contiguous()
    P, n, _ = q.shape
    loss = torch.empty(P, dtype=torch.float64, device=q.device)
    g = torch.empty_like(q) if grad else None
    check(N.load().ht_anisotropy_loss(q.data_ptr(), P, n, mode, n_rad, n_ang, loss.data_ptr(),
                                      g.data_ptr() if g is not None else None, _stream(stream)))
    return loss, g


class Trainer:
    """ht_train: one iteration of the training step (forward + backward) on device."""

    def __init__(self, policy: Policy, crop_hw: Tuple[int, int], max_crops: int, n_samples: int = 4,
                 n_gray: int = 0, gray_n: int = 256, las_mode: int = 1, n_rad: int = 32, n_ang: int = 16,
                 w_a: float = 0.002, reward: Optional[N.RewardOpts] = None, estimator: int = N.HT_EST_LE,
                 ckpt_stride: int = 0):
        d = N.TrainDesc()
        d.estimator = estimator
        d.ckpt_stride = ckpt_stride
        d.max_crops, (d.crop_h, d.crop_w) = max_crops, crop_hw
        d.n_gray, d.gray_n, d.n_samples = n_gray, gray_n, n_samples
        d.las_mode, d.n_rad, d.n_ang, d.w_a = las_mode, n_rad, n_ang, w_a
        d.reward = reward or reward_opts()
        h = C.c_void_p()
        check(N.load().ht_train_create(policy.handle, C.byref(d), C.byref(h)))
        self._h, self.policy, self.desc = h, policy, d

    def close(self):
        if getattr(self, "_h", None):
            N.load().ht_train_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, crops: Sequence[torch.Tensor], gray_levels: Sequence[float] = (), seed: int = 0,
                stream=None) -> Tuple[float, float, float, float]:
        """(L_total, L_MARL, L_AS, mean reward)."""
        out = (C.c_double * 4)()
        lv = np.ascontiguousarray(gray_levels, np.float32) if len(gray_levels) else np.zeros(1, np.float32)
        check(N.load().ht_train_step_fwd(self._h, _images(crops), len(crops), lv.ctypes.data, seed, out,
                                         _stream(stream)))
        self._crops = list(crops)      # the backward re-reads the crops (first-layer input)
        return tuple(out)

    def backward(self, grad_w: Optional[torch.Tensor] = None, grad_b: Optional[torch.Tensor] = None, stream=None):
        n_w = sum(self.policy.channels[i] * self.policy.channels[i + 1] * 9 for i in range(len(self.policy.channels) - 1))
        n_b = sum(self.policy.channels[1:])
        dev = torch.device("cuda", torch.cuda.current_device())
        grad_w = grad_w if grad_w is not None else torch.empty(n_w, dtype=torch.float32, device=dev)
        grad_b = grad_b if grad_b is not None else torch.empty(n_b, dtype=torch.float32, device=dev)
        check(N.load().ht_train_step_bwd(self._h, grad_w.data_ptr(), grad_b.data_ptr(), _stream(stream)))
        return grad_w, grad_b


def allreduce_grads(grads: Sequence[torch.Tensor], group=None) -> Sequence[torch.Tensor]:
    """Data-parallel training over the ranks of a process group (each rank steps on its own
    crops): averages the gradient tensors in place with one all-reduce of their
    concatenation -- the training path's only exchange (0.9 MB of FP32 for the 8-layer
    64-wide policy).  No-op without an initialised process group of size > 1."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return grads
    world = dist.get_world_size(group)
    if world == 1:
        return grads
    flat = torch.cat([g.reshape(-1) for g in grads])
    dist.all_reduce(flat, group=group)
    flat.div_(world)
    off = 0
    for g in grads:
        g.copy_(flat[off:off + g.numel()].view_as(g))
        off += g.numel()
    return grads


class HalftonePolicyFn(torch.autograd.Function):
    """torch.autograd.Function driving one training iteration of the library.

    forward(w_flat, b_flat, trainer, crops, gray_levels, seed) loads the FP32 master
    weights into the policy, runs ht_train_step_fwd and returns L_total as a 0-d
    tensor; backward returns dL_total/dw and dL_total/db from ht_train_step_bwd
    (the local-expectation gradient of L_MARL plus w_a times the anisotropy-loss
    gradient), scaled by the incoming gradient.  The optimiser stays in torch."""

    @staticmethod
    def forward(ctx, w_flat, b_flat, trainer, crops, gray_levels, seed):
        trainer.policy.set_weights(w_flat.detach().contiguous(), b_flat.detach().contiguous())
        losses = trainer.forward(crops, gray_levels, seed)
        ctx.trainer = trainer
        ctx.losses = losses
        return torch.tensor(losses[0], dtype=torch.float64, device=w_flat.device)

    @staticmethod
    def backward(ctx, g):
        gw, gb = ctx.trainer.backward()
        s = g.to(torch.float32)
        return gw * s, gb * s, None, None, None, None


def profile_begin() -> None:
    check(N.load().ht_profile_begin())


def profile_end() -> dict:
    """{kernel name: (launches, total device ms)} since profile_begin (synchronises)."""
    arr = (N.KernelStat * 32)()
    n = C.c_int(0)
    check(N.load().ht_profile_end(arr, 32, C.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}


def _flat_f32(x) -> np.ndarray:
    """A flat float32 host array from a torch tensor (any device), an array or a
    sequence of per-layer arrays."""
    if isinstance(x, torch.Tensor):
        return np.ascontiguousarray(x.detach().to("cpu", torch.float32).reshape(-1).numpy())
    if isinstance(x, np.ndarray):
        return np.ascontiguousarray(x.astype(np.float32, copy=False).reshape(-1))
    return np.ascontiguousarray(np.concatenate([np.asarray(
        t.detach().cpu() if isinstance(t, torch.Tensor) else t, np.float32).ravel() for t in x]))


def save_checkpoint(path: str, channels: Sequence[int], weights, biases, head: int = N.HT_HEAD_SIGMOID,
                    precision: int = N.HT_FP32, levels: int = 4, arch: int = N.HT_ARCH_PLAIN,
                    act_scales: Optional[Sequence[float]] = None, step: int = 0) -> None:
    """ht_checkpoint_save: the policy's descriptor and canonical float32 parameters (flat
    tensors such as a training run's master weights, or per-layer OIHW arrays), the FP8
    activation scales and the training iteration.  The optimiser's state is saved by torch."""
    d = N.PolicyDesc()
    d.arch = arch
    d.n_layers = len(channels) - 1
    for k, c in enumerate(channels):
        d.channels[k] = int(c)
    d.head, d.precision = head, precision
    d.levels = levels if head == N.HT_HEAD_MULTITONE else 0
    w, b = _flat_f32(weights), _flat_f32(biases)
    sc = None if act_scales is None else np.ascontiguousarray(act_scales, np.float32)
    if sc is not None and sc.size != d.n_layers:
        raise ValueError(f"act_scales needs {d.n_layers} values")
    check(N.load().ht_checkpoint_save(os.fsencode(path), C.byref(d), w.ctypes.data, b.ctypes.data,
                                      None if sc is None else sc.ctypes.data, int(step)))


def load_checkpoint(path: str) -> dict:
    """ht_checkpoint_load.  Returns channels, head, precision, levels, arch, step,
    act_scales, the flat parameters (w_flat, b_flat), the per-layer weights (OIHW) and
    biases, and policy_kwargs such that Policy(**policy_kwargs) rebuilds the policy."""
    L = N.load()
    info = N.CheckpointInfo()
    check(L.ht_checkpoint_load(os.fsencode(path), C.byref(info), None, 0, None, 0))
    w = np.empty(info.n_weights, np.float32)
    b = np.empty(info.n_biases, np.float32)
    check(L.ht_checkpoint_load(os.fsencode(path), C.byref(info), w.ctypes.data, w.size, b.ctypes.data, b.size))
    d = info.desc
    chs = tuple(int(d.channels[k]) for k in range(d.n_layers + 1))
    ws, bs, ow, ob = [], [], 0, 0
    for l in range(d.n_layers):
        nw = chs[l + 1] * chs[l] * 9
        ws.append(w[ow:ow + nw].reshape(chs[l + 1], chs[l], 3, 3))
        bs.append(b[ob:ob + chs[l + 1]])
        ow, ob = ow + nw, ob + chs[l + 1]
    levels = d.levels if d.head == N.HT_HEAD_MULTITONE else 4
    out = dict(channels=chs, head=d.head, precision=d.precision, levels=levels, arch=d.arch, step=int(info.step),
               act_scales=[float(info.act_scale[l]) for l in range(d.n_layers)], w_flat=w, b_flat=b,
               weights=ws, biases=bs)
    out["policy_kwargs"] = dict(channels=chs, weights=ws, biases=bs, head=d.head, precision=d.precision,
                                levels=levels, arch=d.arch)
    return out


def sync(stream=None) -> None:
    check(N.load().ht_sync(_stream(stream)))


def unpack_bits(bits: torch.Tensor, h: int, w: int, head: int = N.HT_HEAD_SIGMOID) -> np.ndarray:
    """Host-side view of a packed halftone as uint8 levels [h][w] (tests and tools)."""
    b = bits.detach().cpu().numpy().view(np.uint32)
    if head == N.HT_HEAD_SIGMOID:
        x = np.arange(w)
        return ((b[:, x // 32] >> (x % 32).astype(np.uint32)) & 1).astype(np.uint8)
    x = np.arange(w)
    return ((b[:, x // 16] >> (2 * (x % 16)).astype(np.uint32)) & 3).astype(np.uint8)


def pack_bits(levels: np.ndarray, head: int = N.HT_HEAD_SIGMOID) -> np.ndarray:
    """Inverse of unpack_bits (host), returns int32 words [h][words]."""
    h, w = levels.shape
    per = 32 if head == N.HT_HEAD_SIGMOID else 16
    shift = 1 if head == N.HT_HEAD_SIGMOID else 2
    words = (w + per - 1) // per
    out = np.zeros((h, words), dtype=np.uint64)
    for x in range(w):
        out[:, x // per] |= levels[:, x].astype(np.uint64) << np.uint64(shift * (x % per))
    return out.astype(np.uint32).view(np.int32)
