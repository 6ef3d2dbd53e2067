"""ctypes loader and prototypes for libht.so (include/ht.h).

The library is built in-tree by paper_2304_12152_gb300.build; loading fails
loudly if it is missing -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

HT_MAX_LAYERS = 40
HT_OK, HT_ERR_INVALID_ARG, HT_ERR_UNSUPPORTED, HT_ERR_OOM, HT_ERR_CUDA, HT_ERR_TIMEOUT, HT_ERR_IO = range(7)
HT_FP32, HT_BF16, HT_FP8_E4M3, HT_FP16 = 0, 1, 2, 3
HT_HEAD_SIGMOID, HT_HEAD_SOFTMAX, HT_HEAD_MULTITONE = 0, 1, 2
HT_MODE_THRESHOLD, HT_MODE_BERNOULLI = 0, 1
HT_EST_LE, HT_EST_COMA = 0, 1
HT_ARCH_PLAIN, HT_ARCH_RESNET = 0, 1

# Every entry point declared in include/ht.h.
EXPORTS = (
    "ht_create_policy", "ht_destroy_policy", "ht_policy_set_weights", "ht_policy_set_act_scales",
    "ht_policy_calibrate",
    "ht_policy_num_params", "ht_policy_flops_per_px", "ht_bits_row_words", "ht_halftone",
    "ht_reward_opts_default", "ht_reward", "ht_reward_noalloc", "ht_toggle_delta", "ht_anisotropy_loss",
    "ht_plan_create", "ht_plan_launch", "ht_plan_destroy", "ht_policy_set_schedule", "ht_policy_autotune",
    "ht_train_create", "ht_train_destroy", "ht_train_step_fwd", "ht_train_step_bwd",
    "ht_checkpoint_save", "ht_checkpoint_load",
    "ht_profile_begin", "ht_profile_end", "ht_sync", "ht_last_error", "ht_version",
)


class PolicyDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("channels", C.c_int * (HT_MAX_LAYERS + 1)), ("head", C.c_int),
                ("precision", C.c_int), ("levels", C.c_int), ("arch", C.c_int)]


class Image(C.Structure):
    _fields_ = [("contone", C.c_void_p), ("h", C.c_int), ("w", C.c_int), ("pitch", C.c_int)]


class RewardOpts(C.Structure):
    _fields_ = [("sigma_hvs", C.c_float), ("sigma_ssim", C.c_float), ("k_contrast", C.c_float), ("w_s", C.c_float),
                ("c1", C.c_float), ("c2", C.c_float), ("radius", C.c_int), ("levels", C.c_int)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


class CheckpointInfo(C.Structure):
    _fields_ = [("desc", PolicyDesc), ("step", C.c_int64), ("n_weights", C.c_int64), ("n_biases", C.c_int64),
                ("act_scale", C.c_float * HT_MAX_LAYERS)]


class TuneResult(C.Structure):
    _fields_ = [("rows_per_unit", C.c_int), ("unit_order", C.c_int), ("cta_pair", C.c_int), ("ms", C.c_float)]


HT_TUNE_CANDIDATES = 18


class TrainDesc(C.Structure):
    _fields_ = [("max_crops", C.c_int), ("crop_h", C.c_int), ("crop_w", C.c_int), ("n_gray", C.c_int),
                ("gray_n", C.c_int), ("n_samples", C.c_int), ("las_mode", C.c_int), ("n_rad", C.c_int),
                ("n_ang", C.c_int), ("w_a", C.c_float), ("reward", RewardOpts), ("estimator", C.c_int),
                ("ckpt_stride", C.c_int)]


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libht.so (building it first if asked and needed).  HT_LIB_PATH selects
    a library built elsewhere (e.g. with other compile-time tile parameters)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("HT_LIB_PATH") or _build.LIB
        if not os.path.exists(path) and path != _build.LIB:
            raise RuntimeError(f"HT_LIB_PATH={path} does not exist")
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libht.so not built ({path}); run paper_2304_12152_gb300.build.build()")
            _build.build()
        L = C.CDLL(path)
        vp, i, i64, u64, f = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_float
        P = C.POINTER
        L.ht_create_policy.argtypes = [P(PolicyDesc), vp, vp, P(vp)]
        L.ht_destroy_policy.argtypes = [vp]
        L.ht_policy_set_weights.argtypes = [vp, vp, vp, vp]
        L.ht_policy_set_act_scales.argtypes = [vp, vp, i]
        L.ht_policy_calibrate.argtypes = [vp, P(Image), u64, vp]
        L.ht_policy_num_params.argtypes = [vp]
        L.ht_policy_num_params.restype = i64
        L.ht_policy_flops_per_px.argtypes = [vp]
        L.ht_policy_flops_per_px.restype = i64
        L.ht_bits_row_words.argtypes = [i, i]
        L.ht_halftone.argtypes = [vp, P(Image), i, i, u64, vp, vp, vp]
        L.ht_reward_opts_default.argtypes = [P(RewardOpts)]
        L.ht_reward_opts_default.restype = None
        L.ht_reward.argtypes = [P(Image), vp, i, P(RewardOpts), vp, vp]
        L.ht_reward_noalloc.argtypes = [P(Image), vp, i, P(RewardOpts), vp, vp]
        L.ht_toggle_delta.argtypes = [P(Image), vp, vp, i, P(RewardOpts), vp, vp]
        L.ht_anisotropy_loss.argtypes = [vp, i, i, i, i, i, vp, vp, vp]
        L.ht_plan_create.argtypes = [vp, P(Image), i, i, u64, vp, vp, P(vp)]
        L.ht_plan_launch.argtypes = [vp, vp]
        L.ht_plan_destroy.argtypes = [vp]
        L.ht_policy_set_schedule.argtypes = [vp, i, i, i]
        L.ht_policy_autotune.argtypes = [vp, P(Image), i, i, u64, vp, vp, i, P(TuneResult), i, P(i), vp]
        L.ht_train_create.argtypes = [vp, P(TrainDesc), P(vp)]
        L.ht_train_destroy.argtypes = [vp]
        L.ht_train_step_fwd.argtypes = [vp, P(Image), i, vp, u64, vp, vp]
        L.ht_train_step_bwd.argtypes = [vp, vp, vp, vp]
        L.ht_profile_begin.argtypes = []
        L.ht_profile_end.argtypes = [P(KernelStat), i, P(i)]
        L.ht_sync.argtypes = [vp]
        L.ht_checkpoint_save.argtypes = [C.c_char_p, P(PolicyDesc), vp, vp, vp, i64]
        L.ht_checkpoint_load.argtypes = [C.c_char_p, P(CheckpointInfo), vp, i64, vp, i64]
        L.ht_last_error.restype = C.c_char_p
        L.ht_version.restype = C.c_char_p
        _lib = L
        return L


class HTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ht status {status}: {msg}")
        self.status = status


def check(status: int) -> None:
    if status != HT_OK:
        raise HTError(status, load().ht_last_error().decode(errors="replace"))
