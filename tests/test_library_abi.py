"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/ht.h declares; host-side argument checks need no GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2304_12152_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ht.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ht_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    L = N.load()
    decl = _declared()
    assert len(decl) >= 15
    missing = [s for s in decl if not hasattr(L, s)]
    assert not missing, missing
    assert set(decl) == set(N.EXPORTS)


def test_host_only_calls():
    L = N.load()
    assert L.ht_version().startswith(b"ht ")
    assert L.ht_bits_row_words(1, 0) == 1 and L.ht_bits_row_words(33, 0) == 2 and L.ht_bits_row_words(17, 1) == 2
    o = N.RewardOpts()
    L.ht_reward_opts_default(C.byref(o))
    assert o.radius == 5 and abs(o.w_s - 0.06) < 1e-7 and abs(o.sigma_hvs - 2.0) < 1e-7


@pytest.mark.parametrize("chs,head,prec,status", [
    ((2, 4, 1), 0, N.HT_FP32, None),             # valid (would need a GPU) -> skipped below
    ((3, 4, 1), 0, N.HT_FP32, N.HT_ERR_INVALID_ARG),
    ((2, 4, 2), 0, N.HT_FP32, N.HT_ERR_INVALID_ARG),
    ((2, 4, 1), 1, N.HT_FP32, N.HT_ERR_INVALID_ARG),
    ((2, 65, 1), 0, N.HT_FP32, N.HT_ERR_INVALID_ARG),
    ((2, 32, 32, 1), 0, N.HT_BF16, N.HT_ERR_UNSUPPORTED),
    ((2, 64, 1), 0, N.HT_BF16, N.HT_ERR_UNSUPPORTED),
])
def test_policy_descriptor_validation(chs, head, prec, status):
    if status is None:
        pytest.skip("valid descriptor needs a device")
    L = N.load()
    d = N.PolicyDesc()
    d.n_layers = len(chs) - 1
    for i, c in enumerate(chs):
        d.channels[i] = c
    d.head, d.precision = head, prec
    w = (C.c_float * 100000)()
    h = C.c_void_p()
    assert L.ht_create_policy(C.byref(d), w, w, C.byref(h)) == status
    assert not h.value
    assert len(L.ht_last_error()) > 0


def test_argument_errors_before_launch():
    L = N.load()
    o = N.RewardOpts()
    L.ht_reward_opts_default(C.byref(o))
    img = (N.Image * 1)(N.Image(None, 8, 8, 8))
    assert L.ht_reward(img, None, 1, C.byref(o), None, None) == N.HT_ERR_INVALID_ARG
    assert L.ht_anisotropy_loss(None, 1, 16, 0, 0, 0, None, None, None) == N.HT_ERR_INVALID_ARG
    q = C.c_void_p(16)
    assert L.ht_anisotropy_loss(q, 1, 12, 0, 0, 0, q, None, None) == N.HT_ERR_INVALID_ARG
    o.radius = 9
    img2 = (N.Image * 1)(N.Image(16, 20, 20, 20))
    assert L.ht_reward(img2, q, 1, C.byref(o), q, None) == N.HT_ERR_INVALID_ARG


def test_null_handles_and_out_of_range_arguments():
    """Every entry point that takes a handle refuses a null one before touching the device,
    with a message; destroying a null handle is a no-op."""
    L = N.load()
    vp = C.c_void_p
    img = (N.Image * 1)(N.Image(16, 8, 8, 8))
    bits = (vp * 1)(16)
    out = vp()
    res = (N.TuneResult * N.HT_TUNE_CANDIDATES)()
    nres = C.c_int()
    losses = (C.c_double * 4)()
    sc = (C.c_float * 8)(*([1.0] * 8))
    calls = [
        lambda: L.ht_halftone(None, img, 1, 0, 0, bits, None, None),
        lambda: L.ht_plan_create(None, img, 1, 0, 0, bits, None, C.byref(out)),
        lambda: L.ht_plan_create(vp(16), img, 1, 0, 0, bits, None, None),
        lambda: L.ht_plan_launch(None, None),
        lambda: L.ht_policy_set_weights(None, vp(16), vp(16), None),
        lambda: L.ht_policy_set_act_scales(None, sc, 8),
        lambda: L.ht_policy_calibrate(None, img, 0, None),
        lambda: L.ht_policy_set_schedule(None, 8, 0, 0),
        lambda: L.ht_policy_autotune(None, img, 1, 0, 0, bits, None, 1, res, N.HT_TUNE_CANDIDATES, C.byref(nres), None),
        lambda: L.ht_train_create(None, None, C.byref(out)),
        lambda: L.ht_train_step_fwd(None, img, 1, None, 0, losses, None),
        lambda: L.ht_train_step_bwd(None, vp(16), vp(16), None),
    ]
    for k, call in enumerate(calls):
        assert call() == N.HT_ERR_INVALID_ARG, k
        assert len(L.ht_last_error()) > 0, k
    assert not out.value
    assert L.ht_destroy_policy(None) == N.HT_OK
    assert L.ht_plan_destroy(None) == N.HT_OK
    assert L.ht_train_destroy(None) == N.HT_OK


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without the CUDA library the binding and the public API raise, naming
    the missing file (checked in a fresh interpreter with HT_LIB_PATH at a missing path)."""
    import subprocess
    import sys
    code = (
        "from paper_2304_12152_gb300 import _native as N, api, synth\n"
        "for f in (N.load, lambda: api.Policy(synth.NET_SMALL, *synth.he_normal_policy(synth.NET_SMALL, 0))):\n"
        "    try:\n"
        "        f()\n"
        "        print('NO ERROR')\n"
        "    except RuntimeError as e:\n"
        "        print('RAISED', e)\n")
    env = dict(os.environ, HT_LIB_PATH=str(tmp_path / "missing_libht.so"))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    lines = r.stdout.strip().splitlines()
    assert len(lines) == 2 and all(ln.startswith("RAISED") and "missing_libht.so" in ln for ln in lines), r.stdout + r.stderr


@pytest.mark.parametrize("fn", ["ht_reward", "ht_reward_noalloc"])
@pytest.mark.parametrize("levels", [0, 1, 5, -3])
def test_reward_entry_points_refuse_bad_levels(fn, levels):
    """Both reward entry points run the same option checks before any CUDA call: a level
    count outside [2, 4] is an argument error (the kernels divide by levels - 1)."""
    L = N.load()
    o = N.RewardOpts()
    L.ht_reward_opts_default(C.byref(o))
    o.levels = levels
    img = (N.Image * 1)(N.Image(16, 20, 20, 20))
    bits = (C.c_void_p * 1)(16)
    st = getattr(L, fn)(img, bits, 1, C.byref(o), C.c_void_p(16), None)
    assert st == N.HT_ERR_INVALID_ARG and b"levels" in L.ht_last_error()


def test_noalloc_reward_source_names_no_allocator():
    """The allocation-free reward and the launcher it shares with ht_reward name no
    allocating routine (a later edit adding one fails here, without a GPU)."""
    src = open(os.path.join(ROOT, "paper_2304_12152_gb300", "csrc", "reward.cu")).read()
    body = src[src.index('extern "C" ht_status ht_reward_noalloc'):]
    body = body[:body.index("\n}\n")]
    launcher = src[src.index("ht_status launch_reward_tiles("):]
    launcher = launcher[:launcher.index("\n}\n")]
    for part in (body, launcher):
        code = re.sub(r"//.*", "", part)
        for name in ("cudaMalloc", "cudaFree", "cudaMallocAsync", "cudaFreeAsync", "malloc(", "new ",
                     "ht_device_error_flag", "ht_policy_ensure_ws"):
            assert name not in code, name
