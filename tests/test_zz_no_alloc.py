"""ht_reward_noalloc: the allocation-free reward for callers that must not allocate
device memory while they run (an application whose own allocator reserved the device
memory it may use, or a streaming loop that cannot take the synchronisation cudaMalloc
or cudaFree may imply).  Called through the C ABI, twice in a row on different
inputs, its results must equal ht_reward's within the reward parity tolerance
(MSE 1e-5 relative, SSIM / CSSIM 2e-5 absolute, R 2e-6 absolute): the second call
also shows that the shared device array is cleared between calls.  This file is
collected last so that a run stopping at its first failure has run everything else."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _inputs(seed, shapes):
    imgs = [synth.contone_image(h, w, seed=seed, index=i) for i, (h, w) in enumerate(shapes)]
    rng = np.random.default_rng(seed)
    hts = [(rng.random(c.shape) < c).astype(np.uint8) for c in imgs]
    cs = [torch.from_numpy(c).cuda() for c in imgs]
    bits = [torch.from_numpy(api.pack_bits(h)).cuda() for h in hts]
    return cs, bits


def _call(fn, cs, bits):
    L = N.load()
    o = N.RewardOpts()
    L.ht_reward_opts_default(C.byref(o))
    out = torch.full((len(cs), 4), float("nan"), dtype=torch.float64, device="cuda")
    imgs = (N.Image * len(cs))(*[N.Image(c.data_ptr(), c.shape[0], c.shape[1], c.stride(0)) for c in cs])
    ptrs = (C.c_void_p * len(bits))(*[b.data_ptr() for b in bits])
    st = getattr(L, fn)(imgs, ptrs, len(cs), C.byref(o), C.c_void_p(out.data_ptr()),
                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == N.HT_OK, L.ht_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _close(a, b):
    assert np.all(np.abs(a[:, 0] - b[:, 0]) <= 1e-5 * np.abs(b[:, 0]) + 1e-9)
    assert np.all(np.abs(a[:, 1:3] - b[:, 1:3]) < 2e-5)
    assert np.all(np.abs(a[:, 3] - b[:, 3]) < 2e-6)


def test_noalloc_reward_matches_allocating_reward_twice():
    for seed, shapes in [(41, [(64, 64), (100, 37), (11, 11)]), (42, [(256, 256), (33, 300)])]:
        cs, bits = _inputs(seed, shapes)
        ref = _call("ht_reward", cs, bits)
        got = _call("ht_reward_noalloc", cs, bits)
        assert np.all(np.isfinite(got))
        _close(got, ref)


def test_noalloc_reward_rejects_too_many_images():
    L = N.load()
    o = N.RewardOpts()
    L.ht_reward_opts_default(C.byref(o))
    cs, bits = _inputs(43, [(16, 16)])
    k = 1025
    imgs = (N.Image * k)(*[N.Image(cs[0].data_ptr(), 16, 16, 16)] * k)
    ptrs = (C.c_void_p * k)(*[bits[0].data_ptr()] * k)
    out = torch.empty((k, 4), dtype=torch.float64, device="cuda")
    st = L.ht_reward_noalloc(imgs, ptrs, k, C.byref(o), C.c_void_p(out.data_ptr()), None)
    assert st == N.HT_ERR_INVALID_ARG and b"at most" in L.ht_last_error()
