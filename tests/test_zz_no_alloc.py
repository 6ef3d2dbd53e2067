"""ht_reward_noalloc: the allocation-free reward for callers that must not allocate
device memory while they run (an application whose own allocator reserved the device
memory it may use, or a streaming loop that cannot take the synchronisation cudaMalloc
or cudaFree may imply).  Called through the C ABI, twice in a row on different
inputs, its results must equal ht_reward's within the reward parity tolerance
(MSE 1e-5 relative, SSIM / CSSIM 2e-5 absolute, R 2e-6 absolute): the second call
also shows that the shared device array is cleared between calls.  Batches of 70
uneven images cross the 32-image tile launches and the 64-image finishing launches;
a 4-level case runs the multi-level path.  A call makes no device allocation: neither
the free device memory nor the high-water mark of the device's default memory pool
moves (ht_reward, which allocates its accumulators from that pool, is the positive
control).  This file is collected last so that a run stopping at its first failure has
run everything else."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _inputs(seed, shapes, levels=2):
    imgs = [synth.contone_image(h, w, seed=seed, index=i) for i, (h, w) in enumerate(shapes)]
    rng = np.random.default_rng(seed)
    head = N.HT_HEAD_SIGMOID if levels == 2 else N.HT_HEAD_SOFTMAX
    if levels == 2:
        hts = [(rng.random(c.shape) < c).astype(np.uint8) for c in imgs]
    else:
        hts = [np.clip(np.floor(c * (levels - 1) + rng.random(c.shape)), 0, levels - 1).astype(np.uint8)
               for c in imgs]
    cs = [torch.from_numpy(c).cuda() for c in imgs]
    bits = [torch.from_numpy(api.pack_bits(h, head)).cuda() for h in hts]
    return cs, bits


def _call(fn, cs, bits, levels=2, out=None):
    L = N.load()
    o = N.RewardOpts()
    L.ht_reward_opts_default(C.byref(o))
    o.levels = levels
    if out is None:
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


def _uneven(n, seed):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(16, 41)), int(rng.integers(16, 41))) for _ in range(n)]


CASES = [(41, [(64, 64), (100, 37), (11, 11)], 2), (42, [(256, 256), (33, 300)], 2),
         (44, _uneven(70, 44), 2), (45, _uneven(70, 45), 4), (46, [(64, 80), (31, 47)], 4)]


def test_noalloc_reward_matches_allocating_reward_twice():
    for levels in (2, 4):
        runs = [(seed, shapes) for seed, shapes, lv in CASES if lv == levels]
        for seed, shapes in runs:            # consecutive calls on different inputs
            cs, bits = _inputs(seed, shapes, levels)
            ref = _call("ht_reward", cs, bits, levels)
            got = _call("ht_reward_noalloc", cs, bits, levels)
            assert np.all(np.isfinite(got))
            _close(got, ref)


class _Pool:
    """The device's default memory pool through the driver API (read-only use, apart from
    resetting the pool's own used-memory high-water mark)."""
    USED_MEM_HIGH = 8           # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def __init__(self):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int()
        assert self.cu.cuCtxGetDevice(C.byref(dev)) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def reset_high(self):
        z = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, C.byref(z)) == 0

    def high(self):
        v = C.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, self.USED_MEM_HIGH, C.byref(v)) == 0
        return v.value


def test_noalloc_reward_allocates_nothing():
    cs, bits = _inputs(47, _uneven(40, 47))
    out = torch.empty((len(cs), 4), dtype=torch.float64, device="cuda")
    _call("ht_reward_noalloc", cs, bits, out=out)        # kernels loaded, address looked up
    _call("ht_reward", cs, bits, out=out)
    pool = _Pool()
    torch.cuda.synchronize()
    pool.reset_high()
    _call("ht_reward", cs, bits, out=out)                # positive control: allocates from the pool
    assert pool.high() > 0
    torch.cuda.synchronize()
    pool.reset_high()
    free0 = torch.cuda.mem_get_info()[0]
    _call("ht_reward_noalloc", cs, bits, out=out)
    free1 = torch.cuda.mem_get_info()[0]
    assert pool.high() == 0 and free1 == free0


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
