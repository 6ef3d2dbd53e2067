"""Policy checkpoints (host only, no GPU): round trips through the C ABI, the documented
file layout read back independently, the error paths (corrupt, truncated, forged or
foreign files, bad descriptors, short output arrays) and a stopped-and-resumed run."""
import os
import struct

import numpy as np
import pytest

from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth


def _fnv1a64(data: bytes) -> int:
    """FNV-1a, 64-bit (offset basis 14695981039346656037, prime 1099511628211)."""
    h = 0xCBF29CE484222325
    for x in data:
        h = ((h ^ x) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def _save(tmp_path, chs=synth.NET_WIDE, head=N.HT_HEAD_SIGMOID, precision=N.HT_BF16, levels=4,
          arch=N.HT_ARCH_PLAIN, step=1234, scales=None, seed=3, name="p.htck"):
    ws, bs = synth.he_normal_policy(chs, seed)
    rng = np.random.default_rng(seed)
    bs = [rng.normal(0, 0.1, b.shape).astype(np.float32) for b in bs]
    path = str(tmp_path / name)
    api.save_checkpoint(path, chs, ws, bs, head=head, precision=precision, levels=levels, arch=arch,
                        act_scales=scales, step=step)
    return path, ws, bs


def test_round_trip_bitwise(tmp_path):
    chs = synth.NET_WIDE
    scales = [1.0] + [2.0 ** -k for k in range(1, len(chs) - 2)] + [1.0]
    path, ws, bs = _save(tmp_path, chs, precision=N.HT_FP8_E4M3, scales=scales, step=200000)
    ck = api.load_checkpoint(path)
    assert ck["channels"] == tuple(chs) and ck["precision"] == N.HT_FP8_E4M3 and ck["head"] == N.HT_HEAD_SIGMOID
    assert ck["arch"] == N.HT_ARCH_PLAIN and ck["step"] == 200000
    assert ck["act_scales"] == scales
    for a, b in zip(ck["weights"], ws):
        assert a.shape == b.shape and np.array_equal(a.view(np.uint32), np.asarray(b, np.float32).view(np.uint32))
    for a, b in zip(ck["biases"], bs):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    kw = ck["policy_kwargs"]
    assert kw["channels"] == tuple(chs) and kw["precision"] == N.HT_FP8_E4M3 and len(kw["weights"]) == len(chs) - 1
    assert not os.path.exists(path + ".tmp")


def test_round_trip_other_heads_and_architectures(tmp_path):
    p1, _, _ = _save(tmp_path, synth.NET_WIDE, head=N.HT_HEAD_MULTITONE, levels=3, name="m.htck")
    c1 = api.load_checkpoint(p1)
    assert c1["head"] == N.HT_HEAD_MULTITONE and c1["levels"] == 3
    p2, _, _ = _save(tmp_path, synth.NET_WIDE_K4, head=N.HT_HEAD_SOFTMAX, name="s.htck")
    assert api.load_checkpoint(p2)["channels"][-1] == 4
    chs = (2,) + (32,) * 5 + (1,)            # stem, two residual blocks, output
    p3, ws, _ = _save(tmp_path, chs, arch=N.HT_ARCH_RESNET, name="r.htck")
    c3 = api.load_checkpoint(p3)
    assert c3["arch"] == N.HT_ARCH_RESNET and len(c3["weights"]) == len(ws)
    # FP32 form, non-64 widths (the small configuration)
    p4, _, _ = _save(tmp_path, synth.NET_SMALL, precision=N.HT_FP32, name="f.htck")
    assert api.load_checkpoint(p4)["channels"] == tuple(synth.NET_SMALL)


def test_file_layout_as_documented(tmp_path):
    chs = synth.NET_SMALL
    path, ws, bs = _save(tmp_path, chs, precision=N.HT_FP32, step=77, scales=[1.0] * (len(chs) - 1))
    raw = open(path, "rb").read()
    assert raw[:8] == b"HTCKPT01"
    (hlen,) = struct.unpack_from("<I", raw, 8)
    L = len(chs) - 1
    hdr = struct.unpack_from(f"<{L + 2}i4iq{L}fqq", raw, 12)
    assert struct.calcsize(f"<{L + 2}i4iq{L}fqq") == hlen
    assert hdr[0] == L and tuple(hdr[1:L + 2]) == tuple(chs)
    head, prec, levels, arch, step = hdr[L + 2:L + 7]
    assert (head, prec, arch, step) == (N.HT_HEAD_SIGMOID, N.HT_FP32, N.HT_ARCH_PLAIN, 77)
    nw, nb = hdr[-2:]
    assert nw == sum(chs[l + 1] * chs[l] * 9 for l in range(L)) and nb == sum(chs[1:])
    off = 12 + hlen
    w = np.frombuffer(raw, "<f4", nw, off)
    b = np.frombuffer(raw, "<f4", nb, off + 4 * nw)
    assert np.array_equal(w, np.concatenate([x.ravel() for x in ws]))
    assert np.array_equal(b, np.concatenate(bs))
    assert len(raw) == off + 4 * (nw + nb) + 8
    (ck,) = struct.unpack_from("<Q", raw, len(raw) - 8)
    assert ck == _fnv1a64(raw[:-8])


def _status(fn, *a, **k):
    with pytest.raises(N.HTError) as e:
        fn(*a, **k)
    return e.value.status, str(e.value)


def test_corrupt_truncated_and_foreign_files(tmp_path):
    path, _, _ = _save(tmp_path, synth.NET_SMALL, precision=N.HT_FP32)
    raw = bytearray(open(path, "rb").read())
    bad = tmp_path / "bad.htck"
    flipped = bytearray(raw)
    flipped[len(raw) // 2] ^= 0x01                       # one bit inside the weights
    bad.write_bytes(bytes(flipped))
    st, msg = _status(api.load_checkpoint, str(bad))
    assert st == N.HT_ERR_IO and "checksum" in msg
    bad.write_bytes(bytes(raw[:-100]))
    assert _status(api.load_checkpoint, str(bad))[0] == N.HT_ERR_IO
    bad.write_bytes(b"PK\x03\x04" + bytes(raw[4:]))
    st, msg = _status(api.load_checkpoint, str(bad))
    assert st == N.HT_ERR_IO and "tag" in msg
    bad.write_bytes(b"")
    assert _status(api.load_checkpoint, str(bad))[0] == N.HT_ERR_IO
    assert _status(api.load_checkpoint, str(tmp_path / "missing.htck"))[0] == N.HT_ERR_IO


def test_forged_header_with_valid_checksum_is_rejected(tmp_path):
    """A header whose parameter counts or descriptor do not describe a valid policy is
    refused even when the checksum matches."""
    path, _, _ = _save(tmp_path, synth.NET_SMALL, precision=N.HT_FP32)
    raw = bytearray(open(path, "rb").read()[:-8])
    (hlen,) = struct.unpack_from("<I", raw, 8)
    forged = tmp_path / "forged.htck"

    def write(body):
        forged.write_bytes(bytes(body) + struct.pack("<Q", _fnv1a64(bytes(body))))

    b1 = bytearray(raw)
    nw_off = 12 + hlen - 16
    struct.pack_into("<q", b1, nw_off, struct.unpack_from("<q", b1, nw_off)[0] + 1)
    write(b1)
    st, msg = _status(api.load_checkpoint, str(forged))
    assert st == N.HT_ERR_IO and "counts" in msg
    b2 = bytearray(raw)
    struct.pack_into("<i", b2, 16, 3)                    # channels[0] = 3: not (contone, noise)
    write(b2)
    st, msg = _status(api.load_checkpoint, str(forged))
    assert st == N.HT_ERR_IO and "descriptor" in msg
    write(raw + b"\0\0\0\0")                             # one float too many
    assert _status(api.load_checkpoint, str(forged))[0] == N.HT_ERR_IO


def test_save_argument_errors_and_atomic_replace(tmp_path):
    ws, bs = synth.he_normal_policy(synth.NET_SMALL, 1)
    path = str(tmp_path / "a.htck")
    bad_chs = (3,) + tuple(synth.NET_SMALL[1:])
    st, _ = _status(api.save_checkpoint, path, bad_chs, ws, bs)
    assert st == N.HT_ERR_INVALID_ARG and not os.path.exists(path)
    st, _ = _status(api.save_checkpoint, path, synth.NET_SMALL, ws, bs, precision=N.HT_BF16)   # 32-wide bf16
    assert st == N.HT_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        api.save_checkpoint(path, synth.NET_SMALL, ws, bs, act_scales=[1.0])
    api.save_checkpoint(path, synth.NET_SMALL, ws, bs, step=1)
    first = open(path, "rb").read()
    st, _ = _status(api.save_checkpoint, str(tmp_path / "no_such_dir" / "b.htck"), synth.NET_SMALL, ws, bs)
    assert st == N.HT_ERR_IO
    api.save_checkpoint(path, synth.NET_SMALL, ws, bs, step=2)
    assert open(path, "rb").read() != first and api.load_checkpoint(path)["step"] == 2
    assert not os.path.exists(path + ".tmp")


def test_load_capacity_and_header_only_query(tmp_path):
    import ctypes as C
    path, _, _ = _save(tmp_path, synth.NET_SMALL, precision=N.HT_FP32)
    L = N.load()
    info = N.CheckpointInfo()
    assert L.ht_checkpoint_load(os.fsencode(path), C.byref(info), None, 0, None, 0) == N.HT_OK
    nw, nb = info.n_weights, info.n_biases
    w = np.empty(nw, np.float32)
    b = np.empty(nb, np.float32)
    assert L.ht_checkpoint_load(os.fsencode(path), C.byref(info), w.ctypes.data, nw - 1, b.ctypes.data,
                                nb) == N.HT_ERR_INVALID_ARG
    assert L.ht_checkpoint_load(os.fsencode(path), C.byref(info), w.ctypes.data, nw, None, 0) == N.HT_ERR_INVALID_ARG
    assert L.ht_checkpoint_load(None, C.byref(info), None, 0, None, 0) == N.HT_ERR_INVALID_ARG
    assert L.ht_checkpoint_load(os.fsencode(path), None, None, 0, None, 0) == N.HT_ERR_INVALID_ARG


def test_resume_continues_a_run_bit_for_bit(tmp_path):
    """The resume workflow: master weights, FP8 scales and the step go through the library's
    checkpoint, the optimiser's state through torch.save; a run stopped after 3 steps and
    resumed reaches the same weights, bit for bit, as one run of 6 steps (a deterministic
    stand-in gradient replaces the training step, which needs the GPU)."""
    import torch
    chs = synth.NET_SMALL
    ws, bs = synth.he_normal_policy(chs, 2)
    w0 = torch.from_numpy(np.concatenate([w.ravel() for w in ws]))
    b0 = torch.from_numpy(np.concatenate(bs))

    def grads(w, b, step):
        g = torch.Generator().manual_seed(1000 + step)
        return (torch.sin(w * 3.0) + 0.01 * torch.randn(w.shape, generator=g),
                torch.cos(b) + 0.01 * torch.randn(b.shape, generator=g))

    def run(w, b, opt, steps, first):
        for step in range(first, first + steps):
            gw, gb = grads(w.detach(), b.detach(), step)
            w.grad, b.grad = gw, gb
            opt.step()

    w, b = w0.clone().requires_grad_(True), b0.clone().requires_grad_(True)
    opt = torch.optim.Adam([w, b], lr=1e-3)
    run(w, b, opt, 6, 0)
    w_ref, b_ref = w.detach().clone(), b.detach().clone()

    w, b = w0.clone().requires_grad_(True), b0.clone().requires_grad_(True)
    opt = torch.optim.Adam([w, b], lr=1e-3)
    run(w, b, opt, 3, 0)
    path = str(tmp_path / "run.htck")
    api.save_checkpoint(path, chs, w, b, precision=N.HT_FP32, step=3)
    torch.save(opt.state_dict(), str(tmp_path / "opt.pt"))
    del w, b, opt

    ck = api.load_checkpoint(path)
    w = torch.from_numpy(ck["w_flat"].copy()).requires_grad_(True)
    b = torch.from_numpy(ck["b_flat"].copy()).requires_grad_(True)
    opt = torch.optim.Adam([w, b], lr=1e-3)
    opt.load_state_dict(torch.load(str(tmp_path / "opt.pt")))
    run(w, b, opt, 6 - ck["step"], ck["step"])
    assert torch.equal(w.detach(), w_ref) and torch.equal(b.detach(), b_ref)
