"""The packed halftone layout documented in include/ht.h, pinned on the host helpers the
GPU tests read the library's output with: 1 bit per pixel LSB-first, bit (x % 32) of word
(y * words + x / 32); 2 bits per pixel for the K-level heads at bits 2 (x % 16) ..
2 (x % 16) + 1; padding bits past w zero; words per row as ht_bits_row_words reports."""
import numpy as np
import pytest
import torch

from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api


@pytest.mark.parametrize("w", [1, 31, 32, 33, 100])
def test_single_pixel_words(w):
    h = 3
    for head, per, bits in ((N.HT_HEAD_SIGMOID, 32, 1), (N.HT_HEAD_SOFTMAX, 16, 2), (N.HT_HEAD_MULTITONE, 16, 2)):
        words = N.load().ht_bits_row_words(w, head)
        assert words == -(-w // per)
        for x in sorted({0, w // 2, w - 1}):
            lev = np.zeros((h, w), np.uint8)
            v = 1 if bits == 1 else 3 - (x % 3)          # some level in 1..3
            lev[1, x] = v
            packed = api.pack_bits(lev, head).view(np.uint32)
            assert packed.shape == (h, words)
            expect = np.zeros((h, words), np.uint64)
            expect[1, x // per] = v << (bits * (x % per))
            assert np.array_equal(packed.astype(np.uint64), expect), (head, w, x)


@pytest.mark.parametrize("w", [1, 17, 32, 33, 129])
def test_round_trip_and_zero_padding(w):
    rng = np.random.default_rng(w)
    h = 5
    for head, nlev, per, bits in ((N.HT_HEAD_SIGMOID, 2, 32, 1), (N.HT_HEAD_SOFTMAX, 4, 16, 2)):
        lev = rng.integers(0, nlev, (h, w)).astype(np.uint8)
        packed = api.pack_bits(lev, head)
        back = api.unpack_bits(torch.from_numpy(packed), h, w, head)
        assert np.array_equal(back, lev)
        used = w - (packed.shape[1] - 1) * per            # pixels in each row's last word
        last = packed.view(np.uint32)[:, -1].astype(np.uint64)
        assert np.all(last >> np.uint64(bits * used) == 0)
