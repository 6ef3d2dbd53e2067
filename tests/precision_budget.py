"""Error budget of the reduced-precision forms (analysis script, run by hand; not collected
by pytest).

Rebuilds the printer workload's policy (2 -> 64 x 7 -> 1, He-normal seed 1) as a float64
torch model on a 512 x 512 centre crop of its first image and applies the reduced-precision
rounding points one group at a time: the inner layers' weights, the inner layers' input
activations, both, in bf16, fp16 and e4m3 (per-output-channel weight scales amax / 448,
per-layer power-of-two activation scales from the crop).  Prints max, 99.9th percentile and
median of |p - p_fp64| away from the crop's 16-pixel border.

    python tests/precision_budget.py
"""
import os
import sys

import numpy as np
import torch
import torch.nn.functional as F

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle as O                                    # noqa: E402
from paper_2304_12152_gb300 import synth              # noqa: E402


def main():
    chs = synth.NET_WIDE
    ws, bs = synth.he_normal_policy(chs, 1)
    n = 512
    c = synth.contone_image(2048, 2048, seed=1, index=0)[768:768 + n, 768:768 + n]
    z = O.uniform_map(1, 0, 0, n, n)
    x0 = torch.from_numpy(np.stack([c.astype(np.float64), z]))[None]
    W = [torch.from_numpy(w.astype(np.float64)) for w in ws]
    B = [torch.from_numpy(b.astype(np.float64)) for b in bs]
    L = len(W)
    inner = lambda l: 0 < l < L - 1                  # noqa: E731  the 64 -> 64 layers

    def bf16(t, l=None):
        return t.float().to(torch.bfloat16).double()

    def fp16(t, l=None):
        return t.float().to(torch.float16).double()

    def e4m3(t):
        return t.clamp(-448, 448).float().to(torch.float8_e4m3fn).double()

    def w_e4m3(w, l=None):
        s = w.abs().amax(dim=(1, 2, 3), keepdim=True) / 448.0
        return e4m3(w / s) * s

    def forward(qw=None, qa=None):
        """qw(w, l): inner layers' weights; qa(x, l): inner layers' input activations."""
        x = x0
        for l in range(L):
            w = W[l]
            if inner(l):
                if qw:
                    w = qw(w, l)
                if qa:
                    x = qa(x, l)
            x = F.conv2d(x, w, B[l], padding=1)
            if l < L - 1:
                x = x.clamp_min(0)
        return torch.sigmoid(x)[0, 0].numpy()

    amax = {}

    def probe(x, l):
        amax[l] = float(x.abs().max())
        return x

    p64 = forward(qa=probe)
    sc = {l: 2.0 ** np.ceil(np.log2(max(a, 1e-6) / 448.0)) for l, a in amax.items()}

    def a_e4m3(x, l):
        return e4m3(x / sc[l]) * sc[l]

    rows = [
        ("bf16 weights and activations (the BF16 form)", bf16, bf16),
        ("bf16 weights only", bf16, None),
        ("bf16 activations only", None, bf16),
        ("fp16 weights and activations", fp16, fp16),
        ("e4m3 weights and activations (the FP8 form)", w_e4m3, a_e4m3),
        ("e4m3 weights only", w_e4m3, None),
        ("e4m3 activations only", None, a_e4m3),
        ("e4m3 inner layers 3-5, bf16 layers 2 and 6",
         lambda w, l: w_e4m3(w) if 1 < l < L - 2 else bf16(w), lambda x, l: a_e4m3(x, l) if 1 < l < L - 2 else bf16(x)),
    ]
    print(f"{'rounding points':48s} {'max':>9s} {'p99.9':>9s} {'median':>9s}")
    for name, qw, qa in rows:
        d = np.abs(forward(qw, qa) - p64)[16:-16, 16:-16]
        print(f"{name:48s} {d.max():9.2e} {np.quantile(d, 0.999):9.2e} {np.median(d):9.1e}")


if __name__ == "__main__":
    torch.set_num_threads(max(1, os.cpu_count() or 1))
    main()
