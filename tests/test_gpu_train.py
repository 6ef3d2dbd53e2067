"""GPU parity of one training iteration (Algorithm 1, TRAIN) against the FP64 oracle.

The oracle side is assembled from the pinned oracle routines: forward with saved
activations, Bernoulli samples h^s = [u^s < p] with u^s from the oracle's Philox
(stream 1 + s), reward and toggle deltas per sample, the local-expectation surrogate
(value and dL/dp = -dR), the anisotropy loss of the gray patches' probability maps
with its gradient, and the hand-written backward (pinned by finite differences and
torch autograd in the CPU tests).  Tolerances: losses 1e-4 relative, gradients 2e-3
of the largest gradient entry of the layer (FP32 forward, FP32 dR sums)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_12152_gb300 import _native as N
from paper_2304_12152_gb300 import api, synth

pytestmark = pytest.mark.gpu


def oracle_step(crops, grays, ws, bs, seed, S, w_a, las_mode, n_rad, n_ang, quant=0, coma=False):
    n, G = len(crops), len(grays)
    gw = [np.zeros(w.shape) for w in ws]
    gb = [np.zeros(b.shape) for b in bs]
    l_marl, rs = 0.0, []
    for i, c in enumerate(crops):
        h, w = c.shape
        lg, p, acts = O.forward(c, ws, bs, noise_seed=seed, image=i, quant=quant, save_acts=True)
        dp = np.zeros((h, w))
        for s in range(S):
            u = O.uniform_map(seed, i, 1 + s, h, w)
            hb = (u < p[0]).astype(np.uint8)
            r = O.reward(c, hb)
            dR = O.toggle_delta(c, hb).reshape(h, w)
            val, grad = (O.coma_surrogate if coma else O.le_surrogate)(p[0], hb, dR, r["R"])
            l_marl += val / (n * S)
            dp += grad / (n * S)
            rs.append(r["R"])
        a, b = O.backward(c, ws, bs, seed, i, acts, lg, dp, quant=quant)
        for l in range(len(ws)):
            gw[l] += a[l]
            gb[l] += b[l]
    l_as = 0.0
    for g, (lev, nn) in enumerate(grays):
        c = np.full((nn, nn), lev, np.float32)
        lg, p, acts = O.forward(c, ws, bs, noise_seed=seed, image=n + g, quant=quant, save_acts=True)
        r = O.anisotropy_loss(p[0], mode=las_mode, n_rad=n_rad, n_ang=n_ang, grad=True)
        l_as += r["loss"] / G
        a, b = O.backward(c, ws, bs, seed, n + g, acts, lg, w_a * r["grad"] / G, quant=quant)
        for l in range(len(ws)):
            gw[l] += a[l]
            gb[l] += b[l]
    return l_marl + w_a * l_as, l_marl, l_as, float(np.mean(rs)) if rs else 0.0, gw, gb


@pytest.mark.parametrize("las_mode,n_rad,n_ang", [(0, 1, 1), (1, 4, 4)])
def test_train_step_matches_oracle(las_mode, n_rad, n_ang):
    chs = (2, 8, 8, 1)
    ws, _ = synth.he_normal_policy(chs, 21)
    bs = synth.random_biases(chs, 22, scale=0.1)
    crops = [synth.contone_image(32, 32, seed=23, index=i) for i in range(2)]
    levels = [0.25, 0.6]
    gn, S, seed, w_a = 16, 2, 7, 0.5
    pol = api.Policy(chs, ws, bs, precision=N.HT_FP32)
    tr = api.Trainer(pol, (32, 32), max_crops=2, n_samples=S, n_gray=2, gray_n=gn, las_mode=las_mode,
                     n_rad=n_rad, n_ang=n_ang, w_a=w_a)
    losses = tr.forward([torch.from_numpy(c).cuda() for c in crops], levels, seed)
    gw, gb = tr.backward()
    torch.cuda.synchronize()
    ref = oracle_step(crops, [(l, gn) for l in levels], ws, bs, seed, S, w_a, las_mode, n_rad, n_ang)
    for k in range(4):
        assert abs(losses[k] - ref[k]) <= 1e-4 * abs(ref[k]) + 1e-9, (k, losses, ref[:4])
    gw = gw.cpu().numpy().astype(np.float64)
    gb = gb.cpu().numpy().astype(np.float64)
    ow = ob = 0
    for l in range(len(ws)):
        rw, rb = ref[4][l].ravel(), ref[5][l].ravel()
        scale = max(np.abs(rw).max(), np.abs(rb).max())
        assert np.abs(gw[ow:ow + rw.size] - rw).max() <= 2e-3 * scale, l
        assert np.abs(gb[ob:ob + rb.size] - rb).max() <= 2e-3 * scale, l
        ow += rw.size
        ob += rb.size


def test_coma_train_step_matches_oracle():
    """FP32 step with the COMA estimator (Eq. coma) against the oracle's COMA surrogate:
    same tolerances as the local-expectation step."""
    chs = (2, 8, 8, 1)
    ws, _ = synth.he_normal_policy(chs, 71)
    bs = synth.random_biases(chs, 72, scale=0.1)
    crops = [synth.contone_image(32, 40, seed=73, index=i) for i in range(2)]
    S, seed = 3, 13
    pol = api.Policy(chs, ws, bs, precision=N.HT_FP32)
    tr = api.Trainer(pol, (32, 40), max_crops=2, n_samples=S, n_gray=0, las_mode=1, n_rad=4, n_ang=4, w_a=0.0,
                     estimator=N.HT_EST_COMA)
    losses = tr.forward([torch.from_numpy(c).cuda() for c in crops], [], seed)
    gw, gb = tr.backward()
    torch.cuda.synchronize()
    ref = oracle_step(crops, [], ws, bs, seed, S, 0.0, 1, 4, 4, coma=True)
    assert abs(losses[1] - ref[1]) <= 1e-4 * abs(ref[1]) + 1e-9, (losses, ref[:4])
    errs = _grad_errors(gw, gb, ref[4], ref[5])
    for ew, eb in errs:
        assert ew <= 2e-3 and eb <= 2e-3, errs


def oracle_step_multitone(crops, ws, bs, seed, S, L, quant=0, band=0.0):
    """Training step of the multitoning prototype (Sec. VI-E) from oracle routines:
    levels h^s sampled from v with u^s (stream 1 + s), reward and toggle deltas of the
    multi-level halftones, the LE surrogate with dL/dv = -(L - 1) dR, the backward.
    With band > 0 it also returns the flip bound: the mean over crops and samples of
    sum |dR_a| over the pixels whose action a form with |dv| <= band may take the other
    way (|frac - u| or the distance of v (L - 1) from a level within (L - 1) band)."""
    n = len(crops)
    gw = [np.zeros(w.shape) for w in ws]
    gb = [np.zeros(b.shape) for b in bs]
    l_marl, rs, flip = 0.0, [], 0.0
    for i, c in enumerate(crops):
        h, w = c.shape
        lg, p, acts = O.forward(c, ws, bs, noise_seed=seed, image=i, quant=quant, save_acts=True)
        v = p[0]
        k, _ = O.multitone_pair(v, L)
        dp = np.zeros((h, w))
        for s in range(S):
            u = O.uniform_map(seed, i, 1 + s, h, w)
            lev = O.sample_multitone(v, L, u)
            r = O.reward(c, lev, levels=L)
            dR = O.toggle_delta(c, lev, levels=L, lo=k.astype(np.uint8)).reshape(h, w)
            val, grad = O.le_surrogate_multitone(v, lev, dR, r["R"], L)
            l_marl += val / (n * S)
            dp += grad / (n * S)
            rs.append(r["R"])
            if band > 0:
                t = v * (L - 1)
                _, frac = O.multitone_pair(v, L)
                near = (np.abs(frac - u) <= (L - 1) * band) | (np.abs(t - np.rint(t)) <= (L - 1) * band)
                flip += float(np.abs(dR[near]).sum()) / (n * S)
        a, b = O.backward(c, ws, bs, seed, i, acts, lg, dp, quant=quant)
        for l in range(len(ws)):
            gw[l] += a[l]
            gb[l] += b[l]
    if band > 0:
        return l_marl, float(np.mean(rs)), gw, gb, flip
    return l_marl, float(np.mean(rs)), gw, gb


def test_multitone_train_step_matches_oracle():
    """FP32 training step of the multitoning prototype (4 levels) against the oracle:
    losses 1e-4 relative, gradients 2e-3 of the layer's largest entry."""
    chs, L = (2, 8, 8, 1), 4
    ws, _ = synth.he_normal_policy(chs, 81)
    bs = synth.random_biases(chs, 82, scale=0.1)
    crops = [synth.contone_image(28, 44, seed=83, index=i) for i in range(2)]
    S, seed = 2, 17
    pol = api.Policy(chs, ws, bs, head=N.HT_HEAD_MULTITONE, precision=N.HT_FP32, levels=L)
    tr = api.Trainer(pol, (28, 44), max_crops=2, n_samples=S, n_gray=0, las_mode=1, n_rad=4, n_ang=4, w_a=0.0)
    losses = tr.forward([torch.from_numpy(c).cuda() for c in crops], [], seed)
    gw, gb = tr.backward()
    torch.cuda.synchronize()
    l_marl, r_mean, ref_w, ref_b = oracle_step_multitone(crops, ws, bs, seed, S, L)
    assert abs(losses[1] - l_marl) <= 1e-4 * abs(l_marl), (losses, l_marl)
    assert abs(losses[3] - r_mean) <= 1e-4 * abs(r_mean), (losses, r_mean)
    errs = _grad_errors(gw, gb, ref_w, ref_b)
    for ew, eb in errs:
        assert ew <= 2e-3 and eb <= 2e-3, errs


def test_bf16_multitone_train_step_matches_bf16_oracle():
    """BF16 tensor-core training of the multitoning prototype (4 levels) against the
    quant-1 oracle.  As in the binary BF16 step, samples flip where the level rule's
    margin is below the forward error (L - 1 times more often than for the binary rule).
    A flip of pixel a moves that sample's reward by its toggle delta dR_a and L_MARL by
    about (h w) dR_a, so the mean reward is held to the oracle's flip bound (the sum of
    |dR_a| over the pixels within (L - 1) x 2e-3 of a decision, 2e-3 being the 99.9th
    percentile bound on |dv| of the 7-layer BF16 rule in tests/_cases.TIGHT), with 1.5x
    for flips that share a window, and L_MARL to h w times that; gradients 4e-2 of the
    layer's largest entry."""
    L = 4
    ws, _ = synth.he_normal_policy(WIDE4, 91)
    bs = synth.random_biases(WIDE4, 92, scale=0.1)
    crops = [synth.contone_image(40, 150, seed=93, index=i) for i in range(2)]
    S, seed = 2, 19
    pol = api.Policy(WIDE4, ws, bs, head=N.HT_HEAD_MULTITONE, precision=N.HT_BF16, levels=L)
    tr = api.Trainer(pol, (40, 150), max_crops=2, n_samples=S, n_gray=0, las_mode=1, n_rad=4, n_ang=4, w_a=0.0)
    losses = tr.forward([torch.from_numpy(c).cuda() for c in crops], [], seed)
    gw, gb = tr.backward()
    torch.cuda.synchronize()
    l_marl, r_mean, ref_w, ref_b, flip = oracle_step_multitone(crops, ws, bs, seed, S, L, quant=1, band=2e-3)
    errs = _grad_errors(gw, gb, ref_w, ref_b)
    print("multitone bf16: losses", losses, l_marl, r_mean, "flip bound", flip, "errors", errs)
    npx = crops[0].size
    assert abs(losses[3] - r_mean) <= 1.5 * flip + 1e-9, (losses, r_mean, flip)
    assert abs(losses[1] - l_marl) <= 1.5 * npx * flip + 1e-6 * abs(l_marl), (losses, l_marl, flip)
    for ew, eb in errs:
        assert ew <= 4e-2 and eb <= 4e-2, errs


def test_autograd_function_drives_adam():
    """torch.autograd.Function wrapper: gradients reach torch parameters and an Adam
    step changes the loss deterministically."""
    chs = (2, 8, 8, 1)
    ws, bs = synth.he_normal_policy(chs, 31)
    pol = api.Policy(chs, ws, bs, precision=N.HT_FP32)
    tr = api.Trainer(pol, (24, 24), max_crops=2, n_samples=2, n_gray=1, gray_n=16, las_mode=1, n_rad=4, n_ang=4)
    w = torch.nn.Parameter(torch.from_numpy(np.concatenate([x.ravel() for x in ws])).cuda())
    b = torch.nn.Parameter(torch.from_numpy(np.concatenate([x.ravel() for x in bs])).cuda())
    crops = [torch.from_numpy(synth.contone_image(24, 24, seed=32, index=i)).cuda() for i in range(2)]
    opt = torch.optim.Adam([w, b], lr=1e-3)
    loss = api.HalftonePolicyFn.apply(w, b, tr, crops, [0.5], 3)
    loss.backward()
    assert w.grad is not None and torch.isfinite(w.grad).all() and w.grad.abs().sum() > 0
    opt.step()
    loss2 = api.HalftonePolicyFn.apply(w, b, tr, crops, [0.5], 3)
    assert torch.isfinite(loss2) and float(loss2) != float(loss)


def _grad_errors(gw, gb, ref_w, ref_b):
    """Per layer: max |error| of the weight and of the bias gradient, each over the
    layer's largest reference gradient entry."""
    gw = gw.cpu().numpy().astype(np.float64)
    gb = gb.cpu().numpy().astype(np.float64)
    ow = ob = 0
    errs = []
    for rw, rb in zip(ref_w, ref_b):
        rw, rb = rw.ravel(), rb.ravel()
        scale = max(np.abs(rw).max(), np.abs(rb).max())
        errs.append((np.abs(gw[ow:ow + rw.size] - rw).max() / scale, np.abs(gb[ob:ob + rb.size] - rb).max() / scale))
        ow += rw.size
        ob += rb.size
    return errs


WIDE4 = (2, 64, 64, 64, 1)      # layer 1, a 64 -> 64 layer, the 64 -> 64 layer with the head partials, head


def test_bf16_backward_anisotropy_only_matches_bf16_oracle():
    """BF16 tensor-core backward without sampling: a step on two 128 x 128 gray patches
    only, so dL/dp is w_a dL_AS/dp of the probability maps and every pass (head
    backward, tcgen05 weight gradients, data gradients on the conv pipeline, layer-1
    weight gradient) is compared with the oracle's quant-1 backward.  The remaining
    differences start in the forward: where an activation's FP32 sum (GPU) and FP64 sum
    (oracle) straddle a bf16 rounding boundary the two sides store values one bf16 ulp
    apart, and through the depth of the net p differs by ~5e-4 typically, 4e-3 at most
    (the BF16 forward bounds).  dL_AS/dp and the gradients inherit a relative
    difference of that size: tolerance 3e-4 on L_AS and 6e-3 of the layer's largest
    gradient entry (measured 9e-5 and 0.04-0.34%)."""
    ws, _ = synth.he_normal_policy(WIDE4, 61)
    bs = synth.random_biases(WIDE4, 62, scale=0.1)
    levels = [0.35, 0.8]
    gn, seed, w_a = 128, 11, 1.0
    pol = api.Policy(WIDE4, ws, bs, precision=N.HT_BF16)
    tr = api.Trainer(pol, (16, 16), max_crops=1, n_samples=1, n_gray=2, gray_n=gn, las_mode=1, n_rad=8, n_ang=8,
                     w_a=w_a)
    losses = tr.forward([], levels, seed)
    gw, gb = tr.backward()
    torch.cuda.synchronize()
    ref = oracle_step([], [(l, gn) for l in levels], ws, bs, seed, 1, w_a, 1, 8, 8, quant=1)
    errs = _grad_errors(gw, gb, ref[4], ref[5])
    print("L_AS", losses[2], ref[2], "relative gradient errors (weights, biases) per layer:", errs)
    assert abs(losses[2] - ref[2]) <= 3e-4 * abs(ref[2]), (losses, ref[:4])
    assert losses[1] == 0.0 and losses[3] == 0.0
    for ew, eb in errs:
        assert ew <= 6e-3 and eb <= 6e-3, errs


def test_bf16_train_step_matches_bf16_oracle():
    """Full BF16 step (crops and gray patches) against the quant-1 oracle.  Crops 40 x 150:
    two 128-pixel column tiles, one ragged, five 8-row units per crop.  The samples
    h = [u < p] of the two sides differ wherever |p - u| is below the forward's BF16
    error (a few of the 24 000 pixel-samples here), and each flip changes the toggle
    deltas in its 21 x 21 neighbourhood; the loss is held to 1e-3 relative and the
    gradients to 2e-2 of the layer's largest entry, which still catches any wiring error
    of the step (measured: 0.6-0.8%)."""
    ws, _ = synth.he_normal_policy(WIDE4, 51)
    bs = synth.random_biases(WIDE4, 52, scale=0.1)
    crops = [synth.contone_image(40, 150, seed=53, index=i) for i in range(2)]
    levels = [0.3, 0.7]
    gn, S, seed, w_a = 32, 2, 9, 0.5
    pol = api.Policy(WIDE4, ws, bs, precision=N.HT_BF16)
    tr = api.Trainer(pol, (40, 150), max_crops=2, n_samples=S, n_gray=2, gray_n=gn, las_mode=1, n_rad=4, n_ang=4,
                     w_a=w_a)
    losses = tr.forward([torch.from_numpy(c).cuda() for c in crops], levels, seed)
    gw, gb = tr.backward()
    torch.cuda.synchronize()
    ref = oracle_step(crops, [(l, gn) for l in levels], ws, bs, seed, S, w_a, 1, 4, 4, quant=1)
    errs = _grad_errors(gw, gb, ref[4], ref[5])
    print("losses", losses, ref[:4], "relative gradient errors (weights, biases) per layer:", errs)
    for k in range(4):
        assert abs(losses[k] - ref[k]) <= 1e-3 * abs(ref[k]) + 1e-7, (k, losses, ref[:4])
    for ew, eb in errs:
        assert ew <= 2e-2 and eb <= 2e-2, errs


@pytest.mark.parametrize("stride", [2, 3])
def test_bf16_activation_recomputation_is_exact(stride):
    """Checkpointed training (every stride-th hidden activation kept, the rest recomputed
    in the backward) gives bit-identical gradients (the recomputed activations are the
    forward's).  No gray patches: their anisotropy bins, like the reward and loss sums, are
    FP64 atomic reductions whose last bits depend on run order, so the losses are compared
    to 1e-12."""
    chs = (2, 64, 64, 64, 64, 64, 1)
    ws, _ = synth.he_normal_policy(chs, 61)
    bs = synth.random_biases(chs, 62, scale=0.1)
    crops = [torch.from_numpy(synth.contone_image(40, 150, seed=63, index=i)).cuda() for i in range(2)]
    pol = api.Policy(chs, ws, bs, precision=N.HT_BF16)
    out = []
    for k in (1, stride):
        tr = api.Trainer(pol, (40, 150), max_crops=2, n_samples=2, n_gray=0, las_mode=1, n_rad=4, n_ang=4,
                         ckpt_stride=k)
        losses = tr.forward(crops, [], 5)
        gw, gb = tr.backward()
        torch.cuda.synchronize()
        out.append((losses, gw.clone(), gb.clone()))
        tr.close()
    assert all(abs(a - b) <= 1e-12 * abs(a) for a, b in zip(out[0][0], out[1][0]))
    assert torch.equal(out[0][1], out[1][1]) and torch.equal(out[0][2], out[1][2])


def test_training_rejects_fp8_policies():
    """Training runs in the FP32 form or the BF16 tensor-core form; an FP8 policy is refused."""
    ws, bs = synth.he_normal_policy(WIDE4, 1)
    pol = api.Policy(WIDE4, ws, bs, precision=N.HT_FP8_E4M3)
    with pytest.raises(N.HTError):
        api.Trainer(pol, (24, 24), max_crops=1, n_samples=1)
