#!/usr/bin/env python3
"""Throughput of one-shot halftoning on GB300 (one JSON line on rank 0).

Workload (default): printer-scale inference -- 8 synthetic 2048x2048 contone images,
8-layer 64-wide policy (2 -> 64 x 7 -> 1) in the BF16 tensor-core form with FP32
accumulation, fused sigmoid + Philox Bernoulli sampling (seed 1) + 1-bit packing.
A step = one ht_halftone call over the whole batch.

  value      : Mpixels/s, inputs resident in HBM, device time (CUDA events)
  e2e        : same metric through the C-ABI call with host buffers (pinned H2D of the
               contones and D2H of the packed halftones inside the timed region, every
               step; copies on their own streams, overlapping the neighbouring steps'
               compute through two buffer sets, as a streaming caller would run it)
  roofline   : dominant kernel (the 64 -> 64 tcgen05 conv) -- algorithmic FLOPs per
               launch / its mean launch time, measured by the library's CUDA-event
               instrumentation over the timed region
  fp32_plain : the plain FP32 CUDA-core form of the same net on the same batch
  cpu_baseline: the FP64 C oracle on a bounded crop of the same workload (host cores)

--impl reference times the oracle (the benchmark's reference arm) on bounded crops.
Multi-GPU (torchrun): independent replicas, weak scaling, max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return dict(FALLBACK_PEAKS), "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's time (all ranks take part): max all-reduce of one float."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_oracle_sample(img, ws, bs, side, seed, image_id=0, quant=1, mode=1, scales=None, levels=0, resnet=False):
    """FP64 oracle (optionally emulating the reduced-precision rounding) forward and
    actions on a side x side centre crop (levels > 0: the multitoning prototype's rule;
    resnet: the residual policy)."""
    import oracle as O
    h, w = img.shape
    side = min(side, h, w)
    y0, x0 = (h - side) // 2, (w - side) // 2
    reg = (y0, x0, side, side)
    t0 = time.perf_counter()
    if resnet:
        _, p1 = O.forward_resnet(img, ws, bs, seed, image_id, quant=quant, region=reg)
        p = p1[None]
    else:
        _, p, _ = O.forward(img, ws, bs, noise_seed=seed, image=image_id, quant=quant, act_scale=scales, region=reg)
    lev, u = O.sample(p, h, w, reg, mode, seed, image_id)
    if levels:
        lev = O.sample_multitone(p[0], levels, u if mode == 1 else None)
    dt = time.perf_counter() - t0
    return dt, reg, p, lev, u


def cpu_oracle_one_thread(img, ws, bs, seed, quant=1, mode=1, levels=0, resnet=False, seconds=5.0):
    """The oracle's rate on one host thread, beside its all-threads rate: a centre crop
    sized (by area, from a small first pass) for about `seconds` of work.  The oracle's
    thread count is restored afterwards; a failure is reported, not raised."""
    import oracle as O
    n0 = O.num_threads()
    try:
        O.set_num_threads(1)
        side = 16
        dt, *_ = cpu_oracle_sample(img, ws, bs, side, seed, quant=quant, mode=mode, levels=levels, resnet=resnet)
        side = int(min(min(img.shape), 512, max(16, side * math.sqrt(seconds / max(dt, 1e-3)))))
        side -= side % 8
        dt, *_ = cpu_oracle_sample(img, ws, bs, side, seed, quant=quant, mode=mode, levels=levels, resnet=resnet)
        return {"value": side * side / dt / 1e6, "unit": "Mpx/s", "cores": 1,
                "sample": f"{side}x{side} centre crop of image 0 (+halo)", "seconds": dt}
    except Exception as e:          # context only: report, never abort the bench line
        return {"error": f"{type(e).__name__}: {str(e)[:200]}"}
    finally:
        O.set_num_threads(n0)


def run_reference(args):
    rank, world, local = dist_info()
    if rank != 0:
        return
    import oracle as O
    from paper_2304_12152_gb300 import synth
    O.build()
    ws, bs = synth.he_normal_policy(synth.NET_WIDE, 1)
    img = synth.contone_image(args.size, args.size, seed=1, index=0)
    side = args.ref_side
    for _ in range(args.warmup):
        cpu_oracle_sample(img, ws, bs, side, 1)
    t = 0.0
    for _ in range(args.steps):
        dt, *_ = cpu_oracle_sample(img, ws, bs, side, 1)
        t += dt
    px = side * side * args.steps
    v = px / t / 1e6
    line = {
        "impl": "reference", "metric": "halftone Mpixels/s", "value": v, "unit": "Mpx/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"printer {args.batch}x{args.size}x{args.size}, 2->64x7->1 policy, BF16, Bernoulli seed 1, 1-bit packed",
                   "sample": f"{side}x{side} centre crop of image 0 per step"},
        "cpu_baseline": {"value": v, "unit": "Mpx/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{side}x{side} crop per step, BF16-emulating FP64 forward + sampling"},
        "e2e": {"value": v, "unit": "Mpx/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


WORKLOADS = {
    # name: (description, precision, head, net, mode, seed)
    "printer": ("printer {b}x{h}x{w}, 2->64x7->1 policy, BF16, Bernoulli seed 1, 1-bit packed", "bf16", 0, "wide", 1, 1),
    "multitone": ("multitone 4x4096x4096, 2->64x7->4 softmax head (levels 0,1/3,2/3,1), FP8 E4M3, Philox seed 2",
                  "fp8", 1, "wide4", 1, 2),
    "uneven": ("uneven batch of 64 images, sizes log-uniform 200x300..4096x3072 (seed 4), BF16, Bernoulli seed 4",
               "bf16", 0, "wide", 1, 4),
    "small": ("one 256x256 image (seed 0), 2->32x5->1 policy, plain FP32, threshold 0.5", "fp32", 0, "small", 0, 0),
    "proto": ("multitoning prototype 4x4096x4096, 2->64x7->1 sigmoid output, action between the 2 of 4 levels "
              "around it, BF16, Philox seed 2", "bf16", 2, "wide", 1, 2),
    "resnet512": ("residual policy (16 blocks x 32 ch, 34 conv layers) on one 512x512 image (the paper's "
                  "runtime setting), BF16, threshold", "bf16", 0, "resnet", 0, 5),
    "resnet": ("residual policy (16 blocks x 32 ch, 34 conv layers) on 8x2048x2048, BF16, Bernoulli seed 1",
               "bf16", 0, "resnet", 1, 1),
}


def build_inputs(args, rank):
    from paper_2304_12152_gb300 import synth
    if args.images and args.side:      # small case of any workload (profiling)
        seed = WORKLOADS[args.workload][5]
        shapes = [(args.side, args.side)] * args.images
        return [synth.contone_image(h, w, seed=seed, index=rank * 1000 + i) for i, (h, w) in enumerate(shapes)], shapes
    if args.workload in ("printer", "resnet"):
        shapes = [(args.size, args.size)] * args.batch
        seed = 1
    elif args.workload in ("multitone", "proto"):
        shapes = [(4096, 4096)] * 4
        seed = 2
    elif args.workload == "resnet512":
        shapes = [(512, 512)]
        seed = 5
    elif args.workload == "uneven":
        shapes = synth.uneven_shapes(64, seed=4)
        seed = 4
    else:
        shapes = [(256, 256)]
        seed = 0
    return [synth.contone_image(h, w, seed=seed, index=rank * 1000 + i) for i, (h, w) in enumerate(shapes)], shapes


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="printer", choices=sorted(list(WORKLOADS) + ["train"]))
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--images", type=int, default=0, help="override: number of images (with --side)")
    ap.add_argument("--side", type=int, default=0, help="override: square image side (with --images)")
    ap.add_argument("--fp32-steps", type=int, default=2)
    ap.add_argument("--torch-fp32-steps", type=int, default=1,
                    help="timed passes of the plain PyTorch FP32 form (cuDNN, TF32 off); 0 skips it")
    ap.add_argument("--ref-side", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", default="",
                    help="ROWS,ORDER[,PAIR]: set the conv schedule instead of autotuning (PAIR 1 = CTA-pair 64->64 layers)")
    ap.add_argument("--ckpt", type=int, default=0, help="train: activation checkpoint stride (recomputation)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "train":
        return run_train(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    from paper_2304_12152_gb300 import _native as N
    from paper_2304_12152_gb300 import api, synth

    desc, precision, head, netname, mode, seed = WORKLOADS[args.workload]
    resnet = netname == "resnet"
    if resnet:
        chs = synth.resnet_channels(synth.RESNET_BLOCKS, synth.RESNET_WIDTH)
        ws, bs = synth.resnet_policy(synth.RESNET_BLOCKS, synth.RESNET_WIDTH, 1)
    else:
        chs = {"wide": synth.NET_WIDE, "wide4": synth.NET_WIDE_K4, "small": synth.NET_SMALL}[netname]
        ws, bs = synth.he_normal_policy(chs, 1)
    prec = {"bf16": N.HT_BF16, "fp8": N.HT_FP8_E4M3, "fp32": N.HT_FP32}[precision]
    pol = api.Policy(chs, ws, bs, head=head, precision=prec, levels=4,
                     arch=N.HT_ARCH_RESNET if resnet else N.HT_ARCH_PLAIN)
    dev = torch.device("cuda", local)
    if prec == N.HT_FP8_E4M3:
        calib = torch.from_numpy(synth.contone_image(256, 256, seed=99)).to(dev)
        pol.calibrate(calib, seed=99)
    imgs_np, shapes = build_inputs(args, rank)
    cs = [torch.from_numpy(c).to(dev) for c in imgs_np]
    bits = [pol.alloc_bits(c.shape[0], c.shape[1], dev) for c in cs]
    px_per_step = sum(c.numel() for c in cs)
    stream = torch.cuda.current_stream()

    def direct_step():
        pol.halftone_into(cs, bits, mode, seed)

    # tensor-core forms: the conv schedule is picked by the library's autotuner on this
    # workload, then the call is captured once into a CUDA graph (ht_plan) and replayed
    tune = None
    plan = None
    if prec != N.HT_FP32:
        if args.schedule:
            sched = [int(x) for x in args.schedule.split(",")]
            ru, order, pair = sched[0], sched[1], (sched[2] if len(sched) > 2 else 0)
            pol.set_schedule(ru, order, pair)
            tune = {"choice": {"rows_per_unit": ru, "unit_order": order, "cta_pair": pair}, "candidates": None}
        else:
            res = pol.autotune(cs, bits, mode, seed, reps=2)
            best = min(res, key=lambda r: r[3])
            tune = {"choice": {"rows_per_unit": best[0], "unit_order": best[1], "cta_pair": best[2]},
                    "candidates": [{"rows_per_unit": r, "unit_order": o, "cta_pair": pr, "ms": ms}
                                   for r, o, pr, ms in res]}
        plan = api.Plan(pol, cs, bits, mode, seed)

    def step():
        if plan is not None:
            plan.launch()
        else:
            direct_step()

    def barrier():
        if world > 1:
            dist.barrier()


    for _ in range(args.warmup):
        step()
    api.sync()

    # ---------------- device-resident timed region (graph replay for the tensor-core forms) ----------------
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    api.sync()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    ms_step = ms / args.steps
    value = world * px_per_step / (ms_step * 1e-3) / 1e6

    # ---------------- per-kernel times: the same call, direct launches bracketed by CUDA events ----------------
    prof_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    api.profile_begin()
    for _ in range(prof_steps):
        direct_step()
    prof = api.profile_end()
    api.sync()

    # ---------------- end-to-end through the C ABI with host buffers ----------------
    host_in = [torch.from_numpy(c).pin_memory() for c in imgs_np]
    host_out = [torch.empty(b.shape, dtype=b.dtype).pin_memory() for b in bits]
    h2d = sum(t.numel() * 4 for t in host_in)
    d2h = sum(t.numel() * 4 for t in host_out)

    # Streamed the way a caller would: two input/output buffer sets, the H2D copy of step
    # i + 1 and the D2H copy of step i on their own streams, overlapping step i's compute.
    # Every step still copies all of its inputs in and its packed halftones out inside the
    # timed region.
    cs_b = [cs, [torch.empty_like(c) for c in cs]]
    bits_b = [bits, [torch.empty_like(b) for b in bits]]
    plans_b = [plan, api.Plan(pol, cs_b[1], bits_b[1], mode, seed)] if plan is not None else None
    h2d_s, d2h_s = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    ev_start = torch.cuda.Event()

    def e2e_run(nsteps):
        ev_start.record(stream)
        h2d_s.wait_event(ev_start)                        # no copy starts before the timed region
        d2h_s.wait_event(ev_start)
        for i in range(nsteps):
            b = i % 2
            with torch.cuda.stream(h2d_s):
                if i >= 2:
                    h2d_s.wait_event(ev_done[b])          # step i - 2 has read buffer set b
                for hi, di in zip(host_in, cs_b[b]):
                    di.copy_(hi, non_blocking=True)
                ev_in[b].record(h2d_s)
            stream.wait_event(ev_in[b])
            if i >= 2:
                stream.wait_event(ev_out[b])              # step i - 2's halftones have left buffer set b
            if plans_b is not None:
                plans_b[b].launch(stream)
            else:
                pol.halftone_into(cs_b[b], bits_b[b], mode, seed, stream=stream)
            ev_done[b].record(stream)
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(ev_done[b])
                for ho, bb in zip(host_out, bits_b[b]):
                    ho.copy_(bb, non_blocking=True)
                ev_out[b].record(d2h_s)
        stream.wait_event(ev_out[(nsteps - 1) % 2])
        if nsteps > 1:
            stream.wait_event(ev_out[(nsteps - 2) % 2])

    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    api.sync()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev) / args.steps
    e2e_val = world * px_per_step / (e2e_ms * 1e-3) / 1e6

    # ---------------- plain FP32 form of the same net ----------------
    fp32 = None
    if prec != N.HT_FP32 and args.fp32_steps > 0 and not resnet:
        pol32 = api.Policy(chs, ws, bs, head=head, precision=N.HT_FP32, levels=4)
        pol32.halftone_into(cs, bits, mode, seed)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp32_steps):
            pol32.halftone_into(cs, bits, mode, seed)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = max_over_ranks(f0.elapsed_time(f1), world, dev) / args.fp32_steps
        fp32 = {"value": world * px_per_step / (fms * 1e-3) / 1e6, "unit": "Mpx/s", "ms_per_step": fms,
                "steps": args.fp32_steps}
        del pol32
        step()
        torch.cuda.synchronize()

    # ---------------- roofline of the dominant kernel ----------------
    pk, src = peaks()
    roof = None
    kname = {N.HT_BF16: "k_conv_tc_bf16", N.HT_FP8_E4M3: "k_conv_tc_fp8", N.HT_FP32: "k_conv3x3_fp32"}[prec]
    if kname in prof:
        launches, tot = prof[kname]
        per_launch_ms = tot / launches
        cmid = chs[1]
        n_mid = len(chs) - 3 if prec != N.HT_FP32 else len(chs) - 2
        # one launch = one C -> C layer over one image group: layers x pixels / launches
        flops_launch = 2 * 9 * cmid * cmid * px_per_step * prof_steps * n_mid / launches
        achieved = flops_launch / (per_launch_ms * 1e-3) / 1e12
        if resnet:
            # 32-wide layers: 18 432 flop/px against 128 B/px (conv1: read + write bf16) or
            # 192 B/px (conv2: + the shortcut read), mean 160 B/px -> 115 flop/B, below the
            # bf16 ridge (~250 flop/B): HBM-bound
            bytes_launch = 160.0 * px_per_step * prof_steps * n_mid / launches
            gbs = bytes_launch / (per_launch_ms * 1e-3) / 1e9
            hbm = pk.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"])
            roof = {"bound": "hbm", "kernel": kname, "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                    "traffic": None, "per_launch_ms": per_launch_ms, "tensor_tflops": achieved,
                    "peak_source": f"{src} HBM copy bandwidth"}
        elif prec == N.HT_FP32:
            roof = {"bound": "alu", "kernel": kname, "achieved": achieved,
                    "peak": fp32_alu_peak(clk.summary()), "unit": "TFLOP/s", "traffic": None,
                    "per_launch_ms": per_launch_ms,
                    "peak_source": "SM count x 128 FP32 FMA/clk x 2 x median SM clock under load"}
            roof["frac"] = achieved / roof["peak"]
        else:
            peak = pk.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"])
            psrc = f"{src} bf16 dense, sustained"
            if prec == N.HT_FP8_E4M3:
                peak *= 2.0
                psrc = f"{src} bf16 dense sustained x 2 (nominal fp8/bf16 ratio 4.5/2.25)"
            roof = {"bound": "tensor", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": conv_traffic(args, kname, px_per_step, launches / prof_steps),
                    "per_launch_ms": per_launch_ms, "peak_source": psrc}
    tot_ms = max(1e-9, sum(x[1] for x in prof.values()))
    kernels = {k: {"launches": v[0], "total_ms": v[1], "share": v[1] / tot_ms} for k, v in prof.items()}
    # HBM-bound passes around the conv stack: algorithmic bytes per pixel, achieved GB/s
    hbm_bytes = {"k_first_input": 4.0 + 16.0}            # contone read, split c / z write
    if head != N.HT_HEAD_SOFTMAX:
        hbm_bytes["k_head_tc"] = 36.0 + 0.25             # 9 partials read, packed levels written
    hbm_peak = pk.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"])
    hbm = {}
    for k, bpp in hbm_bytes.items():
        if k in prof and prof[k][1] > 0:
            gbs = bpp * px_per_step * prof_steps / (prof[k][1] * 1e-3) / 1e9
            hbm[k] = {"bytes_per_px": bpp, "achieved_gbs": gbs, "frac": gbs / hbm_peak}
    # launches inside the timed region: the replayed graph holds the same launches as one direct call
    gpu_launches = sum(v[0] for v in prof.values()) * args.steps // prof_steps

    # ---------------- CPU oracle baseline on a bounded sample ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        quant = {N.HT_BF16: 1, N.HT_FP8_E4M3: 2, N.HT_FP32: 0}[prec]
        side = 32
        lv = 4 if head == N.HT_HEAD_MULTITONE else 0
        dt, *_ = cpu_oracle_sample(imgs_np[0], ws, bs, side, seed, quant=quant, mode=mode, scales=None, levels=lv,
                                   resnet=resnet)
        side = int(min(min(imgs_np[0].shape), 1024, max(32, side * math.sqrt(15.0 / max(dt, 1e-3)))))
        side -= side % 8
        dt, reg, p, lev_or, u = cpu_oracle_sample(imgs_np[0], ws, bs, side, seed, quant=quant, mode=mode, scales=None,
                                                  levels=lv, resnet=resnet)
        cpu = {"value": side * side / dt / 1e6, "unit": "Mpx/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": f"{side}x{side} centre crop of image 0 (+halo), FP64 forward"
                         f"{' emulating the ' + precision.upper() + ' rounding' if quant else ''} + actions",
               "seconds": dt}
        cpu["one_thread"] = cpu_oracle_one_thread(imgs_np[0], ws, bs, seed, quant=quant, mode=mode, levels=lv,
                                                  resnet=resnet)
        if quant != 2:   # FP8 scales come from the library's calibration: no bit comparison
            y0, x0, rh, rw = reg
            lev_gpu = api.unpack_bits(bits[0], imgs_np[0].shape[0], imgs_np[0].shape[1], head)[y0:y0 + rh, x0:x0 + rw]
            if lv:
                t = p[0] * (lv - 1)
                _, frac = O.multitone_pair(p[0], lv)
                decided = (np.abs(frac - (u if mode == 1 else 0.5)) > 1e-4) & (np.abs(t - np.rint(t)) > 1e-4)
            elif p.shape[0] == 1:
                decided = np.abs(p[0] - u) > 1e-4
            else:
                cdf = np.cumsum(p, 0)
                decided = np.all(np.abs(cdf - u[None]) > 1e-4, 0) if mode == 1 else np.ones_like(u, bool)
            mism = int(((lev_gpu != lev_or) & decided).sum())
            cpu["bit_match"] = {"decided": int(decided.sum()), "mismatch": mism,
                                "rate": 1.0 - mism / max(1, int(decided.sum())), "margin": 1e-4}

    # ---------------- the plain PyTorch FP32 form (context; after every other measurement) ----------------
    torch32 = None
    if rank == 0 and world == 1 and args.torch_fp32_steps > 0 and not resnet:
        torch32 = torch_fp32_form(args.torch_fp32_steps, cs, ws, bs, head == N.HT_HEAD_SOFTMAX, px_per_step)

    if rank == 0:
        wdesc = desc.format(b=args.batch, h=args.size, w=args.size)
        line = {
            "metric": "halftone Mpixels/s", "value": value, "unit": "Mpx/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": precision if precision != "fp8" else "e4m3",
            "data": "synthetic",
            "config": {"workload": wdesc, "images": len(shapes), "pixels_per_step": px_per_step,
                       "parallelism": f"replicas x{world}", "l2": "inputs and activations larger than L2"},
            "e2e": {"value": e2e_val, "unit": "Mpx/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms,
                    "method": "pinned host buffers; per step all inputs H2D and all halftones D2H inside the "
                              "timed region, on two copy streams overlapping the neighbouring steps' compute "
                              "(two buffer sets, one CUDA-graph plan each)"},
            "roofline": roof, "fp32_plain": fp32, "torch_fp32": torch32, "cpu_baseline": cpu, "kernels": kernels,
            "gpu_launches": gpu_launches, "clocks": clk.summary(),
            "timing": ("value and e2e: CUDA-graph replay of the call (ht_plan); kernels and roofline: "
                       f"{prof_steps} direct calls, each launch bracketed by CUDA events") if plan is not None
                      else "direct calls",
            "autotune": tune, "hbm_kernels": hbm,
        }
        if args.workload == "uneven":
            line["config"]["shapes"] = shapes
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def fp32_alu_peak(clocks):
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def code_hash(path):
    """sha256 of a C/CUDA source with comments and blank lines removed, so that a change of
    comments alone keeps a committed counter capture valid."""
    import hashlib
    import re
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in txt.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln.strip()).encode()).hexdigest()


def torch_fp32_form(steps, cs, ws, bs, softmax_head, px_per_step):
    """The same policy as plain PyTorch FP32 operators, for context beside the library's
    forms: cuDNN convolutions with TF32 off (3x3, zero padding 1) and ReLU, then the sigmoid
    (softmax over 4 logits) and a Bernoulli comparison against torch uniforms, one image at
    a time, into an unpacked per-pixel map.  One untimed pass, then `steps` timed ones
    (CUDA events on a GPU, wall clock on the CPU).  Any failure, out-of-memory included, is
    returned as an error string rather than raised."""
    import time

    import torch
    import torch.nn.functional as F
    prev = (torch.backends.cudnn.allow_tf32, torch.backends.cuda.matmul.allow_tf32)
    try:
        torch.backends.cudnn.allow_tf32 = False
        torch.backends.cuda.matmul.allow_tf32 = False
        dev = cs[0].device
        wt = [torch.from_numpy(w).to(dev) for w in ws]
        bt = [torch.from_numpy(b).to(dev) for b in bs]
        gen = torch.Generator(device=dev)
        gen.manual_seed(1)
        zs = [torch.rand(tuple(c.shape), device=dev, generator=gen) for c in cs]

        def one_pass():
            out = []
            for c, z in zip(cs, zs):
                x = torch.stack([c, z])[None]
                for l in range(len(wt)):
                    x = F.conv2d(x, wt[l], bt[l], padding=1)
                    if l < len(wt) - 1:
                        x = torch.relu_(x)
                u = torch.rand(tuple(c.shape), device=dev, generator=gen)
                if softmax_head:
                    h = (torch.cumsum(torch.softmax(x[0], 0), 0) <= u[None]).sum(0)
                else:
                    h = u < torch.sigmoid(x[0, 0])
                out.append(h)
            return out

        cuda = dev.type == "cuda"
        one_pass()
        if cuda:
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
        t0 = time.perf_counter()
        for _ in range(steps):
            one_pass()
        if cuda:
            e1.record()
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
        else:
            ms = (time.perf_counter() - t0) * 1e3 / steps
        return {"value": px_per_step / (ms * 1e-3) / 1e6, "unit": "Mpx/s", "ms_per_step": ms, "steps": steps,
                "form": "torch F.conv2d FP32 (cuDNN, TF32 off) + ReLU, sigmoid / softmax, Bernoulli comparison; "
                        "one image at a time, unpacked output"}
    except Exception as e:          # context only: report, never abort the bench line
        return {"error": f"{type(e).__name__}: {str(e)[:200]}"}
    finally:
        torch.backends.cudnn.allow_tf32, torch.backends.cuda.matmul.allow_tf32 = prev
        if torch.cuda.is_available():
            torch.cuda.empty_cache()


def conv_traffic(args, kname, px_per_step, launches_per_step):
    """DRAM bytes per launch of the conv kernel, from the committed ncu summary when its
    recorded source hash matches the current kernel source (else null)."""
    import re
    src = os.path.join(ROOT, "paper_2304_12152_gb300", "csrc", "conv_tc.cu")
    summ = os.path.join(ROOT, "profiles", "k_conv_tc_bf16_2048.md")
    try:
        h = code_hash(src)
        txt = open(summ).read()
    except OSError:
        return None
    m = re.search(r"code_sha256:\s*([0-9a-f]{64})", txt)
    b = re.search(r"dram_bytes_per_px_per_layer:\s*([0-9.]+)", txt)
    if not m or not b or m.group(1) != h or kname != "k_conv_tc_bf16":
        return None
    # one launch = one 64 -> 64 layer over one image (six layers per image)
    return float(b.group(1)) * px_per_step * 6.0 / launches_per_step


def run_train(args):
    """Training step (Algorithm 1 TRAIN) timing: 16 crops 256x256 + 4 gray patches, S = 4,
    BF16 tensor-core form (FP32 master weights), with the FP32 CUDA-core form beside it."""
    import torch
    from paper_2304_12152_gb300 import _native as N
    from paper_2304_12152_gb300 import api, synth
    import torch.distributed as dist
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl")
    chs = synth.NET_WIDE
    ws, bs = synth.he_normal_policy(chs, 3)
    # data parallel: each rank its own 16 crops; gradients averaged with one all-reduce per step
    crops = [torch.from_numpy(synth.contone_image(256, 256, seed=3, index=rank * 1000 + i)).cuda() for i in range(16)]
    levels = [0.1, 0.25, 0.5, 0.75]
    gw = torch.empty(sum(chs[i] * chs[i + 1] * 9 for i in range(len(chs) - 1)), device="cuda")
    gb = torch.empty(sum(chs[1:]), device="cuda")
    stream = torch.cuda.current_stream()

    def timed(prec, steps, warmup, profile):
        pol = api.Policy(chs, ws, bs, precision=prec)
        tr = api.Trainer(pol, (256, 256), max_crops=16, n_samples=4, n_gray=4, gray_n=256, las_mode=1, n_rad=32,
                         n_ang=16, w_a=0.002, ckpt_stride=args.ckpt if prec == N.HT_BF16 else 0)
        for _ in range(warmup):
            tr.forward(crops, levels, 1)
            tr.backward(gw, gb)
            api.allreduce_grads([gw, gb])
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if profile:
            api.profile_begin()
        with Clocks(local) as clk:
            e0.record(stream)
            for k in range(steps):
                losses = tr.forward(crops, levels, 1 + k)
                tr.backward(gw, gb)
                api.allreduce_grads([gw, gb])
            e1.record(stream)
            torch.cuda.synchronize()
        prof = api.profile_end() if profile else {}
        return max_over_ranks(e0.elapsed_time(e1), world, dev) / steps, losses, prof, clk.summary()

    ms, losses, prof, clocks = timed(N.HT_BF16, args.steps, args.warmup, True)
    fp32 = None
    if args.fp32_steps > 0 and world == 1:
        ms32, _, _, _ = timed(N.HT_FP32, args.fp32_steps, 1, False)
        fp32 = {"value": ms32, "unit": "ms", "steps": args.fp32_steps}
    if rank != 0:
        dist.barrier()
        dist.destroy_process_group()
        return
    # reward window sums and toggle deltas: algorithmic bytes per crop-sample pixel
    # (contone 4 B + 1/8 B bits; toggles: + 7 moment maps written and read, dR written)
    px_samples = 16 * 4 * 256 * 256 * args.steps
    hbm_peak = peaks()[0].get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"])
    filt = {}
    for k, bpp in (("k_reward", 4.125), ("k_toggle_delta", 4.125 + 28.0 + 28.0 + 4.125 + 4.0)):
        if k in prof and prof[k][1] > 0:
            gbs = bpp * px_samples / (prof[k][1] * 1e-3) / 1e9
            filt[k] = {"bytes_per_px": bpp, "achieved_gbs": gbs, "frac": gbs / hbm_peak,
                       "note": "ALU-bound stencils (5-6 window sums; toggles ~3.6 kflop/px)"}
    print(json.dumps({
        "metric": "training step time", "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "train: 16 crops 256x256 + 4 gray 256x256 {0.1,0.25,0.5,0.75}, S=4, "
                               "2->64x7->1, w_s 0.06, w_a 0.002, 32x16-bin anisotropy loss, FP32 master weights"},
        "losses": {"total": losses[0], "marl": losses[1], "las": losses[2], "mean_R": losses[3]},
        "fp32_plain": fp32,
        "kernels": {k: {"launches": v[0], "total_ms": v[1]} for k, v in prof.items()},
        "gpu_launches": sum(v[0] for v in prof.values()), "clocks": clocks,
        "parallelism": f"data parallel x{world}, one gradient all-reduce per step", "hbm_kernels": filt,
        "ckpt_stride": args.ckpt}), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
