#!/usr/bin/env python3
"""Throughput of one-shot halftoning on GB300 (one JSON line on rank 0).

Workload (default): printer-scale inference -- 8 synthetic 2048x2048 contone images,
8-layer 64-wide policy (2 -> 64 x 7 -> 1) in the BF16 tensor-core form with FP32
accumulation, fused sigmoid + Philox Bernoulli sampling (seed 1) + 1-bit packing.
A step = one ht_halftone call over the whole batch.

  value      : Mpixels/s, inputs resident in HBM, device time (CUDA events)
  e2e        : same metric through the C-ABI call with host buffers (pinned H2D of the
               contones and D2H of the packed halftones inside the timed region)
  roofline   : dominant kernel (the 64 -> 64 tcgen05 conv) -- algorithmic FLOPs per
               launch / its mean launch time, measured by the library's CUDA-event
               instrumentation over the timed region
  fp32_plain : the plain FP32 CUDA-core form of the same net on the same batch
  cpu_baseline: the FP64 C oracle on a bounded crop of the same workload (host cores)

--impl reference times the oracle (the reference arm of this build) on bounded crops.
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


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_images(args, rank):
    from paper_2304_12152_gb300 import synth
    shapes = [(args.size, args.size)] * args.batch
    # every rank its own images (replicas): the generator index carries the rank
    return [synth.contone_image(h, w, seed=1, index=rank * 1000 + i) for i, (h, w) in enumerate(shapes)]


def cpu_oracle_sample(img, ws, bs, side, seed, image_id=0):
    """FP64 oracle (BF16-emulating) forward + Bernoulli actions on a side x side crop."""
    import oracle as O
    h, w = img.shape
    y0, x0 = (h - side) // 2, (w - side) // 2
    reg = (y0, x0, side, side)
    t0 = time.perf_counter()
    _, p, _ = O.forward(img, ws, bs, noise_seed=seed, image=image_id, quant=1, region=reg)
    lev, u = O.sample(p, h, w, reg, 1, seed, image_id)
    dt = time.perf_counter() - t0
    return dt, reg, p, lev, u


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
        "config": {"workload": f"printer {args.batch}x{args.size}x{args.size}, 2->64x7->1 policy, Bernoulli seed 1",
                   "sample": f"{side}x{side} centre crop of image 0 per step"},
        "cpu_baseline": {"value": v, "unit": "Mpx/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{side}x{side} crop per step, BF16-emulating FP64 forward + sampling"},
        "e2e": {"value": v, "unit": "Mpx/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--fp32-steps", type=int, default=2)
    ap.add_argument("--ref-side", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    from paper_2304_12152_gb300 import _native as N
    from paper_2304_12152_gb300 import api, synth

    chs = synth.NET_WIDE
    ws, bs = synth.he_normal_policy(chs, 1)
    prec = N.HT_BF16 if args.precision == "bf16" else N.HT_FP32
    pol = api.Policy(chs, ws, bs, precision=prec)
    imgs_np = workload_images(args, rank)
    dev = torch.device("cuda", local)
    cs = [torch.from_numpy(c).to(dev) for c in imgs_np]
    bits = [pol.alloc_bits(c.shape[0], c.shape[1], dev) for c in cs]
    px_per_step = sum(c.numel() for c in cs)
    stream = torch.cuda.current_stream()

    def step():
        pol.halftone_into(cs, bits, N.HT_MODE_BERNOULLI, 1)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    for _ in range(args.warmup):
        step()
    api.sync()

    # ---------------- device-resident timed region ----------------
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    api.profile_begin()
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    prof = api.profile_end()
    barrier()
    api.sync()
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms)
    ms_step = ms / args.steps
    value = world * px_per_step / (ms_step * 1e-3) / 1e6

    # ---------------- end-to-end through the C ABI with host buffers ----------------
    host_in = [torch.from_numpy(c).pin_memory() for c in imgs_np]
    host_out = [torch.empty(b.shape, dtype=b.dtype).pin_memory() for b in bits]
    h2d = sum(t.numel() * 4 for t in host_in)
    d2h = sum(t.numel() * 4 for t in host_out)

    def e2e_step():
        for hi, di in zip(host_in, cs):
            di.copy_(hi, non_blocking=True)
        step()
        for ho, b in zip(host_out, bits):
            ho.copy_(b, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1)) / args.steps
    e2e_val = world * px_per_step / (e2e_ms * 1e-3) / 1e6

    # ---------------- plain FP32 form of the same net ----------------
    fp32 = None
    if prec != N.HT_FP32 and args.fp32_steps > 0:
        pol32 = api.Policy(chs, ws, bs, precision=N.HT_FP32)
        pol32.halftone_into(cs, bits, N.HT_MODE_BERNOULLI, 1)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp32_steps):
            pol32.halftone_into(cs, bits, N.HT_MODE_BERNOULLI, 1)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = max_over_ranks(f0.elapsed_time(f1)) / args.fp32_steps
        fp32 = {"value": world * px_per_step / (fms * 1e-3) / 1e6, "unit": "Mpx/s", "ms_per_step": fms,
                "steps": args.fp32_steps}
        del pol32
        step()
        torch.cuda.synchronize()

    # ---------------- roofline of the dominant kernel ----------------
    pk, src = peaks()
    roof = None
    kname = "k_conv_tc_bf16" if prec != N.HT_FP32 else "k_conv3x3_fp32"
    if kname in prof:
        launches, tot = prof[kname]
        per_launch_ms = tot / launches
        flops_launch = 2 * 9 * 64 * 64 * (px_per_step / args.batch)   # one 64->64 layer on one image
        achieved = flops_launch / (per_launch_ms * 1e-3) / 1e12
        peak = pk.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"])
        roof = {"bound": "tensor", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "per_launch_ms": per_launch_ms,
                "peak_source": f"{src} bf16 dense, sustained"}
    kernels = {k: {"launches": v[0], "total_ms": v[1], "share": v[1] / max(1e-9, sum(x[1] for x in prof.values()))}
               for k, v in prof.items()}
    gpu_launches = sum(v[0] for v in prof.values())

    # ---------------- CPU oracle baseline on a bounded sample ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        side = 64
        dt, *_ = cpu_oracle_sample(imgs_np[0], ws, bs, side, 1)
        side = int(min(1024, max(64, side * math.sqrt(15.0 / max(dt, 1e-3)))))
        side -= side % 8
        dt, reg, p, lev_or, u = cpu_oracle_sample(imgs_np[0], ws, bs, side, 1)
        y0, x0, rh, rw = reg
        lev_gpu = api.unpack_bits(bits[0], args.size, args.size)[y0:y0 + rh, x0:x0 + rw]
        decided = np.abs(p[0] - u) > 1e-4
        mism = int(((lev_gpu != lev_or) & decided).sum())
        cpu = {"value": side * side / dt / 1e6, "unit": "Mpx/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": f"{side}x{side} centre crop of image 0 (+8 px halo), BF16-emulating FP64 forward + "
                         f"Bernoulli actions", "seconds": dt,
               "bit_match": {"decided": int(decided.sum()), "mismatch": mism,
                             "rate": 1.0 - mism / max(1, int(decided.sum())), "margin": 1e-4}}

    if rank == 0:
        line = {
            "metric": "halftone Mpixels/s", "value": value, "unit": "Mpx/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if prec != N.HT_FP32 else "f32",
            "data": "synthetic",
            "config": {"workload": f"printer {args.batch}x{args.size}x{args.size}, 2->64x7->1 policy, "
                                   f"Bernoulli seed 1, 1-bit packed", "batch": args.batch,
                       "image": [args.size, args.size], "parallelism": f"replicas x{world}",
                       "l2": "inputs and activations larger than L2"},
            "e2e": {"value": e2e_val, "unit": "Mpx/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms},
            "roofline": roof, "fp32_plain": fp32, "cpu_baseline": cpu, "kernels": kernels,
            "gpu_launches": gpu_launches, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
