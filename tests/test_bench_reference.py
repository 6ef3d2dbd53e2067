"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one JSON line
with the keys the bench contract names; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-side", "32"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["warmup"] >= 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_torch_fp32_form_runs_and_reports_errors_on_cpu():
    """The bench's plain PyTorch FP32 form (context beside the library's forms) on small CPU
    tensors: both heads give a throughput line; a failure comes back as an error string."""
    import numpy as np
    import torch

    import bench
    from paper_2304_12152_gb300 import synth
    prev = (torch.backends.cudnn.allow_tf32, torch.backends.cuda.matmul.allow_tf32)
    cs = [torch.from_numpy(synth.contone_image(24, 31, seed=1, index=i)) for i in range(2)]
    px = sum(c.numel() for c in cs)
    for chs, softmax in ((synth.NET_SMALL, False), ((2, 8, 8, 4), True)):
        ws, bs = synth.he_normal_policy(chs, 1)
        r = bench.torch_fp32_form(1, cs, ws, bs, softmax, px)
        assert "error" not in r, r
        assert r["value"] > 0 and r["unit"] == "Mpx/s" and r["steps"] == 1
    ws, bs = synth.he_normal_policy(synth.NET_SMALL, 1)
    bad = bench.torch_fp32_form(1, cs, ws[1:], bs[1:], False, px)      # first layer missing
    assert set(bad) == {"error"} and "RuntimeError" in bad["error"]
    assert (torch.backends.cudnn.allow_tf32, torch.backends.cuda.matmul.allow_tf32) == prev   # restored
    assert np.isfinite(r["ms_per_step"])


def test_clock_summary_rules():
    """The bench's clocks record: median SM clock, the highest maximum seen, and every
    throttle reason reported active (a run with a hardware or thermal slowdown is the
    one to reject); unparsable samples are skipped, no samples reads as unsampled."""
    import bench
    c = bench.Clocks(0)
    c.lines = ["2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, 1390.2, 0x4, Not Active, Not Active, Not Active, Active",
               "2010, 2070, 1200.0, 0x8, Active, Not Active, Not Active, Not Active",
               "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
               "garbage"]
    s = c.summary()
    assert s["sm_mhz"] == 2010 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_code_hash_ignores_comments_only(tmp_path):
    """The committed counter capture stays attached to the kernel source: comment and blank
    line edits keep the hash, a code edit changes it."""
    import bench
    a = tmp_path / "a.cu"
    a.write_text("int f(int x) {\n    return x + 1;   // add one\n}\n")
    h0 = bench.code_hash(str(a))
    a.write_text("/* doc\n   block */\nint f(int x) {\n\n    return x + 1;   // add 1\n}\n")
    assert bench.code_hash(str(a)) == h0
    a.write_text("int f(int x) {\n    return x + 2;\n}\n")
    assert bench.code_hash(str(a)) != h0


def test_cpu_oracle_one_thread_rate():
    import oracle as O

    import bench
    from paper_2304_12152_gb300 import synth
    O.build()
    n0 = O.num_threads()
    img = synth.contone_image(96, 96, seed=1)
    ws, bs = synth.he_normal_policy(synth.NET_SMALL, 1)
    r = bench.cpu_oracle_one_thread(img, ws, bs, 1, quant=0, mode=1, seconds=0.3)
    assert "error" not in r, r
    assert r["cores"] == 1 and r["value"] > 0 and r["seconds"] > 0
    assert O.num_threads() == n0
