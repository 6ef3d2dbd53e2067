"""Mutation check of the oracle's pins (test infrastructure beside the oracle it checks, run by
hand; pytest does not collect it).

Plants one plausible mistake at a time in a scratch copy of the repository -- a wrong
constant, a dropped term, a flipped sign or index, a transposed operand, a misplaced ring
or bin edge -- in the C oracle or its Python helpers, rebuilds the oracle there, and runs the
CPU suite (`-m "not gpu"`).  Every mutation must make some test fail ("killed"); one that
passes ("SURVIVED") marks a part of the oracle its pins do not fix, unless the mutation
cannot change any result (an equivalent mutation; the two known ones are listed below).

    python oracle/mutation_check.py --scratch /path/to/empty/dir [name-filter ...]

Each mutation reruns the CPU suite (about 5-10 s); the whole check takes 10-15 minutes.  Run
it with nothing else busy on the cores: the oracle's OpenMP thread pools spin while they wait,
and two suites sharing the cores slow each other down many times over.

Known equivalent mutations: including the DC ring (it holds one sample, and rings with fewer
than two samples are skipped) and mapping frequency index n/2 to +n/2 instead of -n/2 (the
radius is unchanged, and the binned form excludes radii >= n/2).
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C = "oracle/ht_oracle.c"
P = "oracle/__init__.py"
M = [
    ("philox multiplier", C, "0xD2511F53u * (uint64_t)c0", "0xD2511F55u * (uint64_t)c0"),
    ("philox 9 rounds", C, "for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {"),
    ("philox key bump", C, "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;"),
    ("philox lo swap", C, "uint32_t n1 = lo1;", "uint32_t n1 = lo0;"),
    ("uniform bits", C, "(double)(x >> 8) * (1.0 / 16777216.0)", "(double)(x >> 9) * (1.0 / 8388608.0)"),
    ("uniform lane", C, "uint32_t x = out[g & 3u];", "uint32_t x = out[(g + 1) & 3u];"),
    ("counter image/stream", C, "{(uint32_t)(g >> 2), image, stream, 0u}", "{(uint32_t)(g >> 2), stream, image, 0u}"),
    ("bf16 spacing", C, "double q = ldexp(1.0, e - 8);", "double q = ldexp(1.0, e - 9);"),
    ("bf16 truncation", C, "return nearbyint(x / q) * q;        /* default", "return trunc(x / q) * q;        /* default"),
    ("e4m3 saturation", C, "if (r > 448.0) r = 448.0;", "if (r > 480.0) r = 480.0;"),
    ("e4m3 subnormal spacing", C, "q = ldexp(1.0, -9);", "q = ldexp(1.0, -10);"),
    ("e4m3 mantissa bits", C, "q = ldexp(1.0, e - 1 - 3);", "q = ldexp(1.0, e - 1 - 2);"),
    ("e4m3 weight scale", C, "s = amax > 0.0 ? amax / 448.0 : 1.0;", "s = amax > 0.0 ? amax / 240.0 : 1.0;"),
    ("forward no bias", C, "for (int k = 0; k < oh * ow; ++k) op[k] = (double)biases[l][o];", "for (int k = 0; k < oh * ow; ++k) op[k] = 0.0;"),
    ("forward kernel flip", C, "double wv = wq[l][(((size_t)o * ci + i) * 3 + ky) * 3 + kx];", "double wv = wq[l][(((size_t)o * ci + i) * 3 + (2 - ky)) * 3 + kx];"),
    ("forward no relu", C, "double v = op[k] > 0.0 ? op[k] : 0.0;", "double v = op[k];"),
    ("forward noise stream", C, "or_uniform(noise_seed, image, 0u, (uint64_t)gy * (uint64_t)w + (uint64_t)gx);", "or_uniform(noise_seed, image, 1u, (uint64_t)gy * (uint64_t)w + (uint64_t)gx);"),
    ("forward noise index transposed", C, "or_uniform(noise_seed, image, 0u, (uint64_t)gy * (uint64_t)w + (uint64_t)gx);", "or_uniform(noise_seed, image, 0u, (uint64_t)gx * (uint64_t)h + (uint64_t)gy);"),
    ("fp8 act quant on last layer", C, "if (quant == 2 && l > 0 && l < L - 1) {", "if (quant == 2 && l > 0) {"),
    ("fp8 act quant skips scale", C, "in[k] = or_round_e4m3(in[k] / s) * s;", "in[k] = or_round_e4m3(in[k]);"),
    ("bf16 act rounding off", C, "if (quant == 1 || quant == 2) v = or_round_bf16(v);", "if (quant == 2) v = or_round_bf16(v);"),
    ("sigmoid sign", C, "prob_out[k] = 1.0 / (1.0 + exp(-in[k]));", "prob_out[k] = 1.0 / (1.0 + exp(in[k]));"),
    ("softmax no max shift denominator", C, "for (int j = 0; j < K; ++j) s += exp(in[(size_t)j * npx + k] - m);", "for (int j = 1; j < K; ++j) s += exp(in[(size_t)j * npx + k] - m);"),
    ("threshold tie", C, "(u < prob[k]) : (prob[k] > 0.5)", "(u < prob[k]) : (prob[k] >= 0.5)"),
    ("bernoulli reversed", C, "(u < prob[k]) : (prob[k] > 0.5)", "(u > prob[k]) : (prob[k] > 0.5)"),
    ("sample stream", C, "double u = mode == 1 ? or_uniform(seed, image, 1u, g) : 0.5;", "double u = mode == 1 ? or_uniform(seed, image, 2u, g) : 0.5;"),
    ("argmax ties", C, "if (prob[(size_t)j * npx + k] > prob[(size_t)lev * npx + k]) lev = j;", "if (prob[(size_t)j * npx + k] >= prob[(size_t)lev * npx + k]) lev = j;"),
    ("gauss sigma^2", C, "/ (2.0 * sigma * sigma));", "/ (sigma * sigma));"),
    ("gauss unnormalised", C, "for (int k = 0; k < n * n; ++k) g[k] /= s;", "for (int k = 0; k < n * n; ++k) g[k] /= 1.0;"),
    ("ssim cov factor", C, "(2.0 * cv2 + o->c2)", "(cv2 + o->c2)"),
    ("ssim var", C, "vh += ww * hv * hv;", "vh += ww * hv;"),
    ("contrast no sqrt", C, "double sig = o->k_contrast * sqrt(vc);", "double sig = o->k_contrast * vc;"),
    ("cssim term", C, "*cssim = sig * s + (1.0 - sig);", "*cssim = sig * s + 1.0;"),
    ("reward sign", C, "out[3] = -out[0] + o->w_s * out[2];", "out[3] = out[0] + o->w_s * out[2];"),
    ("valid width", C, "int vh = h - 2 * r, vw = w - 2 * r;", "int vh = h - 2 * r, vw = w - 2 * r - 1;"),
    ("hvs uses ssim window", C, "double gh = ghvs[(i + r) * n + (j + r)], ww = gw[(i + r) * n + (j + r)];", "double gh = gw[(i + r) * n + (j + r)], ww = gw[(i + r) * n + (j + r)];"),
    ("toggle sign", C, "out[t] = (sum1 - sum0) / M;", "out[t] = (sum0 - sum1) / M;"),
    ("toggle drops first valid row", C, "if (y < r || y >= h - r) continue;\n            for (int x = ax - r;", "if (y <= r || y >= h - r) continue;\n            for (int x = ax - r;"),
    ("toggle multitone unscaled", C, "or_img im = {c, cpitch, hb, hpitch, ay, ax, lev * hscale, hscale};", "or_img im = {c, cpitch, hb, hpitch, ay, ax, lev, hscale};"),
    ("psd normalisation", C, "P[k] = (Fr[k] * Fr[k] + Fi[k] * Fi[k]) / (double)N;", "P[k] = (Fr[k] * Fr[k] + Fi[k] * Fi[k]) / (double)n;"),
    ("dc ring included", C, "if (rr == 0 || cnt[rr] < 2) continue;\n            double mean", "if (cnt[rr] < 2) continue;\n            double mean"),
    ("ring floor", C, "int rr = (int)lround(sqrt((double)(u * u + v * v)));", "int rr = (int)floor(sqrt((double)(u * u + v * v)));"),
    ("centred boundary", C, "static inline int centred(int k, int n) { return k < n / 2 ? k : k - n; }", "static inline int centred(int k, int n) { return k <= n / 2 ? k : k - n; }"),
    ("ring grad factor", C, "G[k] = 2.0 * d;", "G[k] = d;"),
    ("grad scale", C, "grad[k] = 2.0 / (double)N * Yr[k];", "grad[k] = 1.0 / (double)N * Yr[k];"),
    ("bin radial scale", C, "int br = (int)floor(r / half * n_rad);", "int br = (int)floor(r / half * (n_rad - 1));"),
    ("bin A normaliser", C, "A /= (double)(K - 1) * m * m;", "A /= (double)K * m * m;"),
    ("bin dm second term", C, " - 2.0 * (ak - m) * (ak - m) / (m * m * m)) / (K - 1);", ") / (K - 1);"),
    ("bin angle axes", C, "double th = atan2((double)u, (double)v);", "double th = atan2((double)v, (double)u);"),
    ("backward sigmoid'", C, "gout[k] = dprob[k] * p * (1.0 - p);", "gout[k] = dprob[k] * p;"),
    ("backward no relu mask", C, "if (!(acts[l - 1][k] > 0.0)) gin[k] = 0.0;", "if (!(acts[l - 1][k] >= 0.0)) gin[k] = 0.0;"),
    ("backward wgrad flip", C, "gw[l][(((size_t)o * ci + i) * 3 + ky) * 3 + kx] += s;", "gw[l][(((size_t)o * ci + i) * 3 + (2 - ky)) * 3 + kx] += s;"),
    ("backward bias", C, "gb[l][o] += s;", "gb[l][o] += 0.5 * s;"),
    ("backward bf16 weights off", C, "if (quant == 1 && l < L - 1) wv = or_round_bf16(wv);", "if (quant == 3) wv = or_round_bf16(wv);"),
    ("resnet no shortcut", C, "double v = u[k] + x[k];", "double v = u[k];"),
    ("resnet no relu after add", C, "            v = v > 0.0 ? v : 0.0;\n            x[k] = quant", "            x[k] = quant"),
    ("ssim c1", P, "c1=0.01 ** 2", "c1=0.01"),
    ("ssim c2", P, "c2=0.03 ** 2", "c2=0.01 ** 2"),
    ("w_s", P, "w_s=0.06", "w_s=0.6"),
    ("contrast k", P, "k_contrast=2.0", "k_contrast=1.0"),
    ("sigma hvs", P, "sigma_hvs=2.0", "sigma_hvs=1.5"),
    ("le r1/r0", P, "r0 = R - hb * dR", "r0 = R - (1.0 - hb) * dR"),
    ("coma advantage sign", P, "adv = np.where(hb > 0, (1.0 - p) * dR, -p * dR)", "adv = np.where(hb > 0, (1.0 - p) * dR, p * dR)"),
    ("multitone pair clamp", P, "k = np.minimum(np.floor(t), levels - 2).astype(np.int64)", "k = np.minimum(np.floor(t), levels - 1).astype(np.int64)"),
    ("multitone grad scale", P, "return float(val), -dR * (levels - 1)", "return float(val), -dR / (levels - 1)"),
    ("region halo short", C, "or_rect rin = rect_grow(y0, x0, rh, rw, L, h, w);", "or_rect rin = rect_grow(y0, x0, rh, rw, L - 1, h, w);"),
    ("bf16 weights of the head", C, "int inner = (l > 0 && l < L - 1);", "int inner = (l > 0);"),
    ("bf16 weights off", C, "if (quant == 1 && inner) v = or_round_bf16(v);", "if (quant == 3 && inner) v = or_round_bf16(v);"),
    ("toggle M over the whole image", C, "double M = (double)(h - 2 * r) * (w - 2 * r);", "double M = (double)h * w;"),
    ("ring anisotropy normaliser", C, "aniso[rr] = dev2[rr] / (cnt[rr] - 1) / (mean * mean);", "aniso[rr] = dev2[rr] / cnt[rr] / (mean * mean);"),
    ("bin diagonal edge", C, "else if (u == v) bt = n_ang / 4;", "else if (u == v) bt = n_ang / 4 - 1;"),
    ("bin keeps r = n/2", C, "if (r <= 0.0 || r >= half) continue;", "if (r <= 0.0 || r > half) continue;"),
    ("gradient transform sign", C, "dft2(Gr, Gi, n, +1, Yr, Yi);", "dft2(Gr, Gi, n, -1, Yr, Yi);"),
    ("backward noise stream", C, "x0[npx + (size_t)y * w + x] = or_uniform(noise_seed, image, 0u, (uint64_t)y * w + x);", "x0[npx + (size_t)y * w + x] = or_uniform(noise_seed, image, 1u, (uint64_t)y * w + x);"),
    ("resnet stem no relu", C, "double v = x[k] > 0.0 ? x[k] : 0.0;", "double v = x[k];"),
    ("resnet inner act not rounded", C, "t[k] = quant == 1 ? or_round_bf16(v) : v;", "t[k] = v;"),
    ("resnet head on block input", C, "conv3x3_full(x, C, 1, h, w, wq, biases[L - 1], t);", "conv3x3_full(x, C, 1, h, w, wq, biases[0], t);"),
    ("reward level scale", P, "rc = lib().or_reward(c, W, hb, W, H, W, 1.0 / (levels - 1),", "rc = lib().or_reward(c, W, hb, W, H, W, 1.0 / levels,"),
    ("toggle level scale", P, "rc = lib().or_toggle_delta(c, W, hb, W, H, W, 1.0 / (levels - 1),", "rc = lib().or_toggle_delta(c, W, hb, W, H, W, 1.0 / levels,"),
    ("multitone threshold tie", P, "up = (frac > 0.5) if u is None", "up = (frac >= 0.5) if u is None"),
    ("multitone le r_lo", P, "r_lo = R - at_hi * dR", "r_lo = R + at_hi * dR"),
    ("coma log-policy gradient", P, "dlogpi = np.where(hb > 0, 1.0 / np.where(hb > 0, p, 1.0), -1.0 / np.where(hb > 0, 1.0, 1.0 - p))", "dlogpi = np.where(hb > 0, 1.0 / np.where(hb > 0, p, 1.0), 1.0 / np.where(hb > 0, 1.0, 1.0 - p))"),
    ("rect grow clamp", C, "r.yhi = y0 + rh + g > h ? h : y0 + rh + g;", "r.yhi = y0 + rh + g > h ? h - 1 : y0 + rh + g;"),
    ("bf16 subnormal exponent", C, "if (e < -125) e = -125;", "if (e < -126) e = -126;"),
    ("e4m3 negative saturation", C, "if (r < -448.0) r = -448.0;", "if (r < -480.0) r = -480.0;"),
    ("backward gradient rounding off", C, "if (quant == 1) gin[k] = or_round_bf16(gin[k]);", "if (quant == 3) gin[k] = or_round_bf16(gin[k]);"),
    ("bin loss over all radial bins", C, "loss /= n_used;", "loss /= n_rad;"),
    ("sample ignores region offset", C, "uint64_t g = (uint64_t)(y0 + y) * (uint64_t)w + (uint64_t)(x0 + x);", "uint64_t g = (uint64_t)y * (uint64_t)w + (uint64_t)x;"),
    ("resnet halo short", C, "or_rect R = rect_grow(y0, x0, rh, rw, L, H, W);", "or_rect R = rect_grow(y0, x0, rh, rw, L - 1, H, W);"),
    ("resnet noise row pitch", C, "in0[np + (size_t)y * w + xx] = or_uniform(noise_seed, image, 0u, (uint64_t)gy * W + gx);", "in0[np + (size_t)y * w + xx] = or_uniform(noise_seed, image, 0u, (uint64_t)gy * w + gx);"),
    ("resnet output column offset", C, "const double v = t[(size_t)(y0 - R.ylo + y) * w + (x0 - R.xlo + xx)];", "const double v = t[(size_t)(y0 - R.ylo + y) * w + (x0 + xx)];"),
    ("ssim cross term", C, "cv2 += ww * hv * cv;", "cv2 += ww * hv * hv;"),
    ("toggle drops first valid column", C, "if (x < r || x >= w - r) continue;", "if (x <= r || x >= w - r) continue;"),
    ("error map sign", C, "if (e_map) e_map[k] = Hh - Hc;", "if (e_map) e_map[k] = Hc - Hh;"),
    ("forward wrapper drops act scales", P, "noise_seed, image, quant, _ptr(sc),", "noise_seed, image, quant, _ptr(None),"),
    ("sample wrapper drops image index", P, "lib().or_sample(np.ascontiguousarray(probs), K, h, w, y0, x0, rh, rw, mode, seed, image, out, _ptr(u))", "lib().or_sample(np.ascontiguousarray(probs), K, h, w, y0, x0, rh, rw, mode, seed, 0, out, _ptr(u))"),
    ("uniform map image/stream swap", P, "lib().or_uniform_map(seed, image, stream, h, w, out)", "lib().or_uniform_map(seed, stream, image, h, w, out)"),
    ("philox key words swapped", C, "uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};", "uint32_t key[2] = {(uint32_t)(seed >> 32), (uint32_t)seed};"),
    ("spectrum with the inverse transform", C, "dft2(q, NULL, n, -1, Fr, Fi);", "dft2(q, NULL, n, +1, Fr, Fi);"),
    ("ssim mean normaliser", C, "out[1] = ssim / M;", "out[1] = ssim / (M + 1.0);"),
    ("threshold uniform", C, "double u = mode == 1 ? or_uniform(seed, image, 1u, g) : 0.5;", "double u = mode == 1 ? or_uniform(seed, image, 1u, g) : 0.5 + 1e-9;"),
    ("resnet conv1 weights exact", C, "wq[k] = quant == 1 ? or_round_bf16((double)weights[l1][k]) : (double)weights[l1][k];", "wq[k] = (double)weights[l1][k];"),
    ("fp16 spacing", C, "double q = ldexp(1.0, e - 11);", "double q = ldexp(1.0, e - 10);"),
    ("fp16 subnormal exponent", C, "if (e < -13) e = -13;", "if (e < -14) e = -14;"),
    ("fp16 overflow saturates", C, "if (fabs(r) > 65504.0) r = r > 0 ? INFINITY : -INFINITY;", "if (fabs(r) > 65504.0) r = r > 0 ? 65504.0 : -65504.0;"),
    ("fp16 weights not rounded", C, "if (quant == 3 && inner) v = or_round_fp16(v);", ""),
    ("fp16 activations not rounded", C, "                    if (quant == 3) v = or_round_fp16(v);\n", ""),
]



def _copy(dst):
    if os.path.exists(dst):
        shutil.rmtree(dst)
    ign = shutil.ignore_patterns(".git", "_work", "gpurun_out", "__pycache__", ".pytest_cache")
    shutil.copytree(ROOT, dst, ignore=ign, symlinks=True)


def _run_suite(cwd):
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "not gpu", "-x", "-q", "-p", "no:cacheprovider",
                        "--ignore=tests/test_dist_cpu.py"], cwd=cwd, capture_output=True, text=True, timeout=1800)
    first = next((ln[:150] for ln in r.stdout.splitlines() if ln.startswith(("FAILED", "ERROR"))), "")
    return r.returncode, first


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scratch", default=None, help="directory for the scratch copy (default: a temporary one)")
    ap.add_argument("only", nargs="*", help="run only mutations whose name contains one of these")
    args = ap.parse_args()
    scratch = args.scratch or tempfile.mkdtemp(prefix="ht_mutation_")
    mut = os.path.join(scratch, "repo")
    _copy(mut)
    survived = []
    for name, f, old, new in M:
        if args.only and not any(o in name for o in args.only):
            continue
        path = os.path.join(mut, f)
        src = open(path).read()
        if src.count(old) != 1:
            print(f"SKIP      {name}: pattern found {src.count(old)} times", flush=True)
            continue
        open(path, "w").write(src.replace(old, new))
        shutil.rmtree(os.path.join(mut, "oracle", "_build"), ignore_errors=True)
        t = time.time()
        rc, first = _run_suite(mut)
        open(path, "w").write(src)
        shutil.rmtree(os.path.join(mut, "oracle", "_build"), ignore_errors=True)
        status = "killed" if rc != 0 else "SURVIVED"
        if rc == 0:
            survived.append(name)
        print(f"{status:9s} {name:34s} {time.time() - t:5.1f}s  {first}", flush=True)
    print("survived:", survived)
    shutil.rmtree(mut, ignore_errors=True)


if __name__ == "__main__":
    main()
