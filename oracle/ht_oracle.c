/*
 * ht_oracle.c -- plain, slow, FP64 CPU oracle for the halftoning hot path of
 * "Efficient Halftoning via Deep Reinforcement Learning" (arXiv 2304.12152).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) may include, link or call this file; only the tests, the
 * package's smoke check and the CPU-baseline leg of the benchmark do.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Every routine follows the paper's definitions literally (direct loops,
 * direct 11x11 windows, a naive DFT), in double precision:
 *   - Philox4x32-10 .............. Salmon et al., "Parallel random numbers:
 *                                   as easy as 1, 2, 3", SC'11 (published def.)
 *   - policy forward ............. Sec. III (state s = concat(c, z), shared FCN
 *                                   policy, pixel-wise sigmoid), Sec. VI-A
 *   - sampling / thresholding .... Eq. (independent), Algorithm 1 (TEST step)
 *   - reward R = -MSE(HVS) + w_s CSSIM ... Eq. (reward), Eq. (final_reward),
 *                                   Eq. (cssim) and the contrast map (Sec. V)
 *   - toggle deltas dR_a ......... Eq. (le) / Eq. (marl), Sec. III-C
 *   - periodogram, RAPSD, anisotropy, L_AS ... Eqs. (psd), (rapsd), (anis),
 *                                   (as); probability-map proxy (Sec. IV)
 *   - backward through the policy (chain rule, for the finite-difference and
 *     GPU-gradient checks), Algorithm 1 TRAIN step.
 *
 * Readings where the paper is silent are stated next to the code that takes
 * them (3x3 kernels with zero padding 1, Gaussian HVS sigma 2 standing in for
 * the Nasanen model whose constants are not reproduced, SSIM constants of
 * Wang et al. 2004, "valid" metric windows, tie rule h = [p > 0.5]).
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * against closed forms, brute force, invariants or numpy library routines.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11): 4x32-bit counter, 2x32-bit key,     */
/* 10 rounds; round multipliers and Weyl key increments from the paper.      */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in [0,1) with 24 random bits for pixel g (row-major index inside its
 * image) of image `image`, stream `stream` (0 = the policy's noise channel z,
 * 1 + s = Bernoulli sample s).  Key = (seed lo, seed hi);
 * counter = (g / 4, image, stream, 0); output lane g % 4. */
double or_uniform(uint64_t seed, uint32_t image, uint32_t stream, uint64_t g)
{
    uint32_t ctr[4] = {(uint32_t)(g >> 2), image, stream, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    uint32_t x = out[g & 3u];
    return (double)(x >> 8) * (1.0 / 16777216.0);
}

void or_uniform_map(uint64_t seed, uint32_t image, uint32_t stream, int h, int w, double *out)
{
    for (int64_t g = 0; g < (int64_t)h * w; ++g)
        out[g] = or_uniform(seed, image, stream, (uint64_t)g);
}

/* ------------------------------------------------------------------------- */
/* Reduced-precision rounding used to emulate the quantised GPU forms.       */
/* Both are round-to-nearest-even from the exact (double) value.             */
/* ------------------------------------------------------------------------- */
double or_round_bf16(double x)
{
    /* bfloat16: 8 significant bits (1 implicit + 7 stored), fp32 exponent range */
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e);                       /* |x| = m * 2^e, m in [0.5, 1) */
    if (e < -125) e = -125;             /* subnormal range of fp32/bf16 */
    double q = ldexp(1.0, e - 8);       /* spacing of 8-significant-bit numbers */
    return nearbyint(x / q) * q;        /* default rounding mode: to nearest, ties to even */
}

double or_round_fp16(double x)
{
    /* IEEE binary16: 11 significant bits, normal range from 2^-14, subnormal spacing 2^-24,
     * largest finite 65504; a value that rounds past it becomes an infinity, as an IEEE
     * round-to-nearest conversion does. */
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e);                       /* |x| = m * 2^e, m in [0.5, 1) */
    if (e < -13) e = -13;               /* subnormal range: spacing stays 2^-24 */
    double q = ldexp(1.0, e - 11);
    double r = nearbyint(x / q) * q;
    if (fabs(r) > 65504.0) r = r > 0 ? INFINITY : -INFINITY;
    return r;
}

double or_round_e4m3(double x)
{
    /* OCP FP8 E4M3 (fn): bias 7, 3 mantissa bits, max normal 448, min normal 2^-6,
     * subnormal spacing 2^-9; out-of-range values saturate to +-448. */
    if (x == 0.0 || !isfinite(x)) return x;
    double ax = fabs(x);
    double q;
    if (ax < ldexp(1.0, -6)) {
        q = ldexp(1.0, -9);
    } else {
        int e;
        frexp(ax, &e);                  /* ax in [2^(e-1), 2^e) */
        q = ldexp(1.0, e - 1 - 3);
    }
    double r = nearbyint(x / q) * q;
    if (r > 448.0) r = 448.0;
    if (r < -448.0) r = -448.0;
    return r;
}

/* ------------------------------------------------------------------------- */
/* Policy forward (Sec. III "State"/"Agents", Sec. VI-A): a stack of 3x3      */
/* convolutions with zero padding 1 and stride 1 (kernel size and padding are */
/* not stated in the paper; 3x3 / pad 1 is the reading taken), ReLU between  */
/* layers, no ReLU after the last layer, then a pixel-wise sigmoid (one      */
/* logit) or a softmax (K logits).  Input channels: c and z ~ U[0,1) (the    */
/* paper finds U(0,1) equivalent to N(0,1) for the noise map, Sec. VI-D).    */
/*                                                                            */
/* The function evaluates the rectangle [y0,y0+rh) x [x0,x0+rw) of an h x w  */
/* image; every layer's input is zero outside the image, and the noise z is  */
/* keyed by the global pixel index, so any crop equals the same pixels of the */
/* whole-image evaluation.                                                    */
/*                                                                            */
/* quant: 0 = exact FP64;                                                     */
/*        1 = BF16 form: inner layers' weights rounded to bf16, every hidden  */
/*            activation (after ReLU) rounded to bf16; first and last layer   */
/*            weights kept exact;                                             */
/*        2 = FP8 E4M3 form: inner layers' weights quantised per output      */
/*            channel with scale amax_o/448, each inner layer's input         */
/*            activations quantised with the static scale act_scale[l]        */
/*            (l = index of the layer that consumes them); the output of every */
/*            hidden layer is first rounded to bf16 (the storage format);     */
/*        3 = FP16 form: as 1 with IEEE binary16 in place of bf16.            */
/* The quantised forms only decide where rounding happens; accumulation is    */
/* exact (double).                                                            */
/* ------------------------------------------------------------------------- */
typedef struct {
    int ylo, yhi, xlo, xhi;   /* half-open rectangle, inside the image */
} or_rect;

static or_rect rect_grow(int y0, int x0, int rh, int rw, int g, int h, int w)
{
    or_rect r;
    r.ylo = y0 - g < 0 ? 0 : y0 - g;
    r.xlo = x0 - g < 0 ? 0 : x0 - g;
    r.yhi = y0 + rh + g > h ? h : y0 + rh + g;
    r.xhi = x0 + rw + g > w ? w : x0 + rw + g;
    return r;
}

int or_forward(const float *contone, int h, int w, int pitch,
               int n_layers, const int *ch,
               const float *const *weights, const float *const *biases,
               uint64_t noise_seed, uint32_t image, int quant, const double *act_scale,
               int y0, int x0, int rh, int rw,
               double *logits_out,   /* [ch[L]][rh][rw] or NULL */
               double *prob_out,     /* [ch[L]][rh][rw] (sigmoid: 1 channel) or NULL */
               double **save_acts)   /* NULL or n_layers-1 arrays [ch[l]][h][w] (full image only) */
{
    const int L = n_layers;
    if (L < 1 || ch[0] != 2 || h < 1 || w < 1 || rh < 1 || rw < 1 ||
        y0 < 0 || x0 < 0 || y0 + rh > h || x0 + rw > w)
        return OR_EINVAL;
    if (save_acts && (y0 != 0 || x0 != 0 || rh != h || rw != w)) return OR_EINVAL;

    /* quantised weight copies */
    double **wq = (double **)calloc((size_t)L, sizeof(double *));
    if (!wq) return OR_ENOMEM;
    for (int l = 0; l < L; ++l) {
        int ci = ch[l], co = ch[l + 1];
        size_t n = (size_t)co * ci * 9;
        wq[l] = (double *)malloc(n * sizeof(double));
        if (!wq[l]) return OR_ENOMEM;
        int inner = (l > 0 && l < L - 1);
        for (int o = 0; o < co; ++o) {
            double s = 1.0;
            if (quant == 2 && inner) {
                double amax = 0.0;
                for (size_t k = 0; k < (size_t)ci * 9; ++k) {
                    double v = fabs((double)weights[l][(size_t)o * ci * 9 + k]);
                    if (v > amax) amax = v;
                }
                s = amax > 0.0 ? amax / 448.0 : 1.0;
            }
            for (size_t k = 0; k < (size_t)ci * 9; ++k) {
                double v = (double)weights[l][(size_t)o * ci * 9 + k];
                if (quant == 1 && inner) v = or_round_bf16(v);
                if (quant == 2 && inner) v = or_round_e4m3(v / s) * s;
                if (quant == 3 && inner) v = or_round_fp16(v);
                wq[l][(size_t)o * ci * 9 + k] = v;
            }
        }
    }

    /* layer-0 input: c and z over the rectangle grown by L */
    or_rect rin = rect_grow(y0, x0, rh, rw, L, h, w);
    int ih = rin.yhi - rin.ylo, iw = rin.xhi - rin.xlo;
    double *in = (double *)malloc((size_t)2 * ih * iw * sizeof(double));
    if (!in) return OR_ENOMEM;
    for (int y = 0; y < ih; ++y)
        for (int x = 0; x < iw; ++x) {
            int gy = rin.ylo + y, gx = rin.xlo + x;
            in[(size_t)y * iw + x] = (double)contone[(size_t)gy * pitch + gx];
            in[(size_t)ih * iw + (size_t)y * iw + x] =
                or_uniform(noise_seed, image, 0u, (uint64_t)gy * (uint64_t)w + (uint64_t)gx);
        }
    or_rect rprev = rin;

    for (int l = 0; l < L; ++l) {
        int ci = ch[l], co = ch[l + 1];
        int last = (l == L - 1);
        or_rect ro = rect_grow(y0, x0, rh, rw, L - 1 - l, h, w);
        int oh = ro.yhi - ro.ylo, ow = ro.xhi - ro.xlo;
        int ph = rprev.yhi - rprev.ylo, pw = rprev.xhi - rprev.xlo;
        double *out = (double *)malloc((size_t)co * oh * ow * sizeof(double));
        if (!out) return OR_ENOMEM;
        /* FP8 form: quantise this layer's input activations (inner layers) */
        if (quant == 2 && l > 0 && l < L - 1) {
            double s = act_scale ? act_scale[l] : 1.0;
            for (size_t k = 0; k < (size_t)ci * ph * pw; ++k)
                in[k] = or_round_e4m3(in[k] / s) * s;
        }
#pragma omp parallel for schedule(static)
        for (int o = 0; o < co; ++o) {
            double *op = out + (size_t)o * oh * ow;
            for (int k = 0; k < oh * ow; ++k) op[k] = (double)biases[l][o];
            for (int i = 0; i < ci; ++i) {
                const double *ip = in + (size_t)i * ph * pw;
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        double wv = wq[l][(((size_t)o * ci + i) * 3 + ky) * 3 + kx];
                        for (int y = 0; y < oh; ++y) {
                            int gy = ro.ylo + y + ky - 1;      /* input row in image coords */
                            if (gy < 0 || gy >= h) continue;   /* zero padding */
                            const double *irow = ip + (size_t)(gy - rprev.ylo) * pw;
                            double *orow = op + (size_t)y * ow;
                            for (int x = 0; x < ow; ++x) {
                                int gx = ro.xlo + x + kx - 1;
                                if (gx < 0 || gx >= w) continue;
                                orow[x] += wv * irow[gx - rprev.xlo];
                            }
                        }
                    }
            }
            if (!last) {
                for (int k = 0; k < oh * ow; ++k) {
                    double v = op[k] > 0.0 ? op[k] : 0.0;
                    if (quant == 1 || quant == 2) v = or_round_bf16(v);
                    if (quant == 3) v = or_round_fp16(v);
                    op[k] = v;
                }
            }
        }
        if (save_acts && !last)
            memcpy(save_acts[l], out, (size_t)co * oh * ow * sizeof(double));
        free(in);
        in = out;
        rprev = ro;
    }

    /* head */
    int K = ch[L];
    size_t npx = (size_t)rh * rw;
    if (logits_out) memcpy(logits_out, in, (size_t)K * npx * sizeof(double));
    if (prob_out) {
        if (K == 1) {
            for (size_t k = 0; k < npx; ++k) prob_out[k] = 1.0 / (1.0 + exp(-in[k]));
        } else {
            for (size_t k = 0; k < npx; ++k) {
                double m = in[k];
                for (int j = 1; j < K; ++j) if (in[(size_t)j * npx + k] > m) m = in[(size_t)j * npx + k];
                double s = 0.0;
                for (int j = 0; j < K; ++j) s += exp(in[(size_t)j * npx + k] - m);
                for (int j = 0; j < K; ++j) prob_out[(size_t)j * npx + k] = exp(in[(size_t)j * npx + k] - m) / s;
            }
        }
    }
    free(in);
    for (int l = 0; l < L; ++l) free(wq[l]);
    free(wq);
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Actions (Eq. independent; Algorithm 1 TEST step).                          */
/*   threshold mode (mode 0): h_a = [p_a > 0.5]  (Thresholding(., 0.5); the   */
/*     tie p = 0.5 maps to 0, i.e. the Bernoulli rule with u = 0.5);           */
/*   Bernoulli mode (mode 1): h_a = [u_a < p_a], u_a from Philox stream 1.     */
/*   K-level softmax head: level index = smallest k with u < sum_{j<=k} q_j   */
/*     (threshold mode: argmax, lowest index on ties).                         */
/* out: one byte per pixel (level index).                                      */
/* ------------------------------------------------------------------------- */
void or_sample(const double *prob, int K, int h, int w, int y0, int x0, int rh, int rw,
               int mode, uint64_t seed, uint32_t image, uint8_t *out, double *u_out)
{
    size_t npx = (size_t)rh * rw;
    for (int y = 0; y < rh; ++y)
        for (int x = 0; x < rw; ++x) {
            size_t k = (size_t)y * rw + x;
            uint64_t g = (uint64_t)(y0 + y) * (uint64_t)w + (uint64_t)(x0 + x);
            double u = mode == 1 ? or_uniform(seed, image, 1u, g) : 0.5;
            if (u_out) u_out[k] = u;
            if (K == 1) {
                out[k] = (uint8_t)(mode == 1 ? (u < prob[k]) : (prob[k] > 0.5));
            } else if (mode == 1) {
                double cdf = 0.0;
                int lev = K - 1;
                for (int j = 0; j < K; ++j) {
                    cdf += prob[(size_t)j * npx + k];
                    if (u < cdf) { lev = j; break; }
                }
                out[k] = (uint8_t)lev;
            } else {
                int lev = 0;
                for (int j = 1; j < K; ++j) if (prob[(size_t)j * npx + k] > prob[(size_t)lev * npx + k]) lev = j;
                out[k] = (uint8_t)lev;
            }
        }
    (void)h;
}

/* ------------------------------------------------------------------------- */
/* Reward (Eq. reward, Eq. final_reward, Eq. cssim, contrast map of Sec. V).  */
/*                                                                            */
/*   HVS(.)  = normalised (2r+1)x(2r+1) Gaussian low-pass, sigma_hvs (the      */
/*             Gaussian sigma 2 filter the paper reports beside Nasanen's).    */
/*   window w_i = normalised (2r+1)x(2r+1) Gaussian, sigma_ssim (1.5).         */
/*   All windows are "valid" (no padding, Sec. VI-A): outputs at positions     */
/*   y in [r, h-r), x in [r, w-r); M = (h-2r)(w-2r).                           */
/*   MSE   = (1/M) sum (HVS(h) - HVS(c))^2                                     */
/*   SSIM_j = (2 mu_h mu_c + C1)(2 cov + C2) / ((mu_h^2+mu_c^2+C1)(var_h+var_c+C2))*/
/*             with var/cov as window-weighted central moments (Wang 2004).    */
/*   sigma_j = k * sqrt(sum_i w_i (c_i - mu_c)^2), k = 2                       */
/*   CSSIM = (1/M) sum_j [sigma_j SSIM_j + (1 - sigma_j)]                      */
/*   R     = -MSE + w_s * CSSIM                                                */
/* ------------------------------------------------------------------------- */
typedef struct {
    double sigma_hvs, sigma_ssim, k_contrast, w_s, c1, c2;
    int radius;
} or_reward_opts;

static void gauss2d(double sigma, int r, double *g)
{
    int n = 2 * r + 1;
    double s = 0.0;
    for (int i = -r; i <= r; ++i)
        for (int j = -r; j <= r; ++j) {
            double v = exp(-(double)(i * i + j * j) / (2.0 * sigma * sigma));
            g[(i + r) * n + (j + r)] = v;
            s += v;
        }
    for (int k = 0; k < n * n; ++k) g[k] /= s;
}

void or_gauss2d(double sigma, int r, double *g) { gauss2d(sigma, r, g); }

/* Per-output-position terms; hval(y,x) returns the halftone value.  */
/* h holds level indices; the halftone value is index * hscale (hscale = 1 for a
 * binary halftone, 1/(L-1) for L ink levels, Sec. VI-E). */
typedef struct {
    const float *c; int cpitch;
    const uint8_t *hb; int hpitch;
    int fy, fx; double fval;   /* optional override of one pixel (toggle), as a value */
    double hscale;
} or_img;

static inline double img_h(const or_img *im, int y, int x)
{
    if (y == im->fy && x == im->fx) return im->fval;
    return (double)im->hb[(size_t)y * im->hpitch + x] * im->hscale;
}
static inline double img_c(const or_img *im, int y, int x)
{
    return (double)im->c[(size_t)y * im->cpitch + x];
}

/* term_j = -(e_j)^2 + w_s (sigma_j SSIM_j + 1 - sigma_j); also the parts */
static void term_at(const or_img *im, int y, int x, const or_reward_opts *o,
                    const double *ghvs, const double *gw,
                    double *e2, double *ssim, double *cssim)
{
    int r = o->radius, n = 2 * r + 1;
    double Hh = 0, Hc = 0, mh = 0, mc = 0;
    for (int i = -r; i <= r; ++i)
        for (int j = -r; j <= r; ++j) {
            double hv = img_h(im, y + i, x + j), cv = img_c(im, y + i, x + j);
            double gh = ghvs[(i + r) * n + (j + r)], ww = gw[(i + r) * n + (j + r)];
            Hh += gh * hv; Hc += gh * cv;
            mh += ww * hv; mc += ww * cv;
        }
    double vh = 0, vc = 0, cv2 = 0;
    for (int i = -r; i <= r; ++i)
        for (int j = -r; j <= r; ++j) {
            double hv = img_h(im, y + i, x + j) - mh, cv = img_c(im, y + i, x + j) - mc;
            double ww = gw[(i + r) * n + (j + r)];
            vh += ww * hv * hv; vc += ww * cv * cv; cv2 += ww * hv * cv;
        }
    double e = Hh - Hc;
    double s = ((2.0 * mh * mc + o->c1) * (2.0 * cv2 + o->c2)) /
               ((mh * mh + mc * mc + o->c1) * (vh + vc + o->c2));
    double sig = o->k_contrast * sqrt(vc);
    *e2 = e * e;
    *ssim = s;
    *cssim = sig * s + (1.0 - sig);
}

/* out[0..3] = MSE, SSIM (mean map), CSSIM, R; maps (optional, each M values,
 * row-major over the valid region): e (HVS(h)-HVS(c)), SSIM_j, sigma_j. */
int or_reward(const float *c, int cpitch, const uint8_t *hb, int hpitch, int h, int w, double hscale,
              const or_reward_opts *o, double out[4], double *e_map, double *ssim_map, double *sig_map)
{
    int r = o->radius;
    if (h < 2 * r + 1 || w < 2 * r + 1) return OR_EINVAL;
    int n = 2 * r + 1;
    double *ghvs = (double *)malloc((size_t)n * n * sizeof(double));
    double *gw = (double *)malloc((size_t)n * n * sizeof(double));
    gauss2d(o->sigma_hvs, r, ghvs);
    gauss2d(o->sigma_ssim, r, gw);
    or_img im = {c, cpitch, hb, hpitch, -1, -1, 0.0, hscale};
    int vh = h - 2 * r, vw = w - 2 * r;
    /* per-row sums, then a serial sum over rows: the result does not depend on the
     * number of threads or on how OpenMP combines partial sums */
    double *rows = (double *)calloc((size_t)3 * (vh > 0 ? vh : 1), sizeof(double));
#pragma omp parallel for schedule(static)
    for (int y = 0; y < vh; ++y)
        for (int x = 0; x < vw; ++x) {
            double e2, s, cs;
            term_at(&im, y + r, x + r, o, ghvs, gw, &e2, &s, &cs);
            rows[3 * y] += e2; rows[3 * y + 1] += s; rows[3 * y + 2] += cs;
            size_t k = (size_t)y * vw + x;
            if (ssim_map) ssim_map[k] = s;
            if (e_map || sig_map) {
                /* recompute the signed error and the contrast separately */
                double Hh = 0, Hc = 0, mc = 0, vc = 0;
                for (int i = -r; i <= r; ++i)
                    for (int j = -r; j <= r; ++j) {
                        Hh += ghvs[(i + r) * n + (j + r)] * img_h(&im, y + r + i, x + r + j);
                        Hc += ghvs[(i + r) * n + (j + r)] * img_c(&im, y + r + i, x + r + j);
                        mc += gw[(i + r) * n + (j + r)] * img_c(&im, y + r + i, x + r + j);
                    }
                for (int i = -r; i <= r; ++i)
                    for (int j = -r; j <= r; ++j) {
                        double d = img_c(&im, y + r + i, x + r + j) - mc;
                        vc += gw[(i + r) * n + (j + r)] * d * d;
                    }
                if (e_map) e_map[k] = Hh - Hc;
                if (sig_map) sig_map[k] = o->k_contrast * sqrt(vc);
            }
        }
    double mse = 0, ssim = 0, cssim = 0;
    for (int y = 0; y < vh; ++y) {
        mse += rows[3 * y]; ssim += rows[3 * y + 1]; cssim += rows[3 * y + 2];
    }
    free(rows);
    double M = (double)vh * vw;
    out[0] = mse / M;
    out[1] = ssim / M;
    out[2] = cssim / M;
    out[3] = -out[0] + o->w_s * out[2];
    free(ghvs); free(gw);
    return OR_OK;
}

/* Toggle deltas (Eq. le / Eq. marl, Sec. III-C): for each requested pixel a,
 * dR_a = R(h with h_a = 1) - R(h with h_a = 0).  Only the reward terms whose
 * window contains a change; they are recomputed from scratch for both values
 * of h_a (direct windows, no moment updates).  idx: pixel indices y*w+x.
 * Multitone prototype (Sec. VI-E): h holds level indices scaled by hscale, and
 * the two actions of pixel a are the levels lo[a] and lo[a] + 1 around its
 * output: dR_a = R(h_a = (lo_a + 1) hscale) - R(h_a = lo_a hscale) (lo NULL:
 * the binary pair 0, 1). */
int or_toggle_delta(const float *c, int cpitch, const uint8_t *hb, int hpitch, int h, int w, double hscale,
                    const uint8_t *lo, const or_reward_opts *o, const int64_t *idx, int64_t n_idx, double *out)
{
    int r = o->radius;
    if (h < 2 * r + 1 || w < 2 * r + 1) return OR_EINVAL;
    int n = 2 * r + 1;
    double *ghvs = (double *)malloc((size_t)n * n * sizeof(double));
    double *gw = (double *)malloc((size_t)n * n * sizeof(double));
    gauss2d(o->sigma_hvs, r, ghvs);
    gauss2d(o->sigma_ssim, r, gw);
    double M = (double)(h - 2 * r) * (w - 2 * r);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_idx; ++t) {
        int ay = (int)(idx[t] / w), ax = (int)(idx[t] % w);
        double sum1 = 0, sum0 = 0;
        for (int y = ay - r; y <= ay + r; ++y) {
            if (y < r || y >= h - r) continue;
            for (int x = ax - r; x <= ax + r; ++x) {
                if (x < r || x >= w - r) continue;
                for (int b = 0; b < 2; ++b) {
                    const double lev = (lo ? (double)lo[(size_t)ay * w + ax] : 0.0) + (double)b;
                    or_img im = {c, cpitch, hb, hpitch, ay, ax, lev * hscale, hscale};
                    double e2, s, cs;
                    term_at(&im, y, x, o, ghvs, gw, &e2, &s, &cs);
                    double term = -e2 + o->w_s * cs;
                    if (b) sum1 += term; else sum0 += term;
                }
            }
        }
        out[t] = (sum1 - sum0) / M;
    }
    free(ghvs); free(gw);
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Spectrum of a constant-gray patch (Eqs. psd, rapsd, anis, as; Sec. IV).    */
/*   F = 2-D DFT of q (n x n), computed from the definition (row transform     */
/*   then column transform, each a direct O(n^2) sum per output);              */
/*   P(f) = |F(f)|^2 / N, N = n^2.                                             */
/*   Frequencies are centred: u = k for k < n/2, k - n otherwise.             */
/*   Paper form: ring rho = round(sqrt(u^2+v^2)) (annuli of width 1); the DC  */
/*   ring rho = 0 is excluded; rings with fewer than two samples are skipped;  */
/*   rings reach the corners.                                                  */
/*     L_AS = sum_rho sum_{f in rho} (P(f) - Pbar_rho)^2                       */
/*     A(rho) = 1/(n_rho - 1) sum (P(f) - Pbar_rho)^2 / Pbar_rho^2             */
/*   Binned form (32 radial x 16 angular bins): radial bin floor(32 r/(n/2))   */
/*   for 0 < r < n/2; angular bin floor(16 theta/pi), theta = atan2(u, v) mod  */
/*   pi (a direction exactly on a bin edge -- 0, 45, 90, 135 degrees -- is in  */
/*   the bin it opens).  Per radial bin: a_k = mean of P over angular bin k,   */
/*   m = mean of P                                                            */
/*   over the whole radial bin, K = number of non-empty angular bins;          */
/*     A_bin(rho) = 1/(K-1) sum_k (a_k - m)^2 / m^2 ;                          */
/*     L_bin = mean over radial bins with K >= 2 of A_bin.                     */
/*   Gradients w.r.t. q: dL/dq(x) = (2/N) Re sum_f G(f) F(f) e^{+2 pi i f.x/n} */
/*   with G(f) = dL/dP(f).                                                     */
/* ------------------------------------------------------------------------- */
static void dft2(const double *re_in, const double *im_in, int n, int sign, double *re_out, double *im_out)
{
    double *cs = (double *)malloc((size_t)n * sizeof(double));
    double *sn = (double *)malloc((size_t)n * sizeof(double));
    for (int k = 0; k < n; ++k) {
        double a = 2.0 * M_PI * (double)k / (double)n;
        cs[k] = cos(a); sn[k] = sin(a);
    }
    double *tr = (double *)malloc((size_t)n * n * sizeof(double));
    double *ti = (double *)malloc((size_t)n * n * sizeof(double));
    /* rows: T(y, v) = sum_x q(y,x) e^{sign i 2 pi v x / n} */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < n; ++y)
        for (int v = 0; v < n; ++v) {
            double sr = 0, si = 0;
            for (int x = 0; x < n; ++x) {
                int k = (int)(((long)v * x) % n);
                double a = re_in[(size_t)y * n + x], b = im_in ? im_in[(size_t)y * n + x] : 0.0;
                double c = cs[k], s = sign * sn[k];
                sr += a * c - b * s;
                si += a * s + b * c;
            }
            tr[(size_t)y * n + v] = sr; ti[(size_t)y * n + v] = si;
        }
    /* columns: F(u, v) = sum_y T(y,v) e^{sign i 2 pi u y / n} */
#pragma omp parallel for schedule(static)
    for (int u = 0; u < n; ++u)
        for (int v = 0; v < n; ++v) {
            double sr = 0, si = 0;
            for (int y = 0; y < n; ++y) {
                int k = (int)(((long)u * y) % n);
                double a = tr[(size_t)y * n + v], b = ti[(size_t)y * n + v];
                double c = cs[k], s = sign * sn[k];
                sr += a * c - b * s;
                si += a * s + b * c;
            }
            re_out[(size_t)u * n + v] = sr; im_out[(size_t)u * n + v] = si;
        }
    free(cs); free(sn); free(tr); free(ti);
}

void or_dft2(const double *re_in, const double *im_in, int n, int sign, double *re_out, double *im_out)
{
    dft2(re_in, im_in, n, sign, re_out, im_out);
}

static inline int centred(int k, int n) { return k < n / 2 ? k : k - n; }

/* mode 0 = paper form (Eq. as), mode 1 = binned form.
 * out[0] = loss; aniso (optional): paper-form A(rho) for rho = 0..n_rings-1
 * (NaN where undefined); grad (optional): dL/dq, n*n. Returns number of rings. */
int or_anisotropy_loss(const double *q, int n, int mode, int n_rad, int n_ang,
                       double *out, double *aniso, int n_aniso, double *psd_out, double *grad)
{
    if (n < 4 || (n & 1)) return -1;
    size_t N = (size_t)n * n;
    double *Fr = (double *)malloc(N * sizeof(double));
    double *Fi = (double *)malloc(N * sizeof(double));
    double *P = (double *)malloc(N * sizeof(double));
    double *G = (double *)calloc(N, sizeof(double));
    dft2(q, NULL, n, -1, Fr, Fi);
    for (size_t k = 0; k < N; ++k) P[k] = (Fr[k] * Fr[k] + Fi[k] * Fi[k]) / (double)N;
    if (psd_out) memcpy(psd_out, P, N * sizeof(double));

    int n_rings = (int)lround(sqrt(2.0) * (n / 2)) + 1;
    double loss = 0.0;
    if (mode == 0) {
        double *sum = (double *)calloc((size_t)n_rings, sizeof(double));
        int *cnt = (int *)calloc((size_t)n_rings, sizeof(int));
        int *ring = (int *)malloc(N * sizeof(int));
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                int u = centred(a, n), v = centred(b, n);
                int rr = (int)lround(sqrt((double)(u * u + v * v)));
                ring[(size_t)a * n + b] = rr;
                sum[rr] += P[(size_t)a * n + b];
                cnt[rr] += 1;
            }
        double *dev2 = (double *)calloc((size_t)n_rings, sizeof(double));
        for (size_t k = 0; k < N; ++k) {
            int rr = ring[k];
            if (rr == 0 || cnt[rr] < 2) continue;
            double mean = sum[rr] / cnt[rr];
            double d = P[k] - mean;
            dev2[rr] += d * d;
            loss += d * d;
            G[k] = 2.0 * d;      /* the derivative through the ring mean cancels */
        }
        if (aniso)
            for (int rr = 0; rr < n_aniso; ++rr) {
                if (rr >= n_rings || rr == 0 || cnt[rr] < 2) { aniso[rr] = NAN; continue; }
                double mean = sum[rr] / cnt[rr];
                aniso[rr] = dev2[rr] / (cnt[rr] - 1) / (mean * mean);
            }
        free(sum); free(cnt); free(ring); free(dev2);
    } else {
        int nb = n_rad * n_ang;
        double *bsum = (double *)calloc((size_t)nb, sizeof(double));
        int *bcnt = (int *)calloc((size_t)nb, sizeof(int));
        int *bidx = (int *)malloc(N * sizeof(int));
        double half = (double)(n / 2);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                int u = centred(a, n), v = centred(b, n);
                double r = sqrt((double)(u * u + v * v));
                size_t k = (size_t)a * n + b;
                bidx[k] = -1;
                if (r <= 0.0 || r >= half) continue;
                int br = (int)floor(r / half * n_rad);
                if (br >= n_rad) br = n_rad - 1;
                int bt;
                if ((n_ang % 4) == 0 && (u == 0 || v == 0 || u == v || u == -v)) {
                    /* directions on a bin edge (0, 45, 90, 135 degrees) open their bin */
                    if (u == 0) bt = 0;
                    else if (v == 0) bt = n_ang / 2;
                    else if (u == v) bt = n_ang / 4;
                    else bt = 3 * n_ang / 4;
                } else {
                    double th = atan2((double)u, (double)v);
                    if (th < 0) th += M_PI;
                    if (th >= M_PI) th -= M_PI;
                    bt = (int)floor(th / M_PI * n_ang);
                    if (bt >= n_ang) bt = n_ang - 1;
                }
                bidx[k] = br * n_ang + bt;
                bsum[br * n_ang + bt] += P[k];
                bcnt[br * n_ang + bt] += 1;
            }
        /* per radial bin statistics and dL/da_k, dL/dm */
        double *dA_da = (double *)calloc((size_t)nb, sizeof(double));
        double *dA_dm = (double *)calloc((size_t)n_rad, sizeof(double));
        int *rcnt = (int *)calloc((size_t)n_rad, sizeof(int));
        int n_used = 0;
        for (int br = 0; br < n_rad; ++br) {
            double tot = 0.0; int cnt = 0, K = 0;
            for (int bt = 0; bt < n_ang; ++bt) {
                tot += bsum[br * n_ang + bt]; cnt += bcnt[br * n_ang + bt];
                if (bcnt[br * n_ang + bt] > 0) K++;
            }
            rcnt[br] = cnt;
            if (K < 2) { rcnt[br] = 0; continue; }
            n_used++;
            double m = tot / cnt;
            double A = 0.0, dm = 0.0;
            for (int bt = 0; bt < n_ang; ++bt) {
                int j = br * n_ang + bt;
                if (bcnt[j] == 0) continue;
                double ak = bsum[j] / bcnt[j];
                A += (ak - m) * (ak - m);
                dA_da[j] = 2.0 * (ak - m) / (m * m) / (K - 1);
                dm += (-2.0 * (ak - m) / (m * m) - 2.0 * (ak - m) * (ak - m) / (m * m * m)) / (K - 1);
            }
            A /= (double)(K - 1) * m * m;
            dA_dm[br] = dm;
            loss += A;
        }
        if (n_used > 0) {
            loss /= n_used;
            for (size_t k = 0; k < N; ++k) {
                int j = bidx[k];
                if (j < 0) continue;
                int br = j / n_ang;
                if (rcnt[br] == 0) continue;
                G[k] = (dA_da[j] / bcnt[j] + dA_dm[br] / rcnt[br]) / n_used;
            }
        }
        if (aniso) for (int k = 0; k < n_aniso; ++k) aniso[k] = NAN;
        free(bsum); free(bcnt); free(bidx); free(dA_da); free(dA_dm); free(rcnt);
    }
    out[0] = loss;
    if (grad) {
        double *Gr = (double *)malloc(N * sizeof(double));
        double *Gi = (double *)malloc(N * sizeof(double));
        double *Yr = (double *)malloc(N * sizeof(double));
        double *Yi = (double *)malloc(N * sizeof(double));
        for (size_t k = 0; k < N; ++k) { Gr[k] = G[k] * Fr[k]; Gi[k] = G[k] * Fi[k]; }
        dft2(Gr, Gi, n, +1, Yr, Yi);
        for (size_t k = 0; k < N; ++k) grad[k] = 2.0 / (double)N * Yr[k];
        free(Gr); free(Gi); free(Yr); free(Yi);
    }
    free(Fr); free(Fi); free(P); free(G);
    return n_rings;
}

/* ------------------------------------------------------------------------- */
/* Backward through the policy (Algorithm 1 TRAIN step, chain rule).          */
/* Given dL/dp on the whole image (sigmoid head), the saved hidden            */
/* activations of or_forward(save_acts) and the exact logits, accumulate      */
/* dL/dW (OIHW) and dL/db into gw/gb (double, caller zeroes them).            */
/* ReLU derivative: 1 where the activation is > 0, else 0.                    */
/* quant 1 (BF16 form, with acts from the quant-1 forward): the data          */
/* gradient of an inner (64 -> 64) layer uses that layer's bf16-rounded        */
/* weights, as its forward does, and every hidden layer's pre-activation       */
/* gradient (after the ReLU mask) is rounded to bf16, the precision it is      */
/* stored in between layers.  The head's and layer 1's weights stay exact.     */
/* ------------------------------------------------------------------------- */
int or_backward(const float *contone, int h, int w, int pitch,
                int n_layers, const int *ch, const float *const *weights,
                uint64_t noise_seed, uint32_t image, int quant,
                const double *const *acts, const double *logits, const double *dprob,
                double **gw, double **gb)
{
    const int L = n_layers;
    if (ch[L] != 1) return OR_EINVAL;
    size_t npx = (size_t)h * w;
    /* input channels */
    double *x0 = (double *)malloc(2 * npx * sizeof(double));
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            x0[(size_t)y * w + x] = (double)contone[(size_t)y * pitch + x];
            x0[npx + (size_t)y * w + x] = or_uniform(noise_seed, image, 0u, (uint64_t)y * w + x);
        }
    /* dL/dz for the logit: sigmoid' = p(1-p) */
    double *gout = (double *)malloc(npx * sizeof(double));
    for (size_t k = 0; k < npx; ++k) {
        double p = 1.0 / (1.0 + exp(-logits[k]));
        gout[k] = dprob[k] * p * (1.0 - p);
    }
    for (int l = L - 1; l >= 0; --l) {
        int ci = ch[l], co = ch[l + 1];
        const double *in = l == 0 ? x0 : acts[l - 1];
        /* bias and weight gradients */
        for (int o = 0; o < co; ++o) {
            double s = 0;
            for (size_t k = 0; k < npx; ++k) s += gout[(size_t)o * npx + k];
            gb[l][o] += s;
        }
#pragma omp parallel for schedule(static)
        for (int o = 0; o < co; ++o)
            for (int i = 0; i < ci; ++i)
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        double s = 0;
                        for (int y = 0; y < h; ++y) {
                            int yy = y + ky - 1;
                            if (yy < 0 || yy >= h) continue;
                            for (int x = 0; x < w; ++x) {
                                int xx = x + kx - 1;
                                if (xx < 0 || xx >= w) continue;
                                s += gout[(size_t)o * npx + (size_t)y * w + x] * in[(size_t)i * npx + (size_t)yy * w + xx];
                            }
                        }
                        gw[l][(((size_t)o * ci + i) * 3 + ky) * 3 + kx] += s;
                    }
        if (l == 0) break;
        /* gradient w.r.t. this layer's input, masked by the previous ReLU */
        double *gin = (double *)calloc((size_t)ci * npx, sizeof(double));
#pragma omp parallel for schedule(static)
        for (int i = 0; i < ci; ++i)
            for (int o = 0; o < co; ++o)
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        double wv = (double)weights[l][(((size_t)o * ci + i) * 3 + ky) * 3 + kx];
                        if (quant == 1 && l < L - 1) wv = or_round_bf16(wv);
                        for (int y = 0; y < h; ++y) {
                            int yy = y + ky - 1;
                            if (yy < 0 || yy >= h) continue;
                            for (int x = 0; x < w; ++x) {
                                int xx = x + kx - 1;
                                if (xx < 0 || xx >= w) continue;
                                gin[(size_t)i * npx + (size_t)yy * w + xx] += wv * gout[(size_t)o * npx + (size_t)y * w + x];
                            }
                        }
                    }
        for (size_t k = 0; k < (size_t)ci * npx; ++k) {
            if (!(acts[l - 1][k] > 0.0)) gin[k] = 0.0;
            if (quant == 1) gin[k] = or_round_bf16(gin[k]);
        }
        free(gout);
        gout = gin;
    }
    free(gout); free(x0);
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Residual policy of Sec. VI-A (He et al. 2016 blocks): a stem convolution   */
/* 2 -> C with ReLU, n_blocks residual blocks                                 */
/*   y = ReLU(x + conv2(ReLU(conv1(x))))   (identity shortcut, C -> C)         */
/* and an output convolution C -> 1 followed by the sigmoid.  All 3x3, stride  */
/* 1, zero padding 1.  Layers in order: stem, (conv1, conv2) per block, out;   */
/* weights OIHW.  Whole image only.  quant 1 (BF16 form): block weights and   */
/* every stored activation (stem output, conv1 output, block output) rounded  */
/* to bf16; the stem and output weights stay exact.                            */
/* ------------------------------------------------------------------------- */
static void conv3x3_full(const double *in, int ci, int co, int h, int w, const double *wt, const float *b,
                         double *out)
{
    size_t np = (size_t)h * w;
#pragma omp parallel for schedule(static)
    for (int o = 0; o < co; ++o) {
        double *op = out + (size_t)o * np;
        for (size_t k = 0; k < np; ++k) op[k] = (double)b[o];
        for (int i = 0; i < ci; ++i)
            for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                    double wv = wt[(((size_t)o * ci + i) * 3 + ky) * 3 + kx];
                    for (int y = 0; y < h; ++y) {
                        int yy = y + ky - 1;
                        if (yy < 0 || yy >= h) continue;
                        for (int x = 0; x < w; ++x) {
                            int xx = x + kx - 1;
                            if (xx < 0 || xx >= w) continue;
                            op[(size_t)y * w + x] += wv * in[(size_t)i * np + (size_t)yy * w + xx];
                        }
                    }
                }
    }
}

int or_forward_resnet(const float *contone, int H, int W, int pitch, int n_blocks, int C,
                      const float *const *weights, const float *const *biases, uint64_t noise_seed, uint32_t image,
                      int quant, int y0, int x0, int rh, int rw, double *logits_out, double *prob_out)
{
    /* outputs over the rectangle (y0, x0, rh, rw): the net runs on the rectangle grown
     * by L pixels (clamped to the image; its cut edges are zero-padded, which only
     * reaches L pixels in) with the noise channel at image coordinates */
    if (H < 1 || W < 1 || n_blocks < 0 || C < 1 || rh < 1 || rw < 1 || y0 < 0 || x0 < 0 || y0 + rh > H ||
        x0 + rw > W)
        return OR_EINVAL;
    const int L = 2 + 2 * n_blocks;
    or_rect R = rect_grow(y0, x0, rh, rw, L, H, W);
    const int h = R.yhi - R.ylo, w = R.xhi - R.xlo;
    size_t np = (size_t)h * w;
    double *x = (double *)malloc((size_t)C * np * sizeof(double));
    double *t = (double *)malloc((size_t)C * np * sizeof(double));
    double *u = (double *)malloc((size_t)C * np * sizeof(double));
    double *in0 = (double *)malloc(2 * np * sizeof(double));
    double *wq = (double *)malloc((size_t)C * C * 9 * sizeof(double));
    if (!x || !t || !u || !in0 || !wq) return OR_ENOMEM;
    for (int y = 0; y < h; ++y)
        for (int xx = 0; xx < w; ++xx) {
            const int gy = R.ylo + y, gx = R.xlo + xx;
            in0[(size_t)y * w + xx] = (double)contone[(size_t)gy * pitch + gx];
            in0[np + (size_t)y * w + xx] = or_uniform(noise_seed, image, 0u, (uint64_t)gy * W + gx);
        }
    /* stem */
    for (size_t k = 0; k < (size_t)C * 2 * 9; ++k) wq[k] = (double)weights[0][k];
    conv3x3_full(in0, 2, C, h, w, wq, biases[0], x);
    for (size_t k = 0; k < (size_t)C * np; ++k) {
        double v = x[k] > 0.0 ? x[k] : 0.0;
        x[k] = quant == 1 ? or_round_bf16(v) : v;
    }
    for (int b = 0; b < n_blocks; ++b) {
        const int l1 = 1 + 2 * b, l2 = l1 + 1;
        for (size_t k = 0; k < (size_t)C * C * 9; ++k)
            wq[k] = quant == 1 ? or_round_bf16((double)weights[l1][k]) : (double)weights[l1][k];
        conv3x3_full(x, C, C, h, w, wq, biases[l1], t);
        for (size_t k = 0; k < (size_t)C * np; ++k) {
            double v = t[k] > 0.0 ? t[k] : 0.0;
            t[k] = quant == 1 ? or_round_bf16(v) : v;
        }
        for (size_t k = 0; k < (size_t)C * C * 9; ++k)
            wq[k] = quant == 1 ? or_round_bf16((double)weights[l2][k]) : (double)weights[l2][k];
        conv3x3_full(t, C, C, h, w, wq, biases[l2], u);
        for (size_t k = 0; k < (size_t)C * np; ++k) {
            double v = u[k] + x[k];
            v = v > 0.0 ? v : 0.0;
            x[k] = quant == 1 ? or_round_bf16(v) : v;
        }
    }
    for (size_t k = 0; k < (size_t)C * 9; ++k) wq[k] = (double)weights[L - 1][k];
    conv3x3_full(x, C, 1, h, w, wq, biases[L - 1], t);
    for (int y = 0; y < rh; ++y)
        for (int xx = 0; xx < rw; ++xx) {
            const double v = t[(size_t)(y0 - R.ylo + y) * w + (x0 - R.xlo + xx)];
            if (logits_out) logits_out[(size_t)y * rw + xx] = v;
            if (prob_out) prob_out[(size_t)y * rw + xx] = 1.0 / (1.0 + exp(-v));
        }
    free(x); free(t); free(u); free(in0); free(wq);
    return OR_OK;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
