// train.cu -- one iteration of Algorithm 1 (TRAIN step): forward and backward.
//
// Two forms.  A BF16 policy of the 2 -> 64 x (L-1) -> 1 shape runs the
// tensor-core form of train_tc.cu (forward on the conv pipeline with saved
// bf16 activations, tcgen05 weight gradients, data gradients on the pipeline);
// an FP32 policy runs the plain form below on CUDA cores.  Steps 2-6 are shared.
//
// Forward (ht_train_step_fwd):
//   1. policy forward on every crop and every constant-gray patch, keeping each
//      hidden activation for the backward pass;
//   2. per crop, S Bernoulli samples h^s = [u^s < p] (Philox stream 1 + s)
//      (Eq. independent: all agents act at once);
//   3. per sample, reward R(h^s) and toggle deltas dR^s (Eq. final_reward,
//      Eq. le, Sec. III-C);
//   4. L_MARL = -(1/(B S)) sum_{i,s} sum_a sum_{h'} R({h'_a, h_-a}) pi_a(h')
//      (Algorithm 1, Eq. marl) with R({h'_a, h_-a}) = R + (h'_a - h_a) dR_a, so
//      dL_MARL/dp_a = -(1/(B S)) sum_s dR^s_a  (or the COMA estimator, k_marl);
//   5. L_AS on the gray patches' probability maps (Sec. IV, Eq. as, proxy
//      p(h = 1 | c_g, z_g)), averaged over patches, with its gradient;
//   6. L_total = L_MARL + w_a L_AS.
// Backward (ht_train_step_bwd): dL/dz = dL/dp p (1 - p) through the sigmoid,
// then per layer a weight-gradient reduction over pixels and a data gradient
// (3x3 convolution with the flipped, transposed weights) masked by the ReLU of
// the layer's input.
#include <string.h>

#include <vector>

#include "head.cuh"

struct ht_train {
    ht_policy *p;
    ht_train_desc d;
    int hidden_ch_sum;             // sum of hidden widths (activations kept per pixel)
    size_t crop_px, gray_px;
    float *acts = nullptr;         // per image: sum_l ch[l+1] planes
    float *prob = nullptr;         // per image: [h][w]
    float *dprob = nullptr;        // per image: [h][w]
    uint32_t *tbits = nullptr;     // threshold bits of the forward (unused output)
    uint32_t *sbits = nullptr;     // [B][S][h][words]
    float *dR = nullptr;           // [B][S][h][w]
    float *gray_img = nullptr;     // [G][n][n]
    float *gbuf[2] = {nullptr, nullptr};
    float *wflip = nullptr;
    float *toggle_scratch = nullptr;
    size_t toggle_scratch_floats = 0;
    void *las_scratch = nullptr;
    size_t las_scratch_bytes = 0;
    double *dacc = nullptr;        // [0] L_MARL, [1..G] L_AS per patch, rewards [B*S*4]
    int n_last = 0;                // crops in the last forward
    bool fwd_done = false;         // a forward has run (its buffers hold what the backward needs)
    uint64_t seed_last = 0;
    std::vector<ht_image> crops_last;
    bool tc = false;               // BF16 tensor-core form (train_tc.cu)
    ht_train_tc_ws tcw;
};

namespace {

__global__ void k_fill(float *p, size_t n, float v)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// h^s = [u^s < p], u^s from Philox stream 1 + s; packed LSB-first, 32 px per warp.
// Multitone prototype (levels > 2, Sec. VI-E): level k + [u^s < frac] with k, frac
// from v (L - 1), 2 bits per pixel.
// blockIdx.z = i S + s over all crops i (probability maps px apart) and samples s.
__global__ void k_sample_bits(const float *__restrict__ prob0, size_t px, int H, int W, int words, uint64_t seed, int S,
                              int levels, uint32_t *__restrict__ bits0)
{
    const int z = blockIdx.z, i = z / S, sm = z % S;
    const float *prob = prob0 + (size_t)i * px;
    uint32_t *bits = bits0 + (size_t)z * H * words;
    const int y = blockIdx.y, x0 = blockIdx.x * 32, x = x0 + threadIdx.x;
    const bool inside = x < W;
    const float u = inside ? ht_uniform24(seed, (uint32_t)i, 1u + (uint32_t)sm, (uint64_t)y * W + x) : 0.f;
    const float v = inside ? prob[(size_t)y * W + x] : 0.f;
    if (levels > 2) {
        const float t = v * (float)(levels - 1);
        const int k = min((int)floorf(t), levels - 2);
        ht_pack2(k + (u < t - (float)k ? 1 : 0), inside, (int)threadIdx.x, x0, y, H, bits, words);
        return;
    }
    const uint32_t word = __ballot_sync(0xffffffffu, inside && u < v);
    if (threadIdx.x == 0) bits[(size_t)y * words + (x0 >> 5)] = word;
}

// Local expectation (Eq. le, Eq. marl):
//   dp_a = -inv * sum_s dR^s_a; L += -inv * sum_s sum_a (R_s + (p_a - h_a) dR_a)
// COMA (Eq. coma, baseline Eq. baseline), R - b_a = (1 - p) dR if h_a = 1, -p dR if 0:
//   dp_a = -inv * sum_s (d log pi_a(h_a) / dp_a) (R - b_a)
//        = -inv * sum_s dR^s_a * ((1 - p) / p if h_a = 1, p / (1 - p) if 0)
//   L += -inv * sum_s sum_a log pi_a(h_a) (R - b_a)
// (h_a = 1 needs u < p, so p > 0; h_a = 0 needs p <= u < 1: no division by zero.)
// Multitone prototype (levels L > 2, Sec. VI-E): actions lo = k, hi = k + 1 around v,
// pi(hi) = frac, dR = R(hi) - R(lo), so dL/dv_a = -(L - 1) sum_s dR^s_a and
//   L += -inv * sum_s sum_a (frac R(hi) + (1 - frac) R(lo)).
// blockIdx.y = crop i (maps npx apart; S samples per crop).
__global__ void k_marl(const float *__restrict__ prob0, const float *__restrict__ dR0, const uint32_t *__restrict__ bits0,
                       const double *__restrict__ rewards0, int S, int H, int W, int words, double inv, int coma,
                       int levels, float *__restrict__ dprob0, double *__restrict__ loss)
{
    const size_t npx = (size_t)H * W;
    const int i = blockIdx.y;
    const float *prob = prob0 + (size_t)i * npx;
    const float *dR = dR0 + (size_t)i * S * npx;
    const uint32_t *bits = bits0 + (size_t)i * S * H * words;
    const double *rewards = rewards0 + (size_t)i * S * 4;
    float *dprob = dprob0 + (size_t)i * npx;
    const size_t a = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (a < npx) {
        const int y = (int)(a / W), x = (int)(a % W);
        const float p = prob[a];
        double g = 0.0;
        const float t = p * (float)(levels - 1);
        const int k = min((int)floorf(t), levels - 2);
        const float frac = t - (float)k;
        for (int s = 0; s < S; ++s) {
            const float d = dR[(size_t)s * npx + a];
            if (levels > 2) {
                const uint32_t wd = bits[(size_t)s * H * words + (size_t)y * words + (x >> 4)];
                const bool at_hi = (int)((wd >> (2 * (x & 15))) & 3u) == k + 1;
                const double R = rewards[4 * s + 3];
                const double r_hi = R + (at_hi ? 0.0 : (double)d), r_lo = R - (at_hi ? (double)d : 0.0);
                g += d * (float)(levels - 1);
                l += -((double)frac * r_hi + (1.0 - (double)frac) * r_lo);
                continue;
            }
            const bool hb = (bits[(size_t)s * H * words + (size_t)y * words + (x >> 5)] >> (x & 31)) & 1u;
            if (coma) {
                g += hb ? d * ((1.f - p) / p) : d * (p / (1.f - p));
                const float adv = hb ? (1.f - p) * d : -p * d;
                l += -(double)(hb ? logf(p) : log1pf(-p)) * (double)adv;
            } else {
                g += d;
                l += -(rewards[4 * s + 3] + ((double)p - (hb ? 1.0 : 0.0)) * (double)d);
            }
        }
        dprob[a] = (float)(-inv * g);
        l *= inv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

__global__ void k_scale_into(const float *__restrict__ src, float s, size_t n, float *__restrict__ dst)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = s * src[i];
}

// dL/dz = dL/dp * p * (1 - p)
__global__ void k_dlogit(const float *__restrict__ dp, const float *__restrict__ p, size_t n, float *__restrict__ g)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) g[i] = dp[i] * p[i] * (1.f - p[i]);
}

// wt[c][o][ky][kx] = W[o][c][2-ky][2-kx]
__global__ void k_flip(const float *__restrict__ w, int Cout, int Cin, float *__restrict__ wt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Cout * Cin * 9) return;
    const int o = i / (Cin * 9), c = (i / 9) % Cin, t = i % 9;
    wt[((size_t)c * Cout + o) * 9 + (8 - t)] = w[i];
}

// Weight and bias gradients of one layer:
//   dW[o][c][ky][kx] += sum_{y,x} g[o][y][x] in[c][y+ky-1][x+kx-1] (zero outside)
//   db[o] += sum g[o]
// Block: 16 output x 16 input channels (thread = (o, c), 9 taps each) over a chunk
// of 32-pixel row segments staged in shared memory; partial sums are added to
// global memory with one atomic per weight per block.
constexpr int WG_O = 16, WG_C = 16, WG_SEGS = 64;

__global__ void __launch_bounds__(256) k_wgrad(const float *__restrict__ g, const float *__restrict__ in,
                                               const float *__restrict__ contone, int cpitch, uint64_t seed,
                                               uint32_t image, int Cout, int Cin, int H, int W,
                                               float *__restrict__ dW, float *__restrict__ db)
{
    __shared__ float s_g[WG_O][32];
    __shared__ float s_in[WG_C][3][34];
    const int tid = threadIdx.x;
    const int o0 = blockIdx.x * WG_O, c0 = blockIdx.y * WG_C;
    const int ol = tid / WG_C, cl = tid % WG_C;
    const int o = o0 + ol, c = c0 + cl;
    const int nseg = (W + 31) / 32;
    const size_t plane = (size_t)H * W;
    float acc[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = 0.f;
    float bacc = 0.f;
    const long seg0 = (long)blockIdx.z * WG_SEGS, seg1 = min((long)H * nseg, seg0 + WG_SEGS);
    for (long sg = seg0; sg < seg1; ++sg) {
        const int y = (int)(sg / nseg), x0 = (int)(sg % nseg) * 32;
        __syncthreads();
        for (int i = tid; i < WG_O * 32; i += 256) {
            const int oo = i / 32, xx = i % 32;
            const int gx = x0 + xx;
            s_g[oo][xx] = (o0 + oo < Cout && gx < W) ? g[(size_t)(o0 + oo) * plane + (size_t)y * W + gx] : 0.f;
        }
        for (int i = tid; i < WG_C * 3 * 34; i += 256) {
            const int cc = i / (3 * 34), r = (i / 34) % 3, xx = i % 34;
            const int gy = y + r - 1, gx = x0 + xx - 1;
            float v = 0.f;
            if (c0 + cc < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W) {
                if (contone) v = (c0 + cc == 0) ? contone[(size_t)gy * cpitch + gx]
                                               : ht_uniform24(seed, image, 0u, (uint64_t)gy * W + gx);
                else v = in[(size_t)(c0 + cc) * plane + (size_t)gy * W + gx];
            }
            s_in[cc][r][xx] = v;
        }
        __syncthreads();
        for (int xx = 0; xx < 32; ++xx) {
            const float gv = s_g[ol][xx];
            bacc += gv;
#pragma unroll
            for (int t = 0; t < 9; ++t) acc[t] = fmaf(gv, s_in[cl][t / 3][xx + t % 3], acc[t]);
        }
    }
    if (o < Cout && c < Cin) {
#pragma unroll
        for (int t = 0; t < 9; ++t) atomicAdd(&dW[((size_t)o * Cin + c) * 9 + t], acc[t]);
    }
    if (c0 == 0 && cl == 0 && o < Cout) atomicAdd(&db[o], bacc);
}

unsigned nblk(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

size_t image_act_floats(const ht_train *t, size_t px) { return (size_t)t->hidden_ch_sum * px; }

float *act_ptr(ht_train *t, int img, int layer)
{
    // images 0..B-1 are crops, B..B+G-1 gray patches
    const ht_policy *p = t->p;
    const int B = t->d.max_crops;
    size_t base = img < B ? image_act_floats(t, t->crop_px) * img
                          : image_act_floats(t, t->crop_px) * B + image_act_floats(t, t->gray_px) * (img - B);
    const size_t px = img < B ? t->crop_px : t->gray_px;
    for (int l = 0; l < layer; ++l) base += (size_t)p->ch[l + 1] * px;
    return t->acts + base;
}

size_t img_px_offset(const ht_train *t, int img)
{
    const int B = t->d.max_crops;
    return img < B ? t->crop_px * img : t->crop_px * B + t->gray_px * (img - B);
}

}  // namespace

extern "C" {

ht_status ht_train_create(ht_policy *p, const ht_train_desc *d, ht_train **out)
{
    HT_RANGE("ht_train_create");
    HT_CHECK_ARG(p && d && out, "null argument");
    *out = nullptr;
    HT_CHECK_ARG(p->head == HT_HEAD_SIGMOID || p->head == HT_HEAD_MULTITONE,
                 "training needs a sigmoid-output head (binary or the multitoning prototype)");
    HT_CHECK_ARG(p->head == HT_HEAD_SIGMOID || d->estimator == HT_EST_LE,
                 "the multitoning prototype trains with the local-expectation estimator");
    if (p->prec == HT_FP8_E4M3 || p->prec == HT_FP16 || (p->prec == HT_BF16 && !ht_train_tc_supported(p))) {
        ht_set_error("training supports the FP32 form and the BF16 form of 2 -> 64 x (L-1) -> 1 policies");
        return HT_ERR_UNSUPPORTED;
    }
    HT_CHECK_ARG(d->max_crops >= 1 && d->crop_h >= 2 * d->reward.radius + 1 && d->crop_w >= 2 * d->reward.radius + 1,
                 "crops must be at least the reward window");
    HT_CHECK_ARG(d->n_samples >= 1 && d->n_samples <= 64, "n_samples must be in [1, 64]");
    HT_CHECK_ARG(d->n_gray >= 0, "n_gray must be >= 0");
    if (d->n_gray > 0)
        HT_CHECK_ARG(d->gray_n >= 8 && d->gray_n <= 1024 && (d->gray_n & (d->gray_n - 1)) == 0,
                     "gray_n must be a power of two in [8, 1024]");
    HT_CHECK_ARG(d->las_mode == 0 || d->las_mode == 1, "las_mode must be 0 or 1");
    HT_CHECK_ARG(d->estimator == HT_EST_LE || d->estimator == HT_EST_COMA, "unknown estimator %d", d->estimator);
    HT_CHECK_ARG(d->ckpt_stride >= 0 && d->ckpt_stride <= 16, "ckpt_stride must be in [0, 16]");
    if (d->las_mode == 1)
        HT_CHECK_ARG(d->n_rad >= 1 && d->n_rad <= 256 && d->n_ang >= 2 && d->n_ang <= 64, "bad bin counts");
    HT_CHECK_ARG(d->reward.radius >= 1 && d->reward.radius <= 7, "reward radius must be in [1, 7]");
    ht_train *t = new ht_train();
    t->p = p;
    t->d = *d;
    t->d.reward.levels = p->levels;            // rewards and toggles of the policy's own halftones
    if (d->las_mode == 0) {
        t->d.n_rad = 1;
        t->d.n_ang = 1;
    }
    t->hidden_ch_sum = 0;
    for (int l = 1; l < p->L; ++l) t->hidden_ch_sum += p->ch[l];
    t->crop_px = (size_t)d->crop_h * d->crop_w;
    t->gray_px = (size_t)d->gray_n * d->gray_n;
    const int B = d->max_crops, G = d->n_gray, S = d->n_samples;
    const int words = ht_bits_row_words(d->crop_w, p->head);
    const size_t all_px = t->crop_px * B + t->gray_px * G;
    int cmax = 1;
    for (int l = 1; l < p->L; ++l) cmax = p->ch[l] > cmax ? p->ch[l] : cmax;
    const size_t max_px = t->crop_px > t->gray_px ? t->crop_px : t->gray_px;
    size_t wmax = 0;
    for (int l = 0; l < p->L; ++l) {
        const size_t n = (size_t)p->ch[l] * p->ch[l + 1] * 9;
        wmax = n > wmax ? n : wmax;
    }
    {
        const int batch = B * S < 32 ? B * S : 32;       // ht_toggle_launch works in batches of up to 32 images
        t->toggle_scratch_floats = (size_t)batch * ht_toggle_scratch_floats(d->crop_h, d->crop_w, d->reward.radius);
    }
    t->las_scratch_bytes = G > 0 ? ht_las_scratch_bytes(G, d->gray_n, t->d.n_rad, t->d.n_ang) : 0;
    const int gmax = (int)(d->crop_h > d->gray_n ? d->crop_h : d->gray_n);
    const int words_max = ht_bits_row_words(d->crop_w > d->gray_n ? d->crop_w : d->gray_n, p->head);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes < 16 ? 16 : bytes);
    };
    const bool tc = ht_train_tc_supported(p);
    if (!tc)
        alloc((void **)&t->acts, sizeof(float) * image_act_floats(t, t->crop_px) * B +
                                     sizeof(float) * image_act_floats(t, t->gray_px) * G);
    alloc((void **)&t->prob, sizeof(float) * all_px);
    alloc((void **)&t->dprob, sizeof(float) * all_px);
    alloc((void **)&t->tbits, sizeof(uint32_t) * (size_t)gmax * words_max);
    alloc((void **)&t->sbits, sizeof(uint32_t) * (size_t)B * S * d->crop_h * words);
    alloc((void **)&t->dR, sizeof(float) * (size_t)B * S * t->crop_px);
    alloc((void **)&t->gray_img, sizeof(float) * t->gray_px * (G > 0 ? G : 1));
    if (!tc) alloc((void **)&t->gbuf[0], sizeof(float) * cmax * max_px);
    if (!tc) alloc((void **)&t->gbuf[1], sizeof(float) * cmax * max_px);
    if (!tc) alloc((void **)&t->wflip, sizeof(float) * wmax);
    alloc((void **)&t->toggle_scratch, sizeof(float) * t->toggle_scratch_floats);
    if (G > 0) alloc(&t->las_scratch, t->las_scratch_bytes);
    alloc((void **)&t->dacc, sizeof(double) * (1 + G + (size_t)B * S * 4));
    t->tc = tc;
    if (t->tc) {
        ht_train_tc_ws &w = t->tcw;
        w.ckpt = d->ckpt_stride > 1 ? d->ckpt_stride : 1;
        size_t arena = 0;
        for (int k = 0; k < B + G; ++k) {
            w.slot_off.push_back(arena);
            arena += ht_train_tc_image_bytes(p, w.ckpt, k < B ? t->crop_px : t->gray_px);
        }
        const int wg = ht_bits_row_words(d->gray_n, p->head);
        int tiles = B * ((d->crop_w + 31) / 32) * ((d->crop_h + 7) / 8) + G * ((d->gray_n + 31) / 32) * ((d->gray_n + 7) / 8);
        size_t total = 0;
        ht_train_tc_scratch_layout(p, tiles, &w.wt_off, &total);
        w.scratch_bytes = total;
        alloc(&w.arena, arena);
        alloc((void **)&w.dz, sizeof(float) * all_px);
        alloc((void **)&w.hbits, sizeof(uint32_t) * ((size_t)B * d->crop_h * words + (size_t)G * d->gray_n * wg));
        alloc(&w.tables, ht_train_tc_table_bytes(p, B + G));
        alloc(&w.scratch, w.scratch_bytes);
        w.prob = t->prob;
    }
    if (e != cudaSuccess) {
        ht_set_error("training workspace: %s", cudaGetErrorString(e));
        ht_train_destroy(t);
        return e == cudaErrorMemoryAllocation ? HT_ERR_OOM : HT_ERR_CUDA;
    }
    (void)words;
    *out = t;
    return HT_OK;
}

ht_status ht_train_destroy(ht_train *t)
{
    if (!t) return HT_OK;
    cudaFree(t->acts);
    cudaFree(t->prob);
    cudaFree(t->dprob);
    cudaFree(t->tbits);
    cudaFree(t->sbits);
    cudaFree(t->dR);
    cudaFree(t->gray_img);
    cudaFree(t->gbuf[0]);
    cudaFree(t->gbuf[1]);
    cudaFree(t->wflip);
    cudaFree(t->toggle_scratch);
    cudaFree(t->las_scratch);
    cudaFree(t->dacc);
    cudaFree(t->tcw.arena);
    cudaFree(t->tcw.dz);
    cudaFree(t->tcw.hbits);
    cudaFree(t->tcw.tables);
    cudaFree(t->tcw.scratch);
    delete t;
    return HT_OK;
}

ht_status ht_train_step_fwd(ht_train *t, const ht_image *crops, int n, const float *gray_levels, uint64_t seed,
                            double *losses_host, void *stream)
{
    HT_RANGE("ht_train_step_fwd");
    HT_CHECK_ARG(t && (crops || n == 0) && losses_host, "null argument");
    const int G = t->d.n_gray, S = t->d.n_samples;
    HT_CHECK_ARG(n >= 0 && n <= t->d.max_crops && n + G >= 1,
                 "n must be in [0, max_crops] (0 only with gray patches)");
    HT_CHECK_ARG(G == 0 || gray_levels, "gray levels required");
    for (int i = 0; i < n; ++i) {
        HT_CHECK_ARG(crops[i].contone && crops[i].h == t->d.crop_h && crops[i].w == t->d.crop_w &&
                         crops[i].pitch >= crops[i].w,
                     "crop %d: expected %dx%d", i, t->d.crop_h, t->d.crop_w);
    }
    ht_policy *p = t->p;
    cudaStream_t s = (cudaStream_t)stream;
    const int H = t->d.crop_h, W = t->d.crop_w, words = ht_bits_row_words(W, p->head);
    const int B = t->d.max_crops;
    HT_CUDA_TRY(cudaMemsetAsync(t->dacc, 0, sizeof(double) * (1 + G), s));
    // 1. forward, keeping activations
    if (t->tc) {
        std::vector<ht_image> imgs(n + G);
        ht_train_tc_ws &w = t->tcw;
        w.img_off.assign(n + G, 0);
        w.prob_off.assign(n + G, 0);
        w.bits_off.assign(n + G, 0);
        const int words_g = ht_bits_row_words(t->d.gray_n, p->head);
        for (int i = 0; i < n + G; ++i) {
            const bool gray = i >= n;
            const int slot = gray ? B + (i - n) : i;
            if (!gray) {
                imgs[i] = crops[i];
            } else {
                const int gidx = i - n;
                float *gi = t->gray_img + t->gray_px * gidx;
                k_fill<<<nblk(t->gray_px), 256, 0, s>>>(gi, t->gray_px, gray_levels[gidx]);
                HT_LAUNCH_CHECK();
                imgs[i].contone = gi;
                imgs[i].h = imgs[i].w = imgs[i].pitch = t->d.gray_n;
            }
            w.img_off[i] = w.slot_off[slot];
            w.prob_off[i] = img_px_offset(t, slot);
            w.bits_off[i] = slot < B ? (size_t)slot * H * words
                                     : (size_t)B * H * words + (size_t)(slot - B) * t->d.gray_n * words_g;
        }
        ht_status st = ht_train_tc_forward(p, w, imgs.data(), n + G, seed, s);
        if (st != HT_OK) return st;
    }
    for (int i = 0; i < n + G && !t->tc; ++i) {
        const bool gray = i >= n;
        const int slot = gray ? B + (i - n) : i;
        ht_image img;
        if (!gray) {
            img = crops[i];
        } else {
            const int gidx = i - n;
            float *gi = t->gray_img + t->gray_px * gidx;
            k_fill<<<nblk(t->gray_px), 256, 0, s>>>(gi, t->gray_px, gray_levels[gidx]);
            HT_LAUNCH_CHECK();
            img.contone = gi;
            img.h = img.w = img.pitch = t->d.gray_n;
        }
        float *acts[HT_MAX_LAYERS];
        for (int l = 0; l + 1 < p->L; ++l) acts[l] = act_ptr(t, slot, l);
        ht_status st = ht_fwd_fp32_save(p, img, (uint32_t)i, seed, acts, t->prob + img_px_offset(t, slot), t->tbits, s);
        if (st != HT_OK) return st;
    }
    // 2.-4. samples, rewards, toggle deltas, L_MARL and its gradient
    double *rewards = t->dacc + 1 + G;
    if (n > 0) {
        // all crops x samples in one launch per kernel (reward / toggle deltas in batches)
        k_sample_bits<<<dim3((W + 31) / 32, H, n * S), 32, 0, s>>>(t->prob, t->crop_px, H, W, words, seed, S,
                                                                   p->levels, t->sbits);
        HT_LAUNCH_CHECK();
        std::vector<ht_image> cimg((size_t)n * S);
        std::vector<const uint32_t *> bp((size_t)n * S);
        std::vector<float *> dp((size_t)n * S);
        std::vector<const float *> vp((size_t)n * S);
        for (int i = 0; i < n; ++i)
            for (int sm = 0; sm < S; ++sm) {
                const size_t k = (size_t)i * S + sm;
                cimg[k] = crops[i];
                bp[k] = t->sbits + k * H * words;
                dp[k] = t->dR + k * t->crop_px;
                vp[k] = t->prob + img_px_offset(t, i);
            }
        ht_status st = ht_reward_launch(cimg.data(), bp.data(), n * S, t->d.reward, rewards, s);
        if (st != HT_OK) return st;
        st = ht_toggle_launch(cimg.data(), bp.data(), vp.data(), n * S, t->d.reward, dp.data(), t->toggle_scratch,
                              t->toggle_scratch_floats, s);
        if (st != HT_OK) return st;
        k_marl<<<dim3(nblk(t->crop_px), n), 256, 0, s>>>(t->prob, t->dR, t->sbits, rewards, S, H, W, words,
                                                         1.0 / ((double)n * S), t->d.estimator, p->levels, t->dprob,
                                                         t->dacc);
        HT_LAUNCH_CHECK();
    }
    // 5. anisotropy loss on the gray patches' probability maps
    if (G > 0) {
        const float *q = t->prob + img_px_offset(t, B);
        float *gq = t->dprob + img_px_offset(t, B);
        ht_status st = ht_las_launch(q, G, t->d.gray_n, t->d.las_mode, t->d.n_rad, t->d.n_ang, t->dacc + 1, gq,
                                     t->las_scratch, t->las_scratch_bytes, s);
        if (st != HT_OK) return st;
        k_scale_into<<<nblk(t->gray_px * G), 256, 0, s>>>(gq, t->d.w_a / (float)G, t->gray_px * G, gq);
        HT_LAUNCH_CHECK();
    }
    // 6. losses to the host
    std::vector<double> h(1 + G + (size_t)n * S * 4);
    HT_CUDA_TRY(cudaMemcpyAsync(h.data(), t->dacc, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    HT_CUDA_TRY(cudaStreamSynchronize(s));
    double las = 0.0, rmean = 0.0;
    for (int g = 0; g < G; ++g) las += h[1 + g];
    if (G > 0) las /= G;
    for (int k = 0; k < n * S; ++k) rmean += h[1 + G + 4 * (size_t)k + 3];
    if (n > 0) rmean /= (double)n * S;
    losses_host[0] = h[0] + (double)t->d.w_a * las;
    losses_host[1] = h[0];
    losses_host[2] = las;
    losses_host[3] = rmean;
    t->n_last = n;
    t->fwd_done = true;
    t->seed_last = seed;
    t->crops_last.assign(crops, crops + n);
    return HT_OK;
}

ht_status ht_train_step_bwd(ht_train *t, float *grad_w, float *grad_b, void *stream)
{
    HT_RANGE("ht_train_step_bwd");
    HT_CHECK_ARG(t && grad_w && grad_b, "null argument");
    HT_CHECK_ARG(t->fwd_done, "no forward to differentiate");
    ht_policy *p = t->p;
    cudaStream_t s = (cudaStream_t)stream;
    HT_CUDA_TRY(cudaMemsetAsync(grad_w, 0, sizeof(float) * p->n_w, s));
    HT_CUDA_TRY(cudaMemsetAsync(grad_b, 0, sizeof(float) * p->n_b, s));
    const int n = t->n_last, G = t->d.n_gray, B = t->d.max_crops;
    if (t->tc) {
        const size_t all_px = t->crop_px * B + t->gray_px * G;
        k_dlogit<<<nblk(all_px), 256, 0, s>>>(t->dprob, t->prob, all_px, t->tcw.dz);
        HT_LAUNCH_CHECK();
        return ht_train_tc_backward(p, t->tcw, n + G, t->seed_last, grad_w, grad_b, s);
    }
    for (int i = 0; i < n + G; ++i) {
        const bool gray = i >= n;
        const int slot = gray ? B + (i - n) : i;
        ht_image img;
        if (!gray) {
            img = t->crops_last[i];
        } else {
            img.contone = t->gray_img + t->gray_px * (i - n);
            img.h = img.w = img.pitch = t->d.gray_n;
        }
        const int H = img.h, W = img.w;
        const size_t npx = (size_t)H * W;
        const size_t off = img_px_offset(t, slot);
        int cur = 0;
        k_dlogit<<<nblk(npx), 256, 0, s>>>(t->dprob + off, t->prob + off, npx, t->gbuf[cur]);
        HT_LAUNCH_CHECK();
        for (int l = p->L - 1; l >= 0; --l) {
            const int Cin = p->ch[l], Cout = p->ch[l + 1];
            const float *in = l > 0 ? act_ptr(t, slot, l - 1) : nullptr;
            const int nseg = (W + 31) / 32;
            const dim3 grid((Cout + WG_O - 1) / WG_O, (Cin + WG_C - 1) / WG_C,
                            (unsigned)(((long)H * nseg + WG_SEGS - 1) / WG_SEGS));
            ht_prof_start(HTK_TRAIN, s);
            k_wgrad<<<grid, 256, 0, s>>>(t->gbuf[cur], in, l == 0 ? img.contone : nullptr, img.pitch, t->seed_last,
                                         (uint32_t)i, Cout, Cin, H, W, grad_w + p->w_off[l], grad_b + p->b_off[l]);
            ht_prof_stop(s);
            HT_LAUNCH_CHECK();
            if (l == 0) break;
            k_flip<<<nblk((size_t)Cout * Cin * 9), 256, 0, s>>>(p->d_w + p->w_off[l], Cout, Cin, t->wflip);
            HT_LAUNCH_CHECK();
            ht_status st = ht_dgrad_fp32(t->gbuf[cur], t->wflip, Cout, Cin, H, W, in, t->gbuf[cur ^ 1], s);
            if (st != HT_OK) return st;
            cur ^= 1;
        }
    }
    return HT_OK;
}

}  // extern "C"

void ht_preload_train()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_fill);
    cudaFuncGetAttributes(&fa, k_sample_bits);
    cudaFuncGetAttributes(&fa, k_marl);
    cudaFuncGetAttributes(&fa, k_scale_into);
    cudaFuncGetAttributes(&fa, k_dlogit);
    cudaFuncGetAttributes(&fa, k_flip);
    cudaFuncGetAttributes(&fa, k_wgrad);
}
