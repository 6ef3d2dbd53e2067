// conv_fp32.cu -- plain FP32 form of the policy forward (CUDA cores).
//
// One launch per 3x3 layer (zero padding 1, stride 1; Sec. III "Agents",
// Sec. VI-A), activations planar [C][H][W] float32 in HBM.  The first layer
// builds its two input channels on the fly: the contone c and the noise
// channel z ~ U[0,1) from Philox stream 0 (Sec. III "State").  The last
// layer's epilogue applies the head (sigmoid, or softmax over K logits), draws
// the action (threshold 0.5 or Bernoulli with Philox stream 1; Algorithm 1,
// Eq. independent) and bit-packs it with a warp ballot.
//
// This is the unfused reference form that the tensor-core path is timed
// against; it is deliberately straightforward (SMEM-tiled direct convolution).
#include <string.h>

#include "head.cuh"

namespace {

constexpr int TX = 32, TY = 8;      // output tile (one warp per tile row)
constexpr int CI_CHUNK = 8;         // input channels staged per step
constexpr int CO_T = 32;            // output channels per block

struct HeadArgs {
    int head;          // -1: hidden layer (ReLU, store), else HT_HEAD_*
    int K;
    int levels;        // multitone head: ink levels
    int mode;
    uint64_t seed;
    uint32_t image;
    uint32_t *bits;
    int words;         // words per bits row
    float *prob;       // nullable [K][H][W]
};

__global__ void __launch_bounds__(TX *TY)
k_conv3x3_fp32(const float *__restrict__ in, const float *__restrict__ contone, int cpitch,
               const float *__restrict__ w, const float *__restrict__ b, int Cin, int Cout, int H, int W,
               float *__restrict__ out, HeadArgs ha, const float *__restrict__ mask)
{
    __shared__ float s_in[CI_CHUNK][TY + 2][TX + 2];
    __shared__ float s_w[CI_CHUNK][9][CO_T];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, co0 = blockIdx.z * CO_T;
    const int x = x0 + tx, y = y0 + ty;
    const bool first = (contone != nullptr);
    const size_t plane = (size_t)H * W;

    float acc[CO_T];
#pragma unroll
    for (int j = 0; j < CO_T; ++j) acc[j] = 0.f;

    for (int c0 = 0; c0 < Cin; c0 += CI_CHUNK) {
        for (int i = tid; i < CI_CHUNK * (TY + 2) * (TX + 2); i += TX * TY) {
            const int ci = i / ((TY + 2) * (TX + 2));
            const int r = i % ((TY + 2) * (TX + 2));
            const int yy = r / (TX + 2), xx = r % (TX + 2);
            const int gy = y0 + yy - 1, gx = x0 + xx - 1;
            float v = 0.f;
            if (c0 + ci < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W) {
                if (first) {
                    v = (c0 + ci == 0) ? contone[(size_t)gy * cpitch + gx]
                                       : ht_uniform24(ha.seed, ha.image, 0u, (uint64_t)gy * W + gx);
                } else {
                    v = in[(size_t)(c0 + ci) * plane + (size_t)gy * W + gx];
                }
            }
            s_in[ci][yy][xx] = v;
        }
        for (int i = tid; i < CI_CHUNK * 9 * CO_T; i += TX * TY) {
            const int ci = i / (9 * CO_T);
            const int r = i % (9 * CO_T);
            const int tap = r / CO_T, co = r % CO_T;
            float v = 0.f;
            if (c0 + ci < Cin && co0 + co < Cout) v = w[((size_t)(co0 + co) * Cin + (c0 + ci)) * 9 + tap];
            s_w[ci][tap][co] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int ci = 0; ci < CI_CHUNK; ++ci) {
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const float v = s_in[ci][ty + tap / 3][tx + tap % 3];
#pragma unroll
                for (int j = 0; j < CO_T; ++j) acc[j] = fmaf(v, s_w[ci][tap][j], acc[j]);
            }
        }
        __syncthreads();
    }

    const bool inside = (x < W) && (y < H);
    if (ha.head < 0) {
        if (inside) {
            if (mask) {
                // data-gradient pass: no bias; gradient masked by the ReLU of the layer's input
#pragma unroll
                for (int j = 0; j < CO_T; ++j)
                    if (co0 + j < Cout) {
                        const size_t k = (size_t)(co0 + j) * plane + (size_t)y * W + x;
                        out[k] = mask[k] > 0.f ? acc[j] : 0.f;
                    }
            } else {
#pragma unroll
                for (int j = 0; j < CO_T; ++j)
                    if (co0 + j < Cout)
                        out[(size_t)(co0 + j) * plane + (size_t)y * W + x] = fmaxf(acc[j] + b[co0 + j], 0.f);
            }
        }
        return;
    }

    // ---- head epilogue (grid.z == 1, Cout = K <= 4) ----
    float z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = (k < ha.K) ? acc[k] + b[k] : 0.f;
    ht_head_emit(z, ha.K, ha.head, ha.mode, ha.seed, ha.image, x0, y, H, W, ha.bits, ha.words, ha.prob, ha.levels);
}

}  // namespace

size_t ht_fp32_ws_bytes(const ht_policy *p, int h, int w)
{
    int cmax = 0;
    for (int l = 1; l < p->L; ++l) cmax = p->ch[l] > cmax ? p->ch[l] : cmax;
    return 2 * (size_t)cmax * h * w * sizeof(float);
}

ht_status ht_run_fp32(ht_policy *p, const ht_image &img, uint32_t image_index, int mode, uint64_t seed,
                      uint32_t *bits, float *prob, float *act_a, float *act_b, cudaStream_t s)
{
    const int H = img.h, W = img.w;
    const dim3 block(TX, TY);
    float *bufs[2] = {act_a, act_b};
    const float *in = nullptr;
    for (int l = 0; l < p->L; ++l) {
        const int Cin = p->ch[l], Cout = p->ch[l + 1];
        const bool last = (l == p->L - 1);
        HeadArgs ha;
        ha.head = last ? p->head : -1;
        ha.K = p->K;
        ha.levels = p->levels;
        ha.mode = mode;
        ha.seed = seed;
        ha.image = image_index;
        ha.bits = bits;
        ha.words = ht_bits_row_words(W, p->head);
        ha.prob = prob;
        const dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY, last ? 1 : (Cout + CO_T - 1) / CO_T);
        float *out = last ? nullptr : bufs[l & 1];
        ht_prof_start(last ? HTK_HEAD_FP32 : HTK_CONV_FP32, s);
        k_conv3x3_fp32<<<grid, block, 0, s>>>(in, l == 0 ? img.contone : nullptr, img.pitch,
                                              p->d_w + p->w_off[l], p->d_b + p->b_off[l], Cin, Cout, H, W,
                                              out, ha, nullptr);
        ht_prof_stop(s);
        HT_LAUNCH_CHECK();
        in = out;
    }
    return HT_OK;
}

// Forward of the FP32 form that keeps every hidden activation (training):
// acts[l] receives layer l's output [ch[l+1]][H][W] for l < L-1; the head
// writes the probability map `prob` and threshold actions into `bits`.
ht_status ht_fwd_fp32_save(ht_policy *p, const ht_image &img, uint32_t image_index, uint64_t seed,
                           float *const *acts, float *prob, uint32_t *bits, cudaStream_t s)
{
    const int H = img.h, W = img.w;
    const dim3 block(TX, TY);
    const float *in = nullptr;
    for (int l = 0; l < p->L; ++l) {
        const int Cin = p->ch[l], Cout = p->ch[l + 1];
        const bool last = (l == p->L - 1);
        HeadArgs ha;
        ha.head = last ? p->head : -1;
        ha.K = p->K;
        ha.levels = p->levels;
        ha.mode = HT_MODE_THRESHOLD;
        ha.seed = seed;
        ha.image = image_index;
        ha.bits = bits;
        ha.words = ht_bits_row_words(W, p->head);
        ha.prob = prob;
        const dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY, last ? 1 : (Cout + CO_T - 1) / CO_T);
        float *out = last ? nullptr : acts[l];
        ht_prof_start(HTK_TRAIN, s);
        k_conv3x3_fp32<<<grid, block, 0, s>>>(in, l == 0 ? img.contone : nullptr, img.pitch,
                                              p->d_w + p->w_off[l], p->d_b + p->b_off[l], Cin, Cout, H, W,
                                              out, ha, nullptr);
        ht_prof_stop(s);
        HT_LAUNCH_CHECK();
        in = out;
    }
    return HT_OK;
}

// Data gradient of one layer: g_in = conv(g_out, W flipped and transposed),
// masked by (act_in > 0).  wt: [Cin][Cout][3][3] flipped weights.
ht_status ht_dgrad_fp32(const float *g_out, const float *wt, int Cout, int Cin, int H, int W, const float *act_in,
                        float *g_in, cudaStream_t s)
{
    HeadArgs ha;
    memset(&ha, 0, sizeof(ha));
    ha.head = -1;
    ha.levels = 2;
    const dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY, (Cin + CO_T - 1) / CO_T);
    ht_prof_start(HTK_TRAIN, s);
    k_conv3x3_fp32<<<grid, dim3(TX, TY), 0, s>>>(g_out, nullptr, 0, wt, nullptr, Cout, Cin, H, W, g_in, ha, act_in);
    ht_prof_stop(s);
    HT_LAUNCH_CHECK();
    return HT_OK;
}

void ht_preload_conv_fp32()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_conv3x3_fp32);
}
