// head.cuh -- action head shared by the FP32 and tensor-core forms.
//
// For one pixel per thread, with a warp covering the 32 consecutive pixels
// x0 .. x0+31 of row y (x0 a multiple of 32): turns the K logits into action
// probabilities (pixel-wise sigmoid, Sec. III "Agents"; softmax over the 4
// levels of the multitone head, Sec. VI-E), draws the action (Algorithm 1:
// Thresholding(., 0.5), i.e. h = [p > 0.5] -- argmax for the softmax head --
// or Bernoulli h = [u < p] with u from Philox stream 1; softmax: smallest k
// with u < q_0 + ... + q_k; multitoning prototype of Sec. VI-E: the level pair
// k, k + 1 around the sigmoid output v, k = floor(v (L - 1)) capped at L - 2, the
// upper one when u < v (L - 1) - k, or when that fraction exceeds 1/2 in threshold
// mode) and packs it LSB-first (1 bit per pixel, or 2 bits for the 4-level and
// multitone heads) with warp-wide ballots / OR-reductions.
#pragma once
#include "ht_internal.cuh"

__device__ __forceinline__ void ht_pack2(int lev, bool inside, int lane, int x0, int y, int H, uint32_t *bits, int words)
{
    const uint32_t v = inside ? ((uint32_t)lev << (2 * (lane & 15))) : 0u;
    const uint32_t w0 = __reduce_or_sync(0xffffffffu, lane < 16 ? v : 0u);
    const uint32_t w1 = __reduce_or_sync(0xffffffffu, lane >= 16 ? v : 0u);
    if (y < H) {
        const int wi = x0 >> 4;
        if (lane == 0 && wi < words) bits[(size_t)y * words + wi] = w0;
        if (lane == 16 && wi + 1 < words) bits[(size_t)y * words + wi + 1] = w1;
    }
}

__device__ __forceinline__ void ht_head_emit(const float *z, int K, int head, int mode, uint64_t seed,
                                             uint32_t image, int x0, int y, int H, int W, uint32_t *bits,
                                             int words, float *prob, int levels = 2)
{
    const int lane = threadIdx.x & 31;
    const int x = x0 + lane;
    const bool inside = (x < W) && (y < H);
    const uint64_t g = (uint64_t)y * (uint64_t)W + (uint64_t)x;
    const float u = (mode == HT_MODE_BERNOULLI && inside) ? ht_uniform24(seed, image, 1u, g) : 0.5f;
    if (head == HT_HEAD_SIGMOID) {
        const float p = 1.f / (1.f + expf(-z[0]));
        const bool hbit = inside && (mode == HT_MODE_BERNOULLI ? (u < p) : (p > 0.5f));
        const uint32_t word = __ballot_sync(0xffffffffu, hbit);
        if (lane == 0 && y < H) bits[(size_t)y * words + (x0 >> 5)] = word;
        if (prob && inside) prob[(size_t)y * W + x] = p;
        return;
    }
    if (head == HT_HEAD_MULTITONE) {
        const float v = 1.f / (1.f + expf(-z[0]));
        const float t = v * (float)(levels - 1);
        const int k = min((int)floorf(t), levels - 2);
        const float frac = t - (float)k;
        const int lev = k + ((mode == HT_MODE_BERNOULLI ? (u < frac) : (frac > 0.5f)) ? 1 : 0);
        ht_pack2(lev, inside, lane, x0, y, H, bits, words);
        if (prob && inside) prob[(size_t)y * W + x] = v;
        return;
    }
    float q[4];
    float m = -INFINITY;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < K) m = fmaxf(m, z[k]);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        q[k] = (k < K) ? expf(z[k] - m) : 0.f;
        s += q[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = q[k] / s;
    int lev = 0;
    if (mode == HT_MODE_BERNOULLI) {
        float cdf = 0.f;
        lev = K - 1;
        for (int k = 0; k < K; ++k) {
            cdf += q[k];
            if (u < cdf) {
                lev = k;
                break;
            }
        }
    } else {
        for (int k = 1; k < K; ++k)
            if (q[k] > q[lev]) lev = k;
    }
    ht_pack2(lev, inside, lane, x0, y, H, bits, words);
    if (prob && inside)
        for (int k = 0; k < K; ++k) prob[(size_t)k * H * W + (size_t)y * W + x] = q[k];
}
