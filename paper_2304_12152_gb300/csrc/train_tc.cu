// train_tc.cu -- BF16 tensor-core form of one training iteration (Algorithm 1,
// TRAIN step) for the 2 -> 64 x (L-1) -> 1 policy.
//
// Forward: the inference pipeline of conv_tc.cu run layer by layer over all
// crops and gray patches of the step, keeping every hidden activation (bf16,
// chunk-planar) and its ReLU mask (64 bits per pixel), and the sigmoid
// probabilities (FP32) of the head.
//
// Backward (chain rule through Eq. marl / Eq. as, ReLU and the convolutions):
//   dz = dL/dp * p (1 - p)                                       (train.cu)
//   head 64 -> 1 (CUDA cores, k_head_bwd): g_{L-2} = mask * sum_tap w dz(shifted),
//        dW_head = sum_px dz * a_{L-2}(shifted), db_head = sum dz
//   every 64 -> 64 layer l:
//        dW_l = sum_px g_l (x) a_{l-1}(shifted)    tcgen05, k_wgrad_tc
//        db_l = sum_px g_l                           (same kernel)
//        g_{l-1} = mask_{l-1} * conv(g_l, W_l flipped and transposed)
//                                                    conv_tc.cu pipeline, dgrad epilogue
//   layer 1 (CUDA cores, k_first_wgrad): dW_1 = sum_px g_1 (x) (c, z)(shifted), db_1.
// Rounding points (the oracle's quant-1 backward follows them): inner-layer
// weights bf16 in both passes, activations and hidden gradients stored bf16,
// FP32 accumulation, weight-gradient partial sums reduced with compensated FP32
// sums in a fixed order (deterministic).
#include <string.h>

#include <vector>

#include "tc_common.cuh"

namespace {

// ---------------------------------------------------------------------------
// Weight gradient of a 64 -> 64 layer on tcgen05.
//
// GEMM over pixels: D[m][n] += sum_k A[m][k] B[n][k], k = 16 pixels per MMA.
//   B[n][k]  = g[n](y, x0 + k): one staged gradient row, chunk-planar, i.e. the
//              MN-major canonical layout (8 channels contiguous, pixels at a
//              16-byte stride).
//   A[m][k]  = a[c](y + dy - 1, x0 + k + dx - 1), m = (row half, c): the two
//              halves of M are two consecutive staged activation rows, so one
//              MMA covers taps (dy, dx) and (dy + 1, dx).  Staged rows sit in a
//              ring whose slot 0 is mirrored after the last slot, so two
//              consecutive rows are always contiguous; the pixel shift dx is a
//              16-byte shift of the descriptor start.
// Six accumulator tiles of 128 lanes x 64 columns (dx x {dy 0|1, dy 2|unused})
// stay in TMEM for the whole persistent CTA; the epilogue warps zero them at
// the start, sum the staged gradient rows per channel while the MMAs run (bias
// gradient), and write the CTA's partial sums at the end.
// ---------------------------------------------------------------------------
// Compensated (Kahan) FP32 accumulation: error ~1 ulp of the sum whatever the
// number of terms, in a fixed order (deterministic), without the GPU's slow FP64 pipe.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

constexpr int WG_NSA = 8;                       // activation-row ring (+1 mirror slot)
constexpr int WG_NSG = 4;                       // gradient-row ring
constexpr int WG_ASLOT = 8 * ROW_PX * 16;       // [chunk][130 px][16 B]
constexpr int WG_GSLOT = 8 * TILE_M * 16;       // [chunk][128 px][16 B]
constexpr int WG_NTHREADS = 192;                // producer, MMA issuer, 4 epilogue warps
constexpr int WG_TILES = 6;
constexpr int WG_SMEM = (WG_NSA + 1) * WG_ASLOT + WG_NSG * WG_GSLOT + 1024 /*align*/ + 1024 /*barriers*/;

struct WgParams {
    const ImgDesc *imgs;      // act[0] = layer input a (chunk-planar bf16), act[1] = gradient g
    int n_imgs, n_units;
    float *partials;          // [grid][6 tiles][64 n][128 lanes]
    float *colsum;            // [grid][64]
    int *err;
};

// instruction descriptor: F32 accumulate, bf16 A/B, both MN-major, N = 64, M = 128
constexpr uint32_t kWgIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((64u >> 3) << 17) |
                              ((128u >> 4) << 24);

__global__ void __launch_bounds__(WG_NTHREADS, 1) k_wgrad_tc(const WgParams P)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *s_a = smem;
    uint8_t *s_g = s_a + (WG_NSA + 1) * WG_ASLOT;
    uint64_t *bars = (uint64_t *)(s_g + WG_NSG * WG_GSLOT);
    uint64_t *a_full = bars, *a_empty = bars + WG_NSA, *g_full = bars + 2 * WG_NSA,
             *g_empty = bars + 2 * WG_NSA + WG_NSG, *tzero = bars + 2 * WG_NSA + 2 * WG_NSG, *done = tzero + 1;
    int2 *a_meta = (int2 *)(done + 1);                          // (r, nrows) of the activation row in each slot
    int2 *g_meta = a_meta + WG_NSA;                             // (j, nrows) of the gradient row in each slot
    uint32_t *s_tmem = (uint32_t *)(g_meta + WG_NSG);
    volatile int *s_abort = (volatile int *)(s_tmem + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < WG_NSA; ++i) {
            mbar_init(smem_u32(&a_full[i]), 1);
            mbar_init(smem_u32(&a_empty[i]), 1);
        }
        for (int i = 0; i < WG_NSG; ++i) {
            mbar_init(smem_u32(&g_full[i]), 1);
            mbar_init(smem_u32(&g_empty[i]), 1 + 4);     // MMA commit + 4 epilogue warps (bias sums)
        }
        mbar_init(smem_u32(tzero), 4);
        mbar_init(smem_u32(done), 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(s_tmem), TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *s_tmem;

    if (warp == 0) {
        // ------------------------- producer -------------------------
        int a_last[WG_NSA], g_last[WG_NSG];
        for (int i = 0; i < WG_NSA; ++i) a_last[i] = -1;
        for (int i = 0; i < WG_NSG; ++i) g_last[i] = -1;
        uint32_t la = 0, lg = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < P.n_units && ok; u += gridDim.x) {
            const UnitInfo ui = unit_info(P.imgs, P.n_imgs, 0, u);
            const int x0 = ui.x0;
            const int lo = max(x0 - 1, 0), hi = min(x0 - 1 + ROW_PX, ui.W);
            for (int r = 0; r < ui.nrows + 2 && ok; ++r) {
                // activation row y0 - 1 + r into ring slot la % NSA (slot 0 also into the mirror)
                {
                    const int slot = (int)(la % WG_NSA);
                    int got = 0;
                    if (lane == 0)
                        got = mbar_wait(smem_u32(&a_empty[slot]), ((la / WG_NSA) & 1u) ^ 1u, s_abort, P.err) ? 1 : 0;
                    if (!__shfl_sync(0xffffffffu, got, 0)) {
                        ok = false;
                        break;
                    }
                    const int ncopy = slot == 0 ? 2 : 1;
                    const int yy = ui.y0 - 1 + r;
                    const bool row_in = (yy >= 0 && yy < ui.H);
                    bool zeroed = false;
                    for (int cp = 0; cp < ncopy; ++cp) {
                        uint8_t *dst = s_a + (cp ? WG_NSA : slot) * WG_ASLOT;
                        if (!row_in) {
                            for (int k = lane; k < 8 * ROW_PX; k += 32)
                                *reinterpret_cast<uint4 *>(dst + (size_t)k * 16) = make_uint4(0, 0, 0, 0);
                            zeroed = true;
                        } else if (lo > x0 - 1 || hi < x0 - 1 + ROW_PX) {
                            const int nl = lo - (x0 - 1), nr = (x0 - 1 + ROW_PX) - hi;
                            for (int k = lane; k < 8 * (nl + nr); k += 32) {
                                const int c = k / (nl + nr), j = k % (nl + nr);
                                const int px = j < nl ? j : (hi - (x0 - 1)) + (j - nl);
                                *reinterpret_cast<uint4 *>(dst + ((size_t)c * ROW_PX + px) * 16) = make_uint4(0, 0, 0, 0);
                            }
                            zeroed = true;
                        }
                    }
                    if (zeroed) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    const uint32_t run = (uint32_t)(hi - lo) * 16u;
                    if (lane == 0) {
                        a_meta[slot] = make_int2(r, ui.nrows);
                        if (row_in && hi > lo) mbar_arrive_expect_tx(smem_u32(&a_full[slot]), run * 8u * (uint32_t)ncopy);
                        else mbar_arrive(smem_u32(&a_full[slot]));
                    }
                    __syncwarp();
                    if (row_in && hi > lo && lane < 8 * ncopy) {     // one bulk copy per (copy, chunk)
                        const int cp = lane >> 3, c = lane & 7;
                        uint8_t *dst = s_a + (cp ? WG_NSA : slot) * WG_ASLOT;
                        bulk_g2s(smem_u32(dst + ((size_t)c * ROW_PX + (lo - (x0 - 1))) * 16),
                                 ui.in + (((size_t)c * ui.H + yy) * ui.W + lo) * 16, run, smem_u32(&a_full[slot]));
                    }
                    a_last[slot] = (int)la;
                    ++la;
                }
                if (r < 2) continue;
                // gradient row y0 + r - 2 into ring slot lg % NSG
                {
                    const int slot = (int)(lg % WG_NSG);
                    int got = 0;
                    if (lane == 0)
                        got = mbar_wait(smem_u32(&g_empty[slot]), ((lg / WG_NSG) & 1u) ^ 1u, s_abort, P.err) ? 1 : 0;
                    if (!__shfl_sync(0xffffffffu, got, 0)) {
                        ok = false;
                        break;
                    }
                    uint8_t *dst = s_g + slot * WG_GSLOT;
                    const int yy = ui.y0 + r - 2;
                    const int nin = min(TILE_M, ui.W - x0);
                    if (nin < TILE_M) {
                        for (int k = lane; k < 8 * (TILE_M - nin); k += 32) {
                            const int c = k / (TILE_M - nin), px = nin + k % (TILE_M - nin);
                            *reinterpret_cast<uint4 *>(dst + ((size_t)c * TILE_M + px) * 16) = make_uint4(0, 0, 0, 0);
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    }
                    __syncwarp();
                    const uint32_t run = (uint32_t)nin * 16u;
                    if (lane == 0) {
                        g_meta[slot] = make_int2(r - 2, ui.nrows);
                        mbar_arrive_expect_tx(smem_u32(&g_full[slot]), run * 8u);
                    }
                    __syncwarp();
                    if (lane < 8)                                    // one bulk copy per chunk
                        bulk_g2s(smem_u32(dst + (size_t)lane * TILE_M * 16),
                                 ui.out + (((size_t)lane * ui.H + yy) * ui.W + x0) * 16, run, smem_u32(&g_full[slot]));
                    g_last[slot] = (int)lg;
                    ++lg;
                }
            }
        }
        if (ok) {
            // end markers (k = -1) for the MMA warp (activation ring) and the bias-sum warps
            // (gradient ring); each is its slot's newest phase, which the drain below waits for
            const int sa = (int)(la % WG_NSA), sg = (int)(lg % WG_NSG);
            int got = 0;
            if (lane == 0)
                got = (mbar_wait(smem_u32(&a_empty[sa]), ((la / WG_NSA) & 1u) ^ 1u, s_abort, P.err) &&
                       mbar_wait(smem_u32(&g_empty[sg]), ((lg / WG_NSG) & 1u) ^ 1u, s_abort, P.err)) ? 1 : 0;
            if (__shfl_sync(0xffffffffu, got, 0)) {
                if (lane == 0) {
                    a_meta[sa] = make_int2(-1, 0);
                    mbar_arrive(smem_u32(&a_full[sa]));
                    g_meta[sg] = make_int2(-1, 0);
                    mbar_arrive(smem_u32(&g_full[sg]));
                }
                a_last[sa] = (int)la;
                g_last[sg] = (int)lg;
            }
        }
        if (lane == 0) {
            for (int s2 = 0; s2 < WG_NSA; ++s2)
                if (a_last[s2] >= 0)
                    mbar_wait(smem_u32(&a_full[s2]), ((uint32_t)a_last[s2] / WG_NSA) & 1u, s_abort, P.err, true);
            for (int s2 = 0; s2 < WG_NSG; ++s2)
                if (g_last[s2] >= 0)
                    mbar_wait(smem_u32(&g_full[s2]), ((uint32_t)g_last[s2] / WG_NSG) & 1u, s_abort, P.err, true);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------- MMA issuer -------------------------
        // The whole warp runs the schedule (warp-uniform state) and one elected lane
        // issues the MMAs and commits.  Each unit's row count comes from the producer's
        // record in the activation ring (an end marker closes the sequence), so no
        // image-table lookups sit in the issuing loop.
        {
            const uint32_t el = elect_one();
            // MN-major, no swizzle: LBO = stride between 8-pixel groups (K), SBO = stride
            // between 8-channel groups (M or N)
            const uint64_t a_base = sdesc(smem_u32(s_a), 128, ROW_PX * 16);
            const uint64_t g_base = sdesc(smem_u32(s_g), 128, TILE_M * 16);
            bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(tzero), 0, s_abort, P.err));
            if (ok) tc_fence_after();
            uint32_t qa = 0, qg = 0;
            while (ok) {
                const uint32_t base = qa;
                ok = mbar_wait_poll_warp(smem_u32(&a_full[base % WG_NSA]), (base / WG_NSA) & 1u, s_abort, P.err);
                if (!ok) break;
                const volatile int *mv = (const volatile int *)&a_meta[base % WG_NSA];
                const int k0 = __shfl_sync(0xffffffffu, mv[0], 0), nrows = __shfl_sync(0xffffffffu, mv[1], 0);
                if (k0 < 0) break;
                ok = mbar_wait_poll_warp(smem_u32(&a_full[(base + 1) % WG_NSA]), ((base + 1) / WG_NSA) & 1u, s_abort, P.err);
                for (int j = 0; j < nrows && ok; ++j, ++qg) {
                    const uint32_t qn = base + (uint32_t)j + 2u;
                    ok = mbar_wait_poll_warp(smem_u32(&a_full[qn % WG_NSA]), (qn / WG_NSA) & 1u, s_abort, P.err) &&
                         mbar_wait_poll_warp(smem_u32(&g_full[qg % WG_NSG]), (qg / WG_NSG) & 1u, s_abort, P.err);
                    if (!ok) break;
                    tc_fence_after();
                    const uint64_t b_q = g_base + (uint64_t)(((qg % WG_NSG) * (uint32_t)WG_GSLOT) >> 4);
#pragma unroll
                    for (int pair = 0; pair < 2; ++pair) {
                        const uint32_t s = (base + (uint32_t)j + 2u * pair) % WG_NSA;
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
                            const uint64_t a_q = a_base + (uint64_t)((s * (uint32_t)WG_ASLOT + dx * 16u) >> 4);
                            const uint32_t d = tmem_base + (uint32_t)(dx * 2 + pair) * 64u;
#pragma unroll
                            for (int ks = 0; ks < 8; ++ks)
                                mma_ss_el<false>(el, d, a_q + (uint64_t)((ks * 256) >> 4), b_q + (uint64_t)((ks * 256) >> 4),
                                                 kWgIdesc);
                        }
                    }
                    mma_commit_el(el, smem_u32(&g_empty[qg % WG_NSG]));
                    mma_commit_el(el, smem_u32(&a_empty[(base + (uint32_t)j) % WG_NSA]));
                }
                if (!ok) break;
                mma_commit_el(el, smem_u32(&a_empty[(base + (uint32_t)nrows) % WG_NSA]));
                mma_commit_el(el, smem_u32(&a_empty[(base + (uint32_t)nrows + 1u) % WG_NSA]));
                qa = base + (uint32_t)nrows + 2u;
            }
            mma_commit_el(el, smem_u32(done));     // all issued MMAs, aborted or not
        }
    } else {
        // ------------------------- epilogue -------------------------
        const int quarter = warp & 3;
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        for (int t = 0; t < WG_TILES; ++t)
            for (int c = 0; c < 64; c += 16) tmem_zero16(lane_base + t * 64 + c);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(tzero));
        // bias gradient: per-channel sums of the staged gradient rows
        const int e = (warp - 2) * 32 + lane;             // 0..127
        const int chunk = e >> 4, pg = e & 15;            // 8 pixels pg*8 .. +7 of one chunk
        float cs[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) cs[i] = 0.f;
        for (uint32_t qg = 0;; ++qg) {
            {
                int got = 0, k = 0;
                if (lane == 0) {
                    got = mbar_wait(smem_u32(&g_full[qg % WG_NSG]), (qg / WG_NSG) & 1u, s_abort, P.err) ? 1 : 0;
                    if (got) k = ((const volatile int *)&g_meta[qg % WG_NSG])[0];
                }
                if (!__shfl_sync(0xffffffffu, got, 0) || __shfl_sync(0xffffffffu, k, 0) < 0) break;
                const uint8_t *src = s_g + (qg % WG_NSG) * WG_GSLOT + ((size_t)chunk * TILE_M + pg * 8) * 16;
#pragma unroll
                for (int px = 0; px < 8; ++px) {
                    const uint4 q = *reinterpret_cast<const uint4 *>(src + px * 16);
                    const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        cs[2 * h] += __uint_as_float(w4[h] << 16);
                        cs[2 * h + 1] += __uint_as_float(w4[h] & 0xFFFF0000u);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&g_empty[qg % WG_NSG]));
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) cs[i] += __shfl_xor_sync(0xffffffffu, cs[i], o);
        }
        if (pg == 0)
            for (int i = 0; i < 8; ++i) P.colsum[(size_t)blockIdx.x * 64 + chunk * 8 + i] = cs[i];
        // weight-gradient partial sums of this CTA
        int got = 0;
        if (lane == 0) got = mbar_wait(smem_u32(done), 0, s_abort, P.err, true) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        tc_fence_after();
        if (got) {
            for (int t = 0; t < WG_TILES; ++t)
                for (int c0 = 0; c0 < 64; c0 += 16) {
                    float v[16];
                    tmem_ld16(lane_base + t * 64 + c0, v);
                    tmem_wait_ld();
                    float *dst = P.partials + (((size_t)blockIdx.x * WG_TILES + t) * 64 + c0) * 128 + quarter * 32 + lane;
#pragma unroll
                    for (int i = 0; i < 16; ++i) dst[(size_t)i * 128] = v[i];
                }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// dW[n][c][dy][dx] and db[n] of a 64 -> 64 layer from the CTAs' partial sums
// (compensated FP32, fixed order: slice r sums CTAs r, r + 4, ..., then the slices
// in order).
// Block = 64 values (tile, n, lane order, so the reads coalesce) x 4 CTA slices.
constexpr int RWG_VALS = WG_TILES * 64 * 128 + 64;
__global__ void __launch_bounds__(256) k_reduce_wgrad_tc(const float *__restrict__ partials,
                                                         const float *__restrict__ colsum, int ncta,
                                                         float *__restrict__ gw, float *__restrict__ gb)
{
    __shared__ float s_part[4][2][64];
    const int v = threadIdx.x & 63, r = threadIdx.x >> 6;
    const int i = blockIdx.x * 64 + v;
    const size_t st = (size_t)WG_TILES * 64 * 128;
    Kahan acc;
    if (i < WG_TILES * 64 * 128) {
#pragma unroll 4
        for (int k = r; k < ncta; k += 4) acc.add(partials[(size_t)k * st + i]);
    } else if (i < RWG_VALS) {
        for (int k = r; k < ncta; k += 4) acc.add(colsum[(size_t)k * 64 + (i - WG_TILES * 64 * 128)]);
    }
    s_part[r][0][v] = acc.s;
    s_part[r][1][v] = acc.c;
    __syncthreads();
    if (r != 0 || i >= RWG_VALS) return;
    for (int k = 1; k < 4; ++k) {
        acc.add(s_part[k][0][v]);
        acc.add(-s_part[k][1][v]);
    }
    const float s = acc.s;
    if (i < WG_TILES * 64 * 128) {
        const int t = i / (64 * 128), n = (i / 128) % 64, lane = i % 128;
        const int dx = t >> 1, pair = t & 1;
        if (pair == 1 && lane >= 64) return;               // rows of no tap
        const int dy = pair ? 2 : (lane >> 6), c = lane & 63;
        gw[((n * 64 + c) * 3 + dy) * 3 + dx] = s;
    } else {
        gb[i - WG_TILES * 64 * 128] = s;
    }
}

// Data-gradient weights of a 64 -> 64 layer in the pipeline's B layout:
// Wt[c][n][dy][dx] = W[n][c][2 - dy][2 - dx] packed as [dx][chunk of n][2 - dy][c][8 n].
__global__ void k_pack_dgrad(const float *__restrict__ w, __nv_bfloat16 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * 8 * 3 * 64 * 8) return;
    const int e = i % 8, o = (i / 8) % 64, s = (i / 512) % 3, k = (i / 1536) % 8, dx = i / 12288;
    const int n = k * 8 + e, c = o;                     // Wt input channel n, output channel c
    // Wt[c][n][dy = 2 - s][dx] = W[n][c][s][2 - dx]
    out[i] = __float2bfloat16_rn(w[((n * 64 + c) * 3 + s) * 3 + (2 - dx)]);
}

// ---------------------------------------------------------------------------
// Head (64 -> 1) backward on CUDA cores, one 32 x 8 tile per block.
// Table: act[0] = a_{L-2} (bf16), act[1] = g_{L-2} output (bf16), mask = ReLU mask
// of a_{L-2}, prob = dz (FP32 [H][W]).
//   g(y,x)[c] = mask * sum_{dy,dx} w[c][dy][dx] dz(y - dy + 1, x - dx + 1)
//   dW[c][dy][dx] += sum dz(y,x) a[c](y + dy - 1, x + dx - 1);  db += sum dz
// Per-block partial sums (576 weights + bias) go to partials[block][577].
// ---------------------------------------------------------------------------
struct HeadBwdParams {
    const ImgDesc *imgs;
    int n_imgs, n_tiles;
    float w[9 * 64];          // [tap][c]
    float *partials;          // [gridDim.x][577]
};

// Persistent: block b handles tiles b, b + grid, ...; its weight-gradient sums stay
// in registers across tiles and are written once.  The data gradient is formed and
// stored 8 channels (one 16-byte chunk) at a time, so that four blocks fit on an SM.
__global__ void __launch_bounds__(HT_X *HT_Y, 4) k_head_bwd(const HeadBwdParams P)
{
    __shared__ float s_dz[HT_Y + 2][HT_X + 2];
    __shared__ __align__(16) __nv_bfloat16 s_a[(HT_Y + 2) * (HT_X + 2) * 64];
    const int tid = threadIdx.y * HT_X + threadIdx.x;
    float wacc[3] = {0.f, 0.f, 0.f};                    // (c, dy) threads: dx = 0, 1, 2; thread 192: bias
    for (int tile = blockIdx.x; tile < P.n_tiles; tile += gridDim.x) {
        const int im = find_image(P.n_imgs, tile, [&](int i) { return __ldg(&P.imgs[i].hd_begin); });
        const ImgDesc *D = P.imgs + im;
        const int lt = tile - D->hd_begin;
        const int H = D->H, W = D->W;
        const int hx = (W + HT_X - 1) / HT_X;
        const int x0 = (lt % hx) * HT_X, y0 = (lt / hx) * HT_Y;
        const float *dz = D->prob;
        const uint8_t *a = D->act[0];
        __syncthreads();                                 // previous tile's shared reads are done
        for (int k = tid; k < (HT_Y + 2) * (HT_X + 2); k += HT_X * HT_Y) {
            const int yy = y0 - 1 + k / (HT_X + 2), xx = x0 - 1 + k % (HT_X + 2);
            s_dz[k / (HT_X + 2)][k % (HT_X + 2)] =
                (yy >= 0 && yy < H && xx >= 0 && xx < W) ? dz[(size_t)yy * W + xx] : 0.f;
        }
        for (int k = tid; k < (HT_Y + 2) * (HT_X + 2) * 8; k += HT_X * HT_Y) {
            const int chunk = k % 8, p = k / 8;
            const int yy = y0 - 1 + p / (HT_X + 2), xx = x0 - 1 + p % (HT_X + 2);
            uint4 q = make_uint4(0, 0, 0, 0);
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                q = *reinterpret_cast<const uint4 *>(a + (((size_t)chunk * H + yy) * W + xx) * 16);
            *reinterpret_cast<uint4 *>(&s_a[(size_t)p * 64 + chunk * 8]) = q;
        }
        __syncthreads();
        // data gradient at this thread's pixel
        const int y = y0 + threadIdx.y, x = x0 + threadIdx.x;
        if (y < H && x < W) {
            float d[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) d[t] = s_dz[threadIdx.y + 2 - t / 3][threadIdx.x + 2 - t % 3];
            const uint2 m = D->mask[(size_t)y * W + x];
            uint8_t *o = D->act[1];
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) {
                float g[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int c = 8 * ch + e;
                    float acc = 0.f;
#pragma unroll
                    for (int t = 0; t < 9; ++t) acc = fmaf(P.w[t * 64 + c], d[t], acc);
                    g[e] = (((c < 32 ? m.x : m.y) >> (c & 31)) & 1u) ? acc : 0.f;
                }
                uint4 q;
                q.x = pack_bf16x2(g[0], g[1]);
                q.y = pack_bf16x2(g[2], g[3]);
                q.z = pack_bf16x2(g[4], g[5]);
                q.w = pack_bf16x2(g[6], g[7]);
                *reinterpret_cast<uint4 *>(o + (((size_t)ch * H + y) * W + x) * 16) = q;
            }
        }
        // weight and bias gradient sums of this tile: thread (c, dy) keeps the three dx
        // taps and slides along the row (one activation load per pixel); thread 192 sums dz
        if (tid < 192) {
            const int c = tid & 63, dy = tid >> 6;
            for (int py = 0; py < HT_Y; ++py) {
                const __nv_bfloat16 *arow = s_a + (size_t)(py + dy) * (HT_X + 2) * 64 + c;
                float a0 = __bfloat162float(arow[0]), a1 = __bfloat162float(arow[64]);
#pragma unroll 8
                for (int px = 0; px < HT_X; ++px) {
                    const float a2 = __bfloat162float(arow[(px + 2) * 64]);
                    const float d = s_dz[py + 1][px + 1];
                    wacc[0] = fmaf(d, a0, wacc[0]);
                    wacc[1] = fmaf(d, a1, wacc[1]);
                    wacc[2] = fmaf(d, a2, wacc[2]);
                    a0 = a1;
                    a1 = a2;
                }
            }
        } else if (tid == 192) {
            for (int py = 0; py < HT_Y; ++py)
                for (int px = 0; px < HT_X; ++px) wacc[0] += s_dz[py + 1][px + 1];
        }
    }
    if (tid < 192) {
        const int c = tid & 63, dy = tid >> 6;
        for (int dx = 0; dx < 3; ++dx) P.partials[(size_t)blockIdx.x * 577 + (dy * 3 + dx) * 64 + c] = wacc[dx];
    } else if (tid == 192) {
        P.partials[(size_t)blockIdx.x * 577 + 576] = wacc[0];
    }
}

// ---------------------------------------------------------------------------
// Layer-1 (2 -> 64) weight gradient on CUDA cores, one 32 x 8 tile per block.
// Table: act[0] = g_1 (bf16), contone, image (Philox index).  Input channels
// c and z (Philox stream 0, the forward's noise) exactly as FP32.
//   dW[n][ci][dy][dx] += sum g[n](y,x) x_ci(y + dy - 1, x + dx - 1); db[n] += sum g[n]
// partials[block][1152 + 64] with weight entry (ci*9 + tap)*64 + n.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(HT_X *HT_Y) k_first_wgrad(const ImgDesc *__restrict__ imgs, int n_imgs, int n_tiles,
                                                           uint64_t seed, float *__restrict__ partials)
{
    __shared__ float s_x[2][HT_Y + 2][HT_X + 2];
    __shared__ __align__(16) __nv_bfloat16 s_g[HT_Y * HT_X * 64];
    __shared__ float s_half[1216];
    const int tid = threadIdx.y * HT_X + threadIdx.x;
    // thread (n, ci, half): the nine taps of weight (n, ci) over tile rows half*4 .. +3;
    // ci = 0 threads also sum g[n] (bias)
    const int n = tid & 63, ci = (tid >> 6) & 1, half = tid >> 7;
    float wacc[9], bacc = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) wacc[t] = 0.f;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int im = find_image(n_imgs, tile, [&](int i) { return __ldg(&imgs[i].hd_begin); });
        const ImgDesc *D = imgs + im;
        const int lt = tile - D->hd_begin;
        const int H = D->H, W = D->W;
        const int hx = (W + HT_X - 1) / HT_X;
        const int x0 = (lt % hx) * HT_X, y0 = (lt / hx) * HT_Y;
        __syncthreads();
        for (int k = tid; k < (HT_Y + 2) * (HT_X + 2); k += HT_X * HT_Y) {
            const int r = k / (HT_X + 2), q = k % (HT_X + 2);
            const int yy = y0 - 1 + r, xx = x0 - 1 + q;
            const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
            s_x[0][r][q] = in ? D->contone[(size_t)yy * D->cpitch + xx] : 0.f;
            s_x[1][r][q] = in ? ht_uniform24(seed, D->image, 0u, (uint64_t)yy * W + xx) : 0.f;
        }
        for (int k = tid; k < HT_Y * HT_X * 8; k += HT_X * HT_Y) {
            const int chunk = k % 8, p = k / 8;
            const int yy = y0 + p / HT_X, xx = x0 + p % HT_X;
            uint4 q = make_uint4(0, 0, 0, 0);
            if (yy < H && xx < W) q = *reinterpret_cast<const uint4 *>(D->act[0] + (((size_t)chunk * H + yy) * W + xx) * 16);
            *reinterpret_cast<uint4 *>(&s_g[(size_t)p * 64 + chunk * 8]) = q;
        }
        __syncthreads();
        for (int py = half * (HT_Y / 2); py < (half + 1) * (HT_Y / 2); ++py) {
            // the 3 x 3 input window slides along the row: one new column per pixel
            const float *r0 = &s_x[ci][py][0], *r1 = &s_x[ci][py + 1][0], *r2 = &s_x[ci][py + 2][0];
            float a00 = r0[0], a01 = r0[1], a10 = r1[0], a11 = r1[1], a20 = r2[0], a21 = r2[1];
#pragma unroll 4
            for (int px = 0; px < HT_X; ++px) {
                const float g = __bfloat162float(s_g[(py * HT_X + px) * 64 + n]);
                bacc += g;
                const float a02 = r0[px + 2], a12 = r1[px + 2], a22 = r2[px + 2];
                wacc[0] = fmaf(g, a00, wacc[0]);
                wacc[1] = fmaf(g, a01, wacc[1]);
                wacc[2] = fmaf(g, a02, wacc[2]);
                wacc[3] = fmaf(g, a10, wacc[3]);
                wacc[4] = fmaf(g, a11, wacc[4]);
                wacc[5] = fmaf(g, a12, wacc[5]);
                wacc[6] = fmaf(g, a20, wacc[6]);
                wacc[7] = fmaf(g, a21, wacc[7]);
                wacc[8] = fmaf(g, a22, wacc[8]);
                a00 = a01;
                a01 = a02;
                a10 = a11;
                a11 = a12;
                a20 = a21;
                a21 = a22;
            }
        }
    }
    // combine the two row halves in a fixed order
    __syncthreads();
    if (half == 1) {
#pragma unroll
        for (int t = 0; t < 9; ++t) s_half[(ci * 9 + t) * 64 + n] = wacc[t];
        if (ci == 0) s_half[1152 + n] = bacc;
    }
    __syncthreads();
    if (half == 0) {
#pragma unroll
        for (int t = 0; t < 9; ++t)
            partials[(size_t)blockIdx.x * 1216 + (ci * 9 + t) * 64 + n] = wacc[t] + s_half[(ci * 9 + t) * 64 + n];
        if (ci == 0) partials[(size_t)blockIdx.x * 1216 + 1152 + n] = bacc + s_half[1152 + n];
    }
}

// Sum of per-block partials (compensated FP32, fixed order: slice r sums blocks r,
// r + 8, ..., then the 8 slices in order).  CTA = 32 values x 8 slices.  mode 0: head, entries
// [tap][c] + bias; mode 1: layer 1, entries [(ci*9 + tap)][n] + 64 biases.
__global__ void __launch_bounds__(256) k_reduce_blocks(const float *__restrict__ partials, int nblk, int nval, int mode,
                                                       float *__restrict__ gw, float *__restrict__ gb)
{
    __shared__ float s_part[8][2][32];
    const int v = threadIdx.x & 31, r = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + v;
    Kahan acc;
    if (i < nval)
        for (int b = r; b < nblk; b += 8) acc.add(partials[(size_t)b * nval + i]);
    s_part[r][0][v] = acc.s;
    s_part[r][1][v] = acc.c;
    __syncthreads();
    if (r != 0 || i >= nval) return;
    for (int k = 1; k < 8; ++k) {
        acc.add(s_part[k][0][v]);
        acc.add(-s_part[k][1][v]);
    }
    const float s = acc.s;
    if (mode == 0) {
        if (i < 576) gw[(i % 64) * 9 + i / 64] = s;              // W_head[0][c][tap]
        else gb[0] = s;
    } else {
        if (i < 1152) {
            const int n = i % 64, k = i / 64;                      // k = ci*9 + tap
            gw[(n * 2 + k / 9) * 9 + k % 9] = s;
        } else {
            gb[i - 1152] = s;
        }
    }
}

unsigned nblk256(size_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
bool ht_train_tc_supported(const ht_policy *p)
{
    if (p->prec != HT_BF16 || (p->head != HT_HEAD_SIGMOID && p->head != HT_HEAD_MULTITONE) || p->K != 1 || p->L < 3)
        return false;
    if (p->ch[0] != 2) return false;
    for (int l = 1; l < p->L; ++l)
        if (p->ch[l] != 64) return false;
    return true;
}

// Per image of a step, in the arena (px = h * w), each region 256-byte aligned:
// activation buffers [nbuf][px][128 B], ReLU masks [L-1][px] x 8 B, layer-1 split
// input [2 chunks][px][16 B], head partials [9][px] x 4 B, gradient ping-pong 2 x [px][128 B].
//
// Activation recomputation (checkpoint stride k > 1): only the hidden activations
// a_l with l % k == 0, and a_{L-2} (the head's input), keep a buffer for the
// backward; the others use k - 1 scratch buffers (a_l in scratch l % k - 1), which
// the forward overwrites segment by segment and the backward refills by running the
// segment's forward layers again from its checkpoint (the kernels are
// deterministic, so the refilled activations and masks are the forward's).
namespace {
inline size_t al256(size_t b) { return (b + 255) / 256 * 256; }
struct ImgRegions {
    size_t acts, masks, split, part9, g0, g1, total;
};
inline bool is_ckpt(int l, int k, int L) { return k <= 1 || l % k == 0 || l == L - 2; }
inline int n_ckpt(int k, int L)
{
    int n = 0;
    for (int l = 0; l <= L - 2; ++l) n += is_ckpt(l, k, L) ? 1 : 0;
    return n;
}
inline int n_act_bufs(int k, int L) { return n_ckpt(k, L) + (k > 1 ? k - 1 : 0); }
// buffer of hidden activation a_l
inline int act_buf(int l, int k, int L)
{
    if (!is_ckpt(l, k, L)) return n_ckpt(k, L) + (l % k) - 1;
    int i = 0;
    for (int j = 0; j < l; ++j) i += is_ckpt(j, k, L) ? 1 : 0;
    return i;
}
ImgRegions img_regions(int nh, int nbuf, size_t px)
{
    ImgRegions r;
    r.acts = 0;
    r.masks = r.acts + al256((size_t)nbuf * px * 128);
    r.split = r.masks + al256((size_t)nh * px * 8);
    r.part9 = r.split + al256(px * 32);
    r.g0 = r.part9 + al256(px * 36);
    r.g1 = r.g0 + al256(px * 128);
    r.total = r.g1 + al256(px * 128);
    return r;
}
}  // namespace

size_t ht_train_tc_image_bytes(const ht_policy *p, int ckpt, size_t px)
{
    return img_regions(p->L - 1, n_act_bufs(ckpt, p->L), px).total;
}

size_t ht_train_tc_table_bytes(const ht_policy *p, int n_img)
{
    return (size_t)(3 * p->L - 2) * n_img * sizeof(ImgDesc);
}

// partial-sum region (CTA partials of the tcgen05 weight gradient, or per-tile
// partials of the CUDA-core ones) followed by the packed data-gradient weights
void ht_train_tc_scratch_layout(const ht_policy *p, int n_tiles, size_t *wt_off, size_t *total)
{
    const size_t wg = (size_t)num_sms() * (WG_TILES * 64 * 128 + 64) * sizeof(float);
    const size_t blk = (size_t)n_tiles * 1216 * sizeof(float);
    const size_t part = ((wg > blk ? wg : blk) + 255) / 256 * 256;
    *wt_off = part;
    *total = part + (size_t)(p->L > 2 ? p->L - 2 : 1) * 36864 * sizeof(__nv_bfloat16);
}

namespace {
// Table indices of one step (each table = one ImgDesc per image of the step).
constexpr int T_FIRST = 0;                               // layer 1
inline int T_FWD(int l) { return l; }                    // inner layer l = 1 .. L-2
inline int T_HEAD(int L) { return L - 1; }               // head forward
inline int T_HB(int L) { return L; }                     // head backward
inline int T_WG(int L, int l) { return L + l; }          // weight gradient of inner layer l
inline int T_W1(int L) { return 2 * L - 1; }             // layer-1 weight gradient
inline int T_DG(int L, int l) { return 2 * L - 1 + l; }  // data gradient through inner layer l
inline int n_tables(int L) { return 3 * L - 2; }

void build_tables(const ht_policy *p, const ht_train_tc_ws &w, const ht_image *imgs, int nimg,
                  std::vector<ImgDesc> &all, int &units, int &hd, int &pre, int &hq)
{
    const int L = p->L, nh = L - 1;
    units = hd = pre = hq = 0;
    std::vector<ImgDesc> D0(nimg);
    for (int i = 0; i < nimg; ++i) {
        ImgDesc D{};
        D.contone = imgs[i].contone;
        D.cpitch = imgs[i].pitch;
        D.H = imgs[i].h;
        D.W = imgs[i].w;
        D.image = (uint32_t)i;
        D.words = ht_bits_row_words(D.W, HT_HEAD_SIGMOID);
        set_begins(D, units, hd, pre, RU, nullptr, &hq);
        D0[i] = D;
    }
    all.assign((size_t)n_tables(L) * nimg, ImgDesc{});
    for (int i = 0; i < nimg; ++i) {
        const size_t px = (size_t)imgs[i].h * imgs[i].w;
        const ImgRegions R = img_regions(nh, n_act_bufs(w.ckpt, L), px);
        uint8_t *b = (uint8_t *)w.arena + w.img_off[i];
        uint8_t *acts = b + R.acts;
        uint2 *masks = (uint2 *)(b + R.masks);
        uint8_t *split = b + R.split;
        float *part9 = (float *)(b + R.part9);
        uint8_t *g0 = b + R.g0;
        uint8_t *g1 = b + R.g1;
        auto act = [&](int l) { return acts + (size_t)act_buf(l, w.ckpt, L) * px * 128; };
        auto msk = [&](int l) { return masks + (size_t)l * px; };
        auto gbuf = [&](int l) { return (l & 1) ? g1 : g0; };   // g_l: gradient at layer l's pre-activation
        auto T = [&](int t) -> ImgDesc & { return all[(size_t)t * nimg + i]; };
        // forward
        T(T_FIRST) = D0[i];
        T(T_FIRST).act[0] = act(0);
        T(T_FIRST).act[1] = split;
        T(T_FIRST).mask = msk(0);
        for (int l = 1; l <= L - 2; ++l) {
            ImgDesc &D = T(T_FWD(l));
            D = D0[i];
            D.act[0] = act(l - 1);
            D.act[1] = l == L - 2 ? (uint8_t *)part9 : act(l);
            D.mask = msk(l);
            D.save = l == L - 2 ? act(l) : nullptr;
        }
        {
            ImgDesc &D = T(T_HEAD(L));
            D = D0[i];
            D.act[0] = (uint8_t *)part9;
            D.prob = w.prob + w.prob_off[i];
            D.bits = w.hbits + w.bits_off[i];
        }
        // backward
        {
            ImgDesc &D = T(T_HB(L));
            D = D0[i];
            D.act[0] = act(L - 2);
            D.act[1] = gbuf(L - 2);
            D.mask = msk(L - 2);
            D.prob = w.dz + w.prob_off[i];
        }
        for (int l = 1; l <= L - 2; ++l) {
            ImgDesc &Wg = T(T_WG(L, l));
            Wg = D0[i];
            Wg.act[0] = act(l - 1);
            Wg.act[1] = gbuf(l);
            ImgDesc &Dg = T(T_DG(L, l));
            Dg = D0[i];
            Dg.act[0] = gbuf(l);
            Dg.act[1] = gbuf(l - 1);
            Dg.mask = msk(l - 1);
        }
        T(T_W1(L)) = D0[i];
        T(T_W1(L)).act[0] = gbuf(0);
    }
}
}  // namespace

ht_status ht_train_tc_forward(ht_policy *p, ht_train_tc_ws &w, const ht_image *imgs, int nimg, uint64_t seed,
                              cudaStream_t s)
{
    const int L = p->L;
    std::vector<ImgDesc> all;
    int units, hd, pre, hq;
    build_tables(p, w, imgs, nimg, all, units, hd, pre, hq);
    w.units = units;
    w.hd = hd;
    HT_CUDA_TRY(cudaMemcpyAsync(w.tables, all.data(), all.size() * sizeof(ImgDesc), cudaMemcpyHostToDevice, s));
    auto tab = [&](int t) { return (const void *)((const ImgDesc *)w.tables + (size_t)t * nimg); };
    ht_status st = ht_tc_first_input(tab(T_FIRST), nimg, pre, seed, s);
    if (st != HT_OK) return st;
    {
        ht_tc_layer a{};
        a.table = tab(T_FIRST);
        a.n_imgs = nimg;
        a.n_units = units;
        a.in_buf = 1;
        a.kind = 2;
        a.wpack = p->d_w1pack;
        a.bias = p->h_b + p->b_off[0];
        a.seed = seed;
        if ((st = ht_tc_conv(a, s)) != HT_OK) return st;
    }
    for (int l = 1; l <= L - 2; ++l) {
        ht_tc_layer a{};
        a.table = tab(T_FWD(l));
        a.n_imgs = nimg;
        a.n_units = units;
        a.in_buf = 0;
        a.kind = l == L - 2 ? 1 : 0;
        a.wpack = (const uint8_t *)p->d_wpack + p->wpack_layer_bytes * (l - 1);
        a.bias = p->h_b + p->b_off[l];
        a.head_w = l == L - 2 ? p->h_headw : nullptr;
        a.seed = seed;
        if ((st = ht_tc_conv(a, s)) != HT_OK) return st;
    }
    return ht_tc_head_partials(tab(T_HEAD(L)), nimg, hq, 0, p->head_bias, HT_MODE_THRESHOLD, seed, s);
}

ht_status ht_train_tc_backward(ht_policy *p, ht_train_tc_ws &w, int nimg, uint64_t seed, float *grad_w, float *grad_b,
                               cudaStream_t s)
{
    const int L = p->L;
    int *err = ht_device_error_flag();
    if (!err) return HT_ERR_CUDA;
    auto tab = [&](int t) { return (const ImgDesc *)w.tables + (size_t)t * nimg; };
    float *wpart = (float *)w.scratch;
    __nv_bfloat16 *wt = (__nv_bfloat16 *)((uint8_t *)w.scratch + w.wt_off);
    // data-gradient weights of every inner layer
    for (int l = 1; l <= L - 2; ++l) {
        k_pack_dgrad<<<nblk256(36864), 256, 0, s>>>(p->d_w + p->w_off[l], wt + (size_t)(l - 1) * 36864);
        HT_LAUNCH_CHECK();
    }
    // head backward: g_{L-2}, dW / db of the head (persistent blocks over the head tiles)
    const int nbg = w.hd < 4 * num_sms() ? w.hd : 4 * num_sms();
    {
        HeadBwdParams P;
        P.imgs = tab(T_HB(L));
        P.n_imgs = nimg;
        P.n_tiles = w.hd;
        memcpy(P.w, p->h_headw, sizeof(P.w));
        P.partials = wpart;
        static bool carveout_set = false;           // 4 blocks x 45 KB of shared memory per SM
        if (!carveout_set) {
            HT_CUDA_TRY(cudaFuncSetAttribute(k_head_bwd, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared));
            carveout_set = true;
        }
        ht_prof_start(HTK_TRAIN, s);
        k_head_bwd<<<nbg, dim3(HT_X, HT_Y), 0, s>>>(P);
        ht_prof_stop(s);
        HT_LAUNCH_CHECK();
        k_reduce_blocks<<<(577 + 31) / 32, 256, 0, s>>>(wpart, nbg, 577, 0, grad_w + p->w_off[L - 1],
                                                       grad_b + p->b_off[L - 1]);
        HT_LAUNCH_CHECK();
    }
    static bool attr = false;
    if (!attr) {
        HT_CUDA_TRY(cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM));
        attr = true;
    }
    const int grid = w.units < num_sms() ? w.units : num_sms();
    int seg_ready = -1;                                     // checkpoint below the segment held in scratch
    for (int l = L - 2; l >= 1; --l) {
        if (!is_ckpt(l - 1, w.ckpt, L)) {
            const int c = (l - 1) - (l - 1) % w.ckpt;
            if (seg_ready != c) {                           // refill a_{c+1} .. a_{l-1} from checkpoint a_c
                for (int j = c + 1; j <= l - 1; ++j) {
                    ht_tc_layer a{};
                    a.table = tab(T_FWD(j));
                    a.n_imgs = nimg;
                    a.n_units = w.units;
                    a.in_buf = 0;
                    a.kind = 0;
                    a.wpack = (const uint8_t *)p->d_wpack + p->wpack_layer_bytes * (j - 1);
                    a.bias = p->h_b + p->b_off[j];
                    a.seed = seed;
                    const ht_status st = ht_tc_conv(a, s);
                    if (st != HT_OK) return st;
                }
                seg_ready = c;
            }
        }
        WgParams P;
        P.imgs = tab(T_WG(L, l));
        P.n_imgs = nimg;
        P.n_units = w.units;
        P.partials = wpart;
        P.colsum = wpart + (size_t)grid * WG_TILES * 64 * 128;
        P.err = err;
        ht_prof_start(HTK_TRAIN, s);
        k_wgrad_tc<<<grid, WG_NTHREADS, WG_SMEM, s>>>(P);
        ht_prof_stop(s);
        HT_LAUNCH_CHECK();
        k_reduce_wgrad_tc<<<(RWG_VALS + 63) / 64, 256, 0, s>>>(P.partials, P.colsum, grid, grad_w + p->w_off[l],
                                                               grad_b + p->b_off[l]);
        HT_LAUNCH_CHECK();
        ht_tc_layer a{};
        a.table = tab(T_DG(L, l));
        a.n_imgs = nimg;
        a.n_units = w.units;
        a.in_buf = 0;
        a.kind = 0;
        a.wpack = wt + (size_t)(l - 1) * 36864;
        a.dgrad = 1;
        a.seed = seed;
        ht_status st = ht_tc_conv(a, s);
        if (st != HT_OK) return st;
    }
    ht_prof_start(HTK_TRAIN, s);
    k_first_wgrad<<<nbg, dim3(HT_X, HT_Y), 0, s>>>(tab(T_W1(L)), nimg, w.hd, seed, wpart);
    ht_prof_stop(s);
    HT_LAUNCH_CHECK();
    k_reduce_blocks<<<(1216 + 31) / 32, 256, 0, s>>>(wpart, nbg, 1216, 1, grad_w + p->w_off[0], grad_b + p->b_off[0]);
    HT_LAUNCH_CHECK();
    return HT_OK;
}

void ht_preload_train_tc()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_wgrad_tc);
    cudaFuncGetAttributes(&fa, k_reduce_wgrad_tc);
    cudaFuncGetAttributes(&fa, k_pack_dgrad);
    cudaFuncGetAttributes(&fa, k_head_bwd);
    cudaFuncGetAttributes(&fa, k_first_wgrad);
    cudaFuncGetAttributes(&fa, k_reduce_blocks);
    cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM);
}
