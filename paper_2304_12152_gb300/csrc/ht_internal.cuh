// ht_internal.cuh -- internal declarations shared by the library's CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <stdio.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ht.h"

// NVTX range over one public entry point, named after it, for timelines and for
// ncu --nvtx filtering.  Header-only NVTX 3: without an attached tool each push / pop
// is a call through a no-op stub.
struct HtRange {
    explicit HtRange(const char *name) { nvtxRangePushA(name); }
    ~HtRange() { nvtxRangePop(); }
    HtRange(const HtRange &) = delete;
    HtRange &operator=(const HtRange &) = delete;
};
#define HT_RANGE(name) HtRange ht_range_(name)

// ---------------------------------------------------------------------------
// Error plumbing
// ---------------------------------------------------------------------------
void ht_set_error(const char *fmt, ...);

#define HT_CHECK_ARG(cond, ...)                 \
    do {                                        \
        if (!(cond)) {                          \
            ht_set_error(__VA_ARGS__);          \
            return HT_ERR_INVALID_ARG;          \
        }                                       \
    } while (0)

#define HT_CUDA_TRY(expr)                                                              \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            ht_set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? HT_ERR_OOM : HT_ERR_CUDA;          \
        }                                                                              \
    } while (0)

#define HT_LAUNCH_CHECK()                                                              \
    do {                                                                               \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess) {                                                       \
            ht_set_error("%s:%d: launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
            return HT_ERR_CUDA;                                                        \
        }                                                                              \
    } while (0)

// Device-side error record (8 ints, one per device context): [0] status
// (HT_ERR_TIMEOUT when a bounded wait expires), [1] set once, [2..7] where the
// first expiry happened (barrier address, threads and warp, block, polls,
// elapsed ns as u64).  ht_sync() reads, reports and clears it.
int *ht_device_error_flag();

// Kernel timing hooks (no-ops unless ht_profile_begin was called).
enum ht_kernel_id { HTK_FIRST_TC = 0, HTK_CONV_TC_BF16, HTK_CONV_TC_FP8, HTK_HEAD_TC, HTK_CONV_FP32, HTK_HEAD_FP32,
                    HTK_REWARD, HTK_TOGGLE, HTK_SPECTRUM, HTK_TRAIN, HTK_FIRST_INPUT, HTK_CONV_TC_FP16, HTK_COUNT };
void ht_prof_start(int kid, cudaStream_t s);
void ht_prof_stop(cudaStream_t s);

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Key (seed lo, seed hi),
// counter (g >> 2, image, stream, 0), output lane g & 3; u = (x >> 8) * 2^-24.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 ht_philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ float ht_uniform24(uint64_t seed, uint32_t image, uint32_t stream, uint64_t g)
{
    const uint4 r = ht_philox4x32_10(make_uint4((uint32_t)(g >> 2), image, stream, 0u),
                                     make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const uint32_t lane = (uint32_t)g & 3u;
    const uint32_t x = lane == 0 ? r.x : lane == 1 ? r.y : lane == 2 ? r.z : r.w;
    return (float)(x >> 8) * (1.0f / 16777216.0f);
}

// ---------------------------------------------------------------------------
// Policy object
// ---------------------------------------------------------------------------
struct ht_policy {
    int L;                          // conv layers
    int ch[HT_MAX_LAYERS + 1];
    int head, K, prec;
    int levels;                     // output levels (2 binary, 4 softmax head, 2..4 multitone head)
    int arch;                       // HT_ARCH_PLAIN or HT_ARCH_RESNET
    int width;                      // hidden width of the tensor-core forms (64; 32 for the residual policy)
    int device;
    int64_t n_w, n_b;
    int64_t w_off[HT_MAX_LAYERS + 1], b_off[HT_MAX_LAYERS + 1];
    float *d_w = nullptr;           // canonical fp32 OIHW, all layers
    float *d_b = nullptr;
    // tensor-core form: packed inner-layer weights ([tap][c8][n][8] per layer)
    void *d_wpack = nullptr;
    size_t wpack_layer_bytes = 0;
    float *d_wscale = nullptr;      // FP8: per (layer, out channel) dequant scale
    float act_scale[HT_MAX_LAYERS];
    // host copies of the small per-channel constants the tensor-core kernels take as
    // kernel parameters (refreshed by every repack)
    float h_b[HT_MAX_LAYERS * HT_MAX_CHANNELS + 4];
    float h_wscale[HT_MAX_LAYERS * 64];
    float h_headw[9 * 64];          // 1-logit head: last-layer weights as [9 taps][64]
    void *d_w1pack = nullptr;       // layer 1 for the tensor cores: bf16 hi/lo split, [dx][chunk][3 dy][n][8]
    void *d_wpack4 = nullptr;       // 4-logit head: [dx][chunk][3 dy][16 n][8] bf16 (FP16 form: binary16),
                                    // n = hi 0..3, lo 4..7
    float head4_inv_scale = 1.f;    // FP16 form: the 4-logit head's weights are stored x 2^k (kept in the
                                    // binary16 normal range), its logits multiplied back by 2^-k
    float head_bias = 0.f;
    // conv schedule of the tensor-core forms (set by ht_policy_autotune): rows per work
    // unit (up to 8: one TMEM accumulator block per row; more: a streaming strip over the
    // TMEM ring) and unit order.  Policies of the 64-wide plain architecture start at
    // 64-row strips, column tiles first.
    int tune_ru = 8, tune_order = 0;
    int tune_pair = 0;              // 1: 64 -> 64 layers of the inference forms run as CTA pairs (M = 256)
    // CTA-pair weight images of the inner 64 -> 64 layers (two per layer, one per CTA of a pair)
    void *d_wpack2 = nullptr;
    size_t wpack2_layer_bytes = 0;
    uint64_t version = 0;           // bumped by every change of weights or scales (plans re-capture)
    // per-call workspace (grown on demand; library owned)
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
};

ht_status ht_policy_ensure_ws(ht_policy *p, size_t bytes);
// Argument checks shared by entry points (host only, no CUDA call): reward options
// (radius, levels, window sigmas) and image descriptors (non-null, min_side <= h, w <= 16384,
// pitch >= w).  Defined in api.cu inside its extern "C" block.
extern "C" ht_status ht_validate_reward_opts(const ht_reward_opts *o);
extern "C" ht_status ht_validate_images(const ht_image *imgs, int n, int min_side);
// The descriptor checks of ht_create_policy (shape, head, precision, architecture).
ht_status ht_validate_desc(const ht_policy_desc *d);
ht_status ht_pack_tc_weights(ht_policy *p, cudaStream_t s);

// ---------------------------------------------------------------------------
// Launchers (one per source file)
// ---------------------------------------------------------------------------
// plain FP32 form, one image
ht_status ht_run_fp32(ht_policy *p, const ht_image &img, uint32_t image_index, int mode, uint64_t seed,
                      uint32_t *bits, float *prob, float *act_a, float *act_b, cudaStream_t s);
size_t ht_fp32_ws_bytes(const ht_policy *p, int h, int w);
ht_status ht_fwd_fp32_save(ht_policy *p, const ht_image &img, uint32_t image_index, uint64_t seed,
                           float *const *acts, float *prob, uint32_t *bits, cudaStream_t s);
ht_status ht_dgrad_fp32(const float *g_out, const float *wt, int Cout, int Cin, int H, int W, const float *act_in,
                        float *g_in, cudaStream_t s);

// tensor-core form, all images of a call (grouped under a workspace budget)
ht_status ht_run_tc_batch(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed,
                          uint32_t *const *bits, float *const *prob, cudaStream_t s);
size_t ht_tc_ws_bytes(const ht_policy *p, int h, int w);
size_t ht_tc_batch_ws_bytes(const ht_policy *p, const ht_image *imgs, int n);

// Kernel preloading: every kernel of the library is loaded when the first policy
// is created (with lazy module loading a first launch can otherwise stall work
// already running on the GPU while the loader runs).
void ht_preload_conv_tc();
void ht_preload_conv_fp32();
void ht_preload_reward();
void ht_preload_spectrum();
void ht_preload_train();
void ht_preload_train_tc();
void ht_preload_kernels();

// CUDA-graph plans and the schedule autotuner of the tensor-core forms (conv_tc.cu)
ht_status ht_plan_create_impl(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed,
                              uint32_t *const *bits, float *const *prob, ht_plan **out);
ht_status ht_plan_launch_impl(ht_plan *pl, cudaStream_t s);
ht_status ht_plan_destroy_impl(ht_plan *pl);
ht_status ht_tc_autotune(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed, uint32_t *const *bits,
                         float *const *prob, int reps, ht_tune_result *out, int max_out, int *n_out, cudaStream_t s);

// single launches of the BF16 conv pipeline over a caller-built image table (training form)
struct ht_tc_layer {
    const void *table;        // device ImgDesc table (tc_common.cuh)
    int n_imgs, n_units, in_buf;
    int kind;                 // 0 hidden 64 -> 64, 1 last hidden + 1-logit head partials, 2 layer 1
    const void *wpack;        // packed bf16 weights ([dx][chunk][3 dy][64][16 B])
    const float *scale, *bias;   // host, 64 each (nullable: 1 / 0)
    const float *head_w;      // host [9][64] (kind 1)
    int dgrad;                // data-gradient layer: no bias / ReLU, mask from the table
    uint64_t seed;
};
ht_status ht_tc_conv(const ht_tc_layer &a, cudaStream_t s);
ht_status ht_tc_first_input(const void *table, int n_imgs, int n_groups, uint64_t seed, cudaStream_t s);
// n_tiles: 128 x 8 head tiles of the table (ImgDesc::hq_begin prefix sums)
ht_status ht_tc_head_partials(const void *table, int n_imgs, int n_tiles, int buf, float bias, int mode,
                              uint64_t seed, cudaStream_t s);

// reward / toggle deltas
ht_status ht_reward_launch(const ht_image *c, const uint32_t *const *bits, int n, const ht_reward_opts &o,
                           double *out, cudaStream_t s);
ht_status ht_toggle_launch(const ht_image *c, const uint32_t *const *bits, const float *const *v, int n,
                           const ht_reward_opts &o, float *const *dR, float *scratch, size_t scratch_floats,
                           cudaStream_t s);
size_t ht_toggle_scratch_floats(int h, int w, int r);
size_t ht_toggle_scratch_floats_batch(const ht_image *c, int n, int r);   // what ht_toggle_launch needs for c[0..n)

// spectrum
ht_status ht_las_launch(const float *q, int n_patches, int n, int mode, int n_rad, int n_ang, double *out_loss,
                        float *grad, void *scratch, size_t scratch_bytes, cudaStream_t s);
size_t ht_las_scratch_bytes(int n_patches, int n, int n_rad, int n_ang);

// BF16 tensor-core training form (train_tc.cu): 2 -> 64 x (L-1) -> 1 sigmoid policies
struct ht_train_tc_ws {
    void *arena = nullptr;            // per-image activations, masks, split input, head partials, gradients
    std::vector<size_t> slot_off;     // per image slot (crops, then gray patches): byte offset into the arena
    std::vector<size_t> img_off;      // per image of the step: byte offset into the arena
    std::vector<size_t> prob_off;     // per image: offset into prob / dz
    std::vector<size_t> bits_off;     // per image: word offset into hbits
    float *prob = nullptr, *dz = nullptr;
    uint32_t *hbits = nullptr;        // thresholded head output (unused by training, written by the head)
    void *tables = nullptr;           // device image tables of the step
    void *scratch = nullptr;          // reduction partials + packed data-gradient weights
    size_t scratch_bytes = 0, wt_off = 0;
    int units = 0, hd = 0;
    int ckpt = 1;                     // activation checkpoint stride (1: keep every hidden activation)
};
bool ht_train_tc_supported(const ht_policy *p);
size_t ht_train_tc_image_bytes(const ht_policy *p, int ckpt, size_t px);
size_t ht_train_tc_table_bytes(const ht_policy *p, int n_img);
void ht_train_tc_scratch_layout(const ht_policy *p, int n_tiles, size_t *wt_off, size_t *total);
ht_status ht_train_tc_forward(ht_policy *p, ht_train_tc_ws &w, const ht_image *imgs, int nimg, uint64_t seed,
                              cudaStream_t s);
ht_status ht_train_tc_backward(ht_policy *p, ht_train_tc_ws &w, int nimg, uint64_t seed, float *grad_w,
                               float *grad_b, cudaStream_t s);
