/*
 * ht.h -- C ABI of the GB300 halftoning library (libht.so).
 *
 * The library implements the data-parallel hot path of "Efficient Halftoning
 * via Deep Reinforcement Learning" (arXiv 2304.12152):
 *   - one-shot halftone generation (Algorithm 1, TEST step): a fully
 *     convolutional policy maps the state s = concat(c, z) (Sec. III, "State")
 *     to per-pixel action probabilities pi_a(h_a = 1) (Eq. independent), which
 *     are thresholded at 0.5 or Bernoulli-sampled and bit-packed;
 *   - the training-time reward R = -MSE(HVS(h), HVS(c)) + w_s CSSIM(h, c)
 *     (Eq. reward, Eq. final_reward, Eq. cssim), the per-pixel toggle deltas of
 *     the local-expectation gradient (Eq. le, Eq. marl, Sec. III-C) and the
 *     anisotropy-suppressing loss on the power spectrum (Eqs. psd, rapsd,
 *     anis, as; Sec. IV);
 *   - one training iteration's forward and backward (Algorithm 1, TRAIN step).
 *
 * Conventions for every entry point:
 *   - Pointers documented "device" must point into memory of the current CUDA
 *     device; "host" pointers are read before the call returns.  The caller
 *     owns every buffer it passes; the library owns ht_policy / ht_train
 *     objects and the device workspaces inside them.  A tensor-core call
 *     splits its images into groups whose activations (256 bytes per pixel)
 *     fit the workspace budget: the environment variable HT_WS_BUDGET_GB if
 *     set, else a quarter of the device's memory (at least 16 GB).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless stated; argument
 *     errors are detected on the host before any launch and return
 *     HT_ERR_INVALID_ARG / HT_ERR_UNSUPPORTED with nothing launched.
 *   - A kernel whose bounded internal wait expires records HT_ERR_TIMEOUT in
 *     a device flag; ht_sync() reports it (and any CUDA error).
 *   - ht_last_error() returns a thread-local description of the last failure.
 *
 * Data layouts:
 *   - contone image: float32 in [0, 1], row-major [h][pitch] (pitch >= w, in
 *     elements), device memory.
 *   - halftone (sigmoid head): 1 bit per pixel, LSB-first in uint32 words,
 *     row-major with ht_bits_row_words(w, 1) words per row; bit (x % 32) of
 *     word (y * words + x / 32) is h at (y, x).  K-level head: 2 bits per pixel
 *     (levels 0..3), 16 pixels per word, bits 2(x % 16)..2(x % 16)+1.  Padding
 *     bits past w are zero.
 *   - probability map (optional): float32 [K][h][w] (K = 1 for sigmoid).
 *   - weights: canonical float32 OIHW per layer, layers concatenated, 3x3
 *     kernels; biases float32, concatenated.
 *
 * Random numbers: the noise channel z and the Bernoulli uniforms u come from
 * Philox4x32-10 (Salmon et al., SC'11) with key (seed lo32, seed hi32),
 * counter (g / 4, image, stream, 0) and output lane g % 4, where g = y*w + x
 * and image is the position in the call's image array; stream 0 = z,
 * stream 1 + s = Bernoulli sample s; u = (x >> 8) * 2^-24.
 */
#ifndef HT_H_
#define HT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HT_MAX_LAYERS 40
#define HT_MAX_CHANNELS 64

typedef enum {
    HT_OK = 0,
    HT_ERR_INVALID_ARG = 1,
    HT_ERR_UNSUPPORTED = 2,
    HT_ERR_OOM = 3,
    HT_ERR_CUDA = 4,
    HT_ERR_TIMEOUT = 5,
    HT_ERR_IO = 6         /* checkpoint files: open / read / write failure, corrupt file */
} ht_status;

typedef enum { HT_FP32 = 0, HT_BF16 = 1, HT_FP8_E4M3 = 2, HT_FP16 = 3 } ht_precision;
typedef enum { HT_HEAD_SIGMOID = 0, HT_HEAD_SOFTMAX = 1, HT_HEAD_MULTITONE = 2 } ht_head;
typedef enum { HT_MODE_THRESHOLD = 0, HT_MODE_BERNOULLI = 1 } ht_mode;

/* Policy network (Sec. III "Agents"; Sec. VI-A): n_layers 3x3 convolutions,
 * stride 1, zero padding 1, ReLU between layers, channels[0] == 2 (c and z),
 * channels[n_layers] == 1 with head SIGMOID or MULTITONE, == 4 with head SOFTMAX
 * (4 output levels {0, 1/3, 2/3, 1}).  Hidden widths <= 64.
 * Heads: SIGMOID = binary halftone, 1 bit/px (Sec. III); SOFTMAX = 4 levels,
 * softmax over 4 logits, 2 bits/px; MULTITONE = the multitoning prototype of
 * Sec. VI-E: sigmoid output v, action between the two levels around v among
 * `levels` (2..4) ink levels k / (levels - 1), the upper one with probability
 * equal to v's distance from the lower one over the level spacing (threshold
 * mode: the nearest level), level index packed in 2 bits/px.
 * precision: FP32 = plain CUDA-core form; BF16 / FP8_E4M3 / FP16 = tensor-core form
 * (hidden widths must then all be 64; FP32 accumulation).  Rounding points of the
 * tensor-core forms: layer 1 is evaluated to float32 accuracy (inputs and weights as
 * exact three-part bf16 splits); the inner layers' weights and every hidden
 * activation are stored in the form's format (BF16: bfloat16; FP16: IEEE binary16, the
 * same bytes and tensor rate as BF16 with three more significand bits; FP8_E4M3: e4m3
 * with per-output-channel weight scales and per-layer activation scales, activations
 * rounded to bfloat16 first); the last layer's weights stay float32 (4-logit head:
 * exact as two 16-bit parts).  FP16 is an inference form: training it returns
 * HT_ERR_UNSUPPORTED. */
typedef enum { HT_ARCH_PLAIN = 0, HT_ARCH_RESNET = 1 } ht_arch;

/* arch RESNET: the residual policy of Sec. VI-A.  Layers: a stem convolution
 * 2 -> C with ReLU, then per residual block conv1 (C -> C, ReLU) and conv2
 * (C -> C) with the identity shortcut y = ReLU(x + conv2(ReLU(conv1(x)))), then
 * the output convolution C -> 1 (sigmoid or multitone head).  n_layers = 2 + 2 x
 * blocks; every hidden width C = 32; BF16 tensor-core form only (other
 * precisions return HT_ERR_UNSUPPORTED).  Weights in the same layer order,
 * canonical OIHW. */
typedef struct {
    int n_layers;
    int channels[HT_MAX_LAYERS + 1];
    int head;
    int precision;
    int levels;           /* MULTITONE head: ink levels, 2..4 (ignored otherwise) */
    int arch;             /* HT_ARCH_PLAIN (the 3x3 conv stack above) or HT_ARCH_RESNET */
} ht_policy_desc;

typedef struct {
    const float *contone; /* device, [h][pitch] */
    int h, w, pitch;
} ht_image;

typedef struct ht_policy ht_policy;

/* Create a policy on the current device from host weights / biases (see the
 * layout above).  Copies and packs them; the caller keeps ownership of its
 * arrays.  Errors: INVALID_ARG (shape), UNSUPPORTED (precision / widths),
 * OOM, CUDA. */
ht_status ht_create_policy(const ht_policy_desc *desc, const float *weights_host,
                           const float *biases_host, ht_policy **out);
ht_status ht_destroy_policy(ht_policy *p);

/* Replace the weights from device float32 arrays (same layout) and repack them
 * on `stream` (used after each optimiser step in training). */
ht_status ht_policy_set_weights(ht_policy *p, const float *weights_dev, const float *biases_dev,
                                void *stream);

/* FP8 form only: per-layer static activation scales (host, n_layers values;
 * entry l scales the input activations of layer l, entries 0 and n_layers-1
 * are ignored).  Each hidden layer's input a is stored as e4m3(a / s_l). */
ht_status ht_policy_set_act_scales(ht_policy *p, const float *scales_host, int n);

/* FP8 form: derive the static activation scales from one calibration image
 * (device contone, Philox noise with `seed`): an FP32 forward records each
 * hidden layer's largest activation a_max and sets its consumer's scale to the
 * power of two 2^ceil(log2(a_max / 448)) (448 = largest e4m3 value), then
 * repacks.  Synchronises `stream`; allocates a temporary activation buffer. */
ht_status ht_policy_calibrate(ht_policy *p, const ht_image *img, uint64_t seed, void *stream);

/* Total parameter count and FLOPs per output pixel (2 x MACs). */
int64_t ht_policy_num_params(const ht_policy *p);
int64_t ht_policy_flops_per_px(const ht_policy *p);

/* uint32 words per halftone row for width w and the given head. */
int ht_bits_row_words(int w, int head);

/* One-shot halftoning (Algorithm 1, TEST step; Eq. independent).
 * imgs: host array of n image descriptors (device pixel pointers).
 * mode: HT_MODE_THRESHOLD (h = [p > 0.5]; softmax head: argmax) or
 *       HT_MODE_BERNOULLI (h = [u < p]; softmax head: smallest k with
 *       u < sum_{j<=k} q_j), u from Philox stream 1 with `seed`; z always
 *       from stream 0 with `seed`.
 * out_bits: host array of n device pointers, each h * ht_bits_row_words words.
 * out_prob: NULL or host array of n device pointers (NULL entries allowed),
 *           each float [K][h][w].
 * Images may differ in size (1 <= h, w <= 16384). */
ht_status ht_halftone(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed,
                      uint32_t *const *out_bits, float *const *out_prob, void *stream);

/* Reward options (Eq. final_reward, Sec. V): HVS = normalised Gaussian
 * (sigma_hvs, 2r+1 taps; the Gaussian sigma-2 filter of Sec. VI-B stands in
 * for the Nasanen model), SSIM window = normalised Gaussian (sigma_ssim,
 * 2r+1 taps), contrast k, weight w_s, SSIM constants c1, c2, radius r (<= 7).
 * All windows are "valid" (Sec. VI-A): outputs on (h-2r) x (w-2r). */
typedef struct {
    float sigma_hvs, sigma_ssim, k_contrast, w_s, c1, c2;
    int radius;
    int levels;           /* 2: binary halftones (1 bit/px); 3 or 4: multi-level halftones of the
                             multitoning prototype (Sec. VI-E), 2-bit level index per px, value
                             index / (levels - 1) */
} ht_reward_opts;

/* Fill opts with the paper's defaults: 2.0, 1.5, 2, 0.06, 1e-4, 9e-4, 5, levels 2. */
void ht_reward_opts_default(ht_reward_opts *opts);

/* Reward of n (contone, halftone) pairs (binary, or multi-level with opts->levels > 2).
 * out: device array of 4*n doubles: MSE, SSIM (mean map), CSSIM, R per image.
 * Requires h, w >= 2r + 1. */
ht_status ht_reward(const ht_image *c, const uint32_t *const *bits, int n, const ht_reward_opts *opts,
                    double *out, void *stream);

/* Allocation-free variant of ht_reward (the paper has no counterpart; it is a
 * service for callers that must not allocate device memory while they run, for
 * example a host application whose own allocator has reserved all the device
 * memory it may use, or a streaming loop that cannot accept the device-wide
 * synchronisation cudaMalloc / cudaFree may imply).  Same arguments, results
 * and tolerances as ht_reward, but it calls no cudaMalloc, cudaFree or other
 * allocating routine: its FP64 per-image accumulators live in a file-scope
 * device array of 3 * HT_REWARD_NOALLOC_MAX_IMAGES doubles (24 KiB), held by
 * every GPU that loads the library until the process exits.
 *   - n must be <= HT_REWARD_NOALLOC_MAX_IMAGES, else HT_ERR_INVALID_ARG.
 *   - The first call on a device looks the array's device address up
 *     (cudaGetSymbolAddress, with that device current) and caches it; make that
 *     first call before any stream capture.
 *   - Every call clears and reuses the same array: calls whose work overlaps on
 *     the GPU (e.g. on unordered streams) race and give wrong results. */
#define HT_REWARD_NOALLOC_MAX_IMAGES 1024
ht_status ht_reward_noalloc(const ht_image *c, const uint32_t *const *bits, int n,
                            const ht_reward_opts *opts, double *out, void *stream);

/* Toggle deltas of the local-expectation gradient (Eq. le, Sec. III-C):
 * dR[a] = R(h with h_a = 1) - R(h with h_a = 0) for every pixel a.
 * Multi-level halftones (opts->levels > 2, Sec. VI-E): the two actions of pixel a
 * are the levels lo = floor(v_a (L - 1)) (at most L - 2) and lo + 1 around the
 * policy output v_a, and dR[a] = R(h_a = lo + 1) - R(h_a = lo).
 * v: NULL for binary halftones, else host array of n device pointers to float [h][w].
 * dR: host array of n device pointers, each float [h][w]. */
ht_status ht_toggle_delta(const ht_image *c, const uint32_t *const *bits, const float *const *v, int n,
                          const ht_reward_opts *opts, float *const *dR, void *stream);

/* Anisotropy-suppressing loss of n_patches probability maps q (device float
 * [n_patches][n][n], n a power of two in [8, 1024]) (Eqs. psd, as; Sec. IV).
 * mode 0: sum over rings (width 1, DC excluded) of squared deviations from
 *         the ring mean (Eq. as);
 * mode 1: mean over n_rad radial bins of the variance over n_ang angular bins
 *         of the bin means divided by the squared ring mean.
 * out_loss: device, n_patches doubles.  grad: NULL or device float
 * [n_patches][n][n], receives dL/dq. */
ht_status ht_anisotropy_loss(const float *q, int n_patches, int n, int mode, int n_rad, int n_ang,
                             double *out_loss, float *grad, void *stream);

/* ------------------------------------------------------------------------ */
/* Plans: one ht_halftone call (tensor-core forms) captured into a CUDA graph */
/* and replayed.  The plan owns its workspace and the image table; images,   */
/* output buffers, mode and seed are fixed at creation (the caller may write  */
/* new pixel values into the same contone buffers between launches).  When  */
/* the policy's weights or scales change, the next launch captures again.     */
/* Returns HT_ERR_UNSUPPORTED for FP32 policies.  The policy must outlive the */
/* plan.                                                                      */
/* ------------------------------------------------------------------------ */
typedef struct ht_plan ht_plan;

ht_status ht_plan_create(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed,
                         uint32_t *const *out_bits, float *const *out_prob, ht_plan **out);
ht_status ht_plan_launch(ht_plan *plan, void *stream);
ht_status ht_plan_destroy(ht_plan *plan);

/* ------------------------------------------------------------------------ */
/* Schedule autotuner (tensor-core forms).  Runs the caller's ht_halftone call */
/* (outputs are written) under every candidate conv schedule -- work units of */
/* 8, 6 or 4 rows (one TMEM accumulator block per row), or streaming strips   */
/* of 32, 64 or 128 rows (eight TMEM blocks used as a ring; every input row   */
/* staged once per strip; 64-wide plain architecture) x unit order (row bands */
/* first, column tiles first) x CTA form of the 64 -> 64 layers (one CTA per  */
/* 128-pixel tile, M = 128 MMAs; or, with 8-row units, a CTA pair per 256-    */
/* pixel tile, M = 256 MMAs of tcgen05 cta_group::2, 64-wide plain            */
/* architecture only) -- reps times each after a warm-up, timed with CUDA     */
/* events on `stream`, and keeps the fastest in the policy (used by later     */
/* ht_halftone calls and plans).  results: nullable host array of up to       */
/* max_results entries, *n_results written (18 candidates; 6 for the residual */
/* architecture).  Outputs are bit-identical under every schedule: each output */
/* pixel accumulates in one TMEM column through the same chain of MMAs.        */
/* ------------------------------------------------------------------------ */
#define HT_TUNE_CANDIDATES 18
typedef struct {
    int rows_per_unit;
    int unit_order;
    int cta_pair;             /* 1: 64 -> 64 layers as CTA pairs */
    float ms;                 /* mean time of one call */
} ht_tune_result;

/* Sets the conv schedule directly, e.g. one found by an earlier ht_policy_autotune
 * run: rows_per_unit in [3, 8] (work units) or in [9, 4096] (streaming strips; the
 * 64-wide plain architecture only, else HT_ERR_INVALID_ARG), unit_order 0 or 1,
 * cta_pair 0 or 1 (the pair form is used only where it applies: 8-row units of the
 * 64-wide plain architecture in BF16 or FP8).  A new policy starts at 64-row strips,
 * column tiles first (64, 1, 0); a residual policy at 8-row units (8, 0, 0). */
ht_status ht_policy_set_schedule(ht_policy *p, int rows_per_unit, int unit_order, int cta_pair);

ht_status ht_policy_autotune(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed,
                             uint32_t *const *out_bits, float *const *out_prob, int reps, ht_tune_result *results,
                             int max_results, int *n_results, void *stream);

/* ------------------------------------------------------------------------ */
/* Training (Algorithm 1, TRAIN step).                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int max_crops;        /* B: crops per step */
    int crop_h, crop_w;   /* crop size (all crops the same size) */
    int n_gray;           /* constant-gray patches per step (Sec. IV), may be 0 */
    int gray_n;           /* gray patch side (power of two) */
    int n_samples;        /* S: Bernoulli samples per crop */
    int las_mode;         /* 0 = Eq. (as), 1 = binned form */
    int n_rad, n_ang;     /* binned form */
    float w_a;            /* anisotropy weight (paper: 0.002) */
    ht_reward_opts reward;
    int estimator;        /* HT_EST_LE: local expectation (Eq. le, the paper's choice);
                             HT_EST_COMA: counterfactual baseline (Eq. coma) */
    int ckpt_stride;      /* BF16 form, activation recomputation for large crops: 0 or 1 keeps
                             every hidden activation for the backward; k >= 2 keeps every k-th
                             (and the head's input) and recomputes the others, segment by
                             segment, during the backward (results unchanged) */
} ht_train_desc;

enum { HT_EST_LE = 0, HT_EST_COMA = 1 };

typedef struct ht_train ht_train;

/* Training workspace for policy p.  An FP32 policy trains in FP32 on CUDA cores;
 * a BF16 policy (2 -> 64 x (L-1) -> 1, sigmoid head) trains on the tensor cores:
 * bf16 weights, activations and hidden gradients, FP32 accumulation, FP32
 * gradients of the FP32 master weights.  FP8 and softmax-head policies return
 * HT_ERR_UNSUPPORTED. */
ht_status ht_train_create(ht_policy *p, const ht_train_desc *d, ht_train **out);
ht_status ht_train_destroy(ht_train *t);

/* Forward part of one iteration: policy forward on the crops and the gray
 * patches (levels: host array of n_gray floats), S samples per crop, reward and
 * toggle deltas per sample, L_MARL (Eq. marl, averaged over crops and samples)
 * and w_a * L_AS (averaged over patches).  Keeps what the backward needs.
 * losses_host (host, 4 doubles, written after the call synchronises `stream`):
 * L_total, L_MARL, L_AS, mean reward R.  n may be 0 when the trainer has gray
 * patches: the step then optimises w_a * L_AS alone (L_MARL and R read 0). */
ht_status ht_train_step_fwd(ht_train *t, const ht_image *crops, int n, const float *gray_levels,
                            uint64_t seed, double *losses_host, void *stream);

/* Backward of the last forward: dL_total/dW and dL_total/db (device float
 * arrays in the canonical layout, overwritten).  The crop images passed to the
 * forward are read again here (first-layer input) and must still be valid. */
ht_status ht_train_step_bwd(ht_train *t, float *grad_w, float *grad_b, void *stream);

/* ------------------------------------------------------------------------ */
/* Kernel timing (library's own instrumentation).                            */
/* Between ht_profile_begin and ht_profile_end every hot kernel launch is    */
/* bracketed by CUDA events on the stream it is launched on; end             */
/* synchronises the device and returns per-kernel launch counts and summed    */
/* device time.  out: host array of max entries; *n_out = entries written.   */
/* ------------------------------------------------------------------------ */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} ht_kernel_stat;

ht_status ht_profile_begin(void);
ht_status ht_profile_end(ht_kernel_stat *out, int max, int *n_out);

/* Policy checkpoints, for stopping and resuming a training run (Algorithm 1, TRAIN
 * step, iterated).  Host only: no device memory, stream or CUDA call.  A checkpoint
 * holds the policy descriptor, the canonical float32 weights and biases (the layout
 * above: OIHW per layer, layers concatenated), the FP8 activation scales and the
 * training iteration `step`; the optimiser's state is the caller's.  File format
 * (little-endian): the tag "HTCKPT01", a u32 header length, the header (i32 n_layers,
 * i32 channels[n_layers + 1], i32 head, precision, levels, arch, i64 step,
 * f32 act_scale[n_layers], i64 n_weights, i64 n_biases), f32 weights, f32 biases and a
 * 64-bit FNV-1a checksum of every preceding byte. */
typedef struct {
    ht_policy_desc desc;
    int64_t step;
    int64_t n_weights, n_biases;      /* parameter counts the descriptor implies */
    float act_scale[HT_MAX_LAYERS];
} ht_checkpoint_info;

/* Write a checkpoint.  desc must be one ht_create_policy accepts; weights_host /
 * biases_host hold the counts it implies; act_scales_host (n_layers values) may be
 * NULL (all 1).  The file is written to "<path>.tmp" and renamed over `path`, so an
 * interrupted save leaves the previous file intact.  Errors: INVALID_ARG /
 * UNSUPPORTED (descriptor, null arrays, negative step), IO. */
ht_status ht_checkpoint_save(const char *path, const ht_policy_desc *desc, const float *weights_host,
                             const float *biases_host, const float *act_scales_host, int64_t step);

/* Read a checkpoint into `info`; with weights_host and biases_host both non-NULL also
 * the parameters (capacities in elements: at least info->n_weights / n_biases, else
 * INVALID_ARG).  Both NULL: header only, to size the arrays.  A wrong tag, checksum,
 * descriptor or length returns IO and leaves `info` untouched. */
ht_status ht_checkpoint_load(const char *path, ht_checkpoint_info *info, float *weights_host, int64_t weights_cap,
                             float *biases_host, int64_t biases_cap);

/* Synchronise `stream` and report device-side errors (timeouts, faults). */
ht_status ht_sync(void *stream);

/* Thread-local description of the last error ("" if none). */
const char *ht_last_error(void);

/* Library version string. */
const char *ht_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HT_H_ */
