// api.cu -- the C ABI declared in include/ht.h: argument validation, object
// lifetime, workspaces and dispatch to the kernels of the other sources.
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "ht_internal.cuh"

namespace {
thread_local char g_err[1024] = "";
std::mutex g_flag_mu;
int *g_flags[64] = {nullptr};   // per-device error flag (device memory)
}  // namespace

void ht_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int *ht_device_error_flag()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> g(g_flag_mu);
    if (!g_flags[dev]) {
        int *p = nullptr;
        if (cudaMalloc((void **)&p, 8 * sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, 8 * sizeof(int)) != cudaSuccess) return nullptr;
        g_flags[dev] = p;
    }
    return g_flags[dev];
}

namespace {
struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_ev_pool;
const char *const g_kernel_names[HTK_COUNT] = {"k_first_tc",   "k_conv_tc_bf16", "k_conv_tc_fp8", "k_head_tc",
                                               "k_conv3x3_fp32", "k_head_fp32",  "k_reward",      "k_toggle_delta",
                                               "k_spectrum",   "k_train", "k_first_input", "k_conv_tc_fp16"};

cudaEvent_t pool_event()
{
    if (!g_ev_pool.empty()) {
        cudaEvent_t e = g_ev_pool.back();
        g_ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

static bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

void ht_prof_start(int kid, cudaStream_t s)
{
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_prof_on || capturing(s)) return;
    ProfRec r;
    r.kid = kid;
    r.a = pool_event();
    r.b = pool_event();
    cudaEventRecord(r.a, s);
    g_prof.push_back(r);
}

void ht_prof_stop(cudaStream_t s)
{
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_prof_on || g_prof.empty() || capturing(s)) return;
    cudaEventRecord(g_prof.back().b, s);
}

extern "C" {

ht_status ht_profile_begin(void)
{
    std::lock_guard<std::mutex> g(g_prof_mu);
    for (auto &r : g_prof) {
        g_ev_pool.push_back(r.a);
        g_ev_pool.push_back(r.b);
    }
    g_prof.clear();
    g_prof_on = true;
    return HT_OK;
}

ht_status ht_profile_end(ht_kernel_stat *out, int max, int *n_out)
{
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof_on = false;
    HT_CUDA_TRY(cudaDeviceSynchronize());
    int64_t cnt[HTK_COUNT] = {0};
    double ms[HTK_COUNT] = {0};
    for (auto &r : g_prof) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            cnt[r.kid] += 1;
            ms[r.kid] += t;
        }
        g_ev_pool.push_back(r.a);
        g_ev_pool.push_back(r.b);
    }
    g_prof.clear();
    int n = 0;
    for (int k = 0; k < HTK_COUNT; ++k) {
        if (!cnt[k]) continue;
        if (out && n < max) {
            memset(out[n].name, 0, sizeof(out[n].name));
            strncpy(out[n].name, g_kernel_names[k], sizeof(out[n].name) - 1);
            out[n].launches = cnt[k];
            out[n].total_ms = ms[k];
        }
        ++n;
    }
    if (n_out) *n_out = n < max ? n : max;
    return HT_OK;
}

const char *ht_last_error(void) { return g_err; }
const char *ht_version(void) { return "ht 0.1 (sm_103a)"; }

int ht_bits_row_words(int w, int head)
{
    if (w <= 0) return 0;
    return head == HT_HEAD_SIGMOID ? (w + 31) / 32 : (w + 15) / 16;
}

void ht_reward_opts_default(ht_reward_opts *o)
{
    if (!o) return;
    o->sigma_hvs = 2.0f;
    o->sigma_ssim = 1.5f;
    o->k_contrast = 2.0f;
    o->w_s = 0.06f;
    o->c1 = 0.01f * 0.01f;
    o->c2 = 0.03f * 0.03f;
    o->radius = 5;
    o->levels = 2;
}

static ht_status validate_desc(const ht_policy_desc *d)
{
    HT_CHECK_ARG(d != nullptr, "null policy descriptor");
    HT_CHECK_ARG(d->n_layers >= 2 && d->n_layers <= HT_MAX_LAYERS, "n_layers must be in [2, %d]", HT_MAX_LAYERS);
    HT_CHECK_ARG(d->channels[0] == 2, "channels[0] must be 2 (contone and noise)");
    for (int l = 1; l < d->n_layers; ++l)
        HT_CHECK_ARG(d->channels[l] >= 1 && d->channels[l] <= HT_MAX_CHANNELS, "hidden width %d out of range",
                     d->channels[l]);
    if (d->head == HT_HEAD_SIGMOID) {
        HT_CHECK_ARG(d->channels[d->n_layers] == 1, "sigmoid head needs 1 output channel");
    } else if (d->head == HT_HEAD_MULTITONE) {
        HT_CHECK_ARG(d->channels[d->n_layers] == 1, "multitone head needs 1 output channel");
        HT_CHECK_ARG(d->levels >= 2 && d->levels <= 4, "multitone levels must be in [2, 4]");
    } else if (d->head == HT_HEAD_SOFTMAX) {
        HT_CHECK_ARG(d->channels[d->n_layers] == 4, "softmax head needs 4 output channels");
    } else {
        HT_CHECK_ARG(false, "unknown head %d", d->head);
    }
    HT_CHECK_ARG(d->precision == HT_FP32 || d->precision == HT_BF16 || d->precision == HT_FP8_E4M3 ||
                     d->precision == HT_FP16,
                 "unknown precision %d", d->precision);
    HT_CHECK_ARG(d->arch == HT_ARCH_PLAIN || d->arch == HT_ARCH_RESNET, "unknown arch %d", d->arch);
    if (d->arch == HT_ARCH_RESNET) {
        HT_CHECK_ARG(d->n_layers >= 4 && d->n_layers % 2 == 0, "residual policy: n_layers = 2 + 2 x blocks");
        HT_CHECK_ARG(d->head != HT_HEAD_SOFTMAX, "residual policy: sigmoid-output heads only");
        for (int l = 1; l < d->n_layers; ++l)
            if (d->channels[l] != 32) {
                ht_set_error("residual policy: every hidden width must be 32");
                return HT_ERR_UNSUPPORTED;
            }
        if (d->precision != HT_BF16) {
            ht_set_error("residual policy: BF16 tensor-core form only");
            return HT_ERR_UNSUPPORTED;
        }
        return HT_OK;
    }
    if (d->precision != HT_FP32) {
        if (d->n_layers < 3) {
            ht_set_error("tensor-core forms need at least one 64 -> 64 layer");
            return HT_ERR_UNSUPPORTED;
        }
        for (int l = 1; l < d->n_layers; ++l)
            if (d->channels[l] != 64) {
                ht_set_error("tensor-core forms need every hidden width = 64");
                return HT_ERR_UNSUPPORTED;
            }
    }
    return HT_OK;
}

ht_status ht_create_policy(const ht_policy_desc *desc, const float *weights_host, const float *biases_host,
                           ht_policy **out)
{
    HT_RANGE("ht_create_policy");
    HT_CHECK_ARG(out != nullptr, "null output pointer");
    *out = nullptr;
    ht_status st = validate_desc(desc);
    if (st != HT_OK) return st;
    HT_CHECK_ARG(weights_host && biases_host, "weights and biases are required");
    ht_preload_kernels();
    ht_policy *p = new ht_policy();
    p->L = desc->n_layers;
    memcpy(p->ch, desc->channels, sizeof(p->ch));
    p->head = desc->head;
    p->levels = desc->head == HT_HEAD_MULTITONE ? desc->levels : desc->head == HT_HEAD_SOFTMAX ? 4 : 2;
    p->arch = desc->arch;
    p->width = desc->arch == HT_ARCH_RESNET ? 32 : 64;
    if (desc->arch != HT_ARCH_RESNET) {       // default schedule: 64-row streaming strips, column tiles first
        p->tune_ru = 64;
        p->tune_order = 1;
    }
    p->K = desc->channels[desc->n_layers];
    p->prec = desc->precision;
    cudaGetDevice(&p->device);
    p->n_w = p->n_b = 0;
    for (int l = 0; l < p->L; ++l) {
        p->w_off[l] = p->n_w;
        p->b_off[l] = p->n_b;
        p->n_w += (int64_t)p->ch[l + 1] * p->ch[l] * 9;
        p->n_b += p->ch[l + 1];
        p->act_scale[l] = 1.f;
    }
    cudaError_t e = cudaMalloc((void **)&p->d_w, sizeof(float) * p->n_w);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_b, sizeof(float) * p->n_b);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_w, weights_host, sizeof(float) * p->n_w, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_b, biases_host, sizeof(float) * p->n_b, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        ht_set_error("policy upload: %s", cudaGetErrorString(e));
        ht_destroy_policy(p);
        return e == cudaErrorMemoryAllocation ? HT_ERR_OOM : HT_ERR_CUDA;
    }
    if (p->prec != HT_FP32) {
        st = ht_pack_tc_weights(p, 0);
        if (st != HT_OK) {
            ht_destroy_policy(p);
            return st;
        }
    }
    *out = p;
    return HT_OK;
}

ht_status ht_destroy_policy(ht_policy *p)
{
    if (!p) return HT_OK;
    cudaFree(p->d_w);
    cudaFree(p->d_b);
    cudaFree(p->d_wpack);
    cudaFree(p->d_wpack2);
    cudaFree(p->d_wscale);
    cudaFree(p->d_w1pack);
    cudaFree(p->d_wpack4);
    cudaFree(p->d_ws);
    delete p;
    return HT_OK;
}

ht_status ht_policy_set_weights(ht_policy *p, const float *weights_dev, const float *biases_dev, void *stream)
{
    HT_RANGE("ht_policy_set_weights");
    HT_CHECK_ARG(p && weights_dev && biases_dev, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    HT_CUDA_TRY(cudaMemcpyAsync(p->d_w, weights_dev, sizeof(float) * p->n_w, cudaMemcpyDeviceToDevice, s));
    HT_CUDA_TRY(cudaMemcpyAsync(p->d_b, biases_dev, sizeof(float) * p->n_b, cudaMemcpyDeviceToDevice, s));
    if (p->prec != HT_FP32) return ht_pack_tc_weights(p, s);
    return HT_OK;
}

ht_status ht_policy_set_act_scales(ht_policy *p, const float *scales_host, int n)
{
    HT_CHECK_ARG(p && scales_host, "null argument");
    HT_CHECK_ARG(n == p->L, "expected %d scales", p->L);
    for (int l = 0; l < n; ++l)
        HT_CHECK_ARG(scales_host[l] > 0.f && isfinite(scales_host[l]), "scale %d must be positive", l);
    for (int l = 0; l < n; ++l) p->act_scale[l] = scales_host[l];
    ++p->version;
    return HT_OK;
}

}  // extern "C"

ht_status ht_validate_desc(const ht_policy_desc *d) { return validate_desc(d); }

namespace {
__global__ void k_absmax(const float *__restrict__ a, size_t n, unsigned int *__restrict__ out)
{
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(a[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));   // non-negative floats order as uints
}
}  // namespace

extern "C" {

ht_status ht_policy_calibrate(ht_policy *p, const ht_image *img, uint64_t seed, void *stream)
{
    HT_RANGE("ht_policy_calibrate");
    HT_CHECK_ARG(p && img && img->contone, "null argument");
    HT_CHECK_ARG(img->h >= 1 && img->w >= 1 && img->pitch >= img->w, "bad calibration image");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t px = (size_t)img->h * img->w;
    size_t tot = 0;
    for (int l = 1; l < p->L; ++l) tot += (size_t)p->ch[l] * px;
    float *acts = nullptr, *prob = nullptr;
    uint32_t *bits = nullptr;
    unsigned int *amax = nullptr;
    cudaError_t e = cudaMalloc((void **)&acts, sizeof(float) * tot);
    if (e == cudaSuccess) e = cudaMalloc((void **)&prob, sizeof(float) * px * p->K);
    if (e == cudaSuccess) e = cudaMalloc((void **)&bits, sizeof(uint32_t) * img->h * ht_bits_row_words(img->w, p->head));
    if (e == cudaSuccess) e = cudaMalloc((void **)&amax, sizeof(unsigned int) * HT_MAX_LAYERS);
    ht_status st = e == cudaSuccess ? HT_OK : HT_ERR_OOM;
    unsigned int h_amax[HT_MAX_LAYERS] = {0};
    if (st == HT_OK) {
        float *ap[HT_MAX_LAYERS];
        size_t off = 0;
        for (int l = 0; l + 1 < p->L; ++l) {
            ap[l] = acts + off;
            off += (size_t)p->ch[l + 1] * px;
        }
        st = ht_fwd_fp32_save(p, *img, 0u, seed, ap, prob, bits, s);
        if (st == HT_OK && cudaMemsetAsync(amax, 0, sizeof(unsigned int) * HT_MAX_LAYERS, s) != cudaSuccess)
            st = HT_ERR_CUDA;
        for (int l = 0; st == HT_OK && l + 1 < p->L; ++l) {
            k_absmax<<<256, 256, 0, s>>>(ap[l], (size_t)p->ch[l + 1] * px, amax + l);
            if (cudaGetLastError() != cudaSuccess) st = HT_ERR_CUDA;
        }
        if (st == HT_OK && (cudaMemcpyAsync(h_amax, amax, sizeof(h_amax), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                            cudaStreamSynchronize(s) != cudaSuccess))
            st = HT_ERR_CUDA;
    }
    cudaFree(acts);
    cudaFree(prob);
    cudaFree(bits);
    cudaFree(amax);
    if (st != HT_OK) {
        ht_set_error("calibration failed");
        return st;
    }
    // activation l (output of layer l) is the input of layer l + 1
    for (int l = 0; l + 1 < p->L; ++l) {
        float a;
        memcpy(&a, &h_amax[l], 4);
        const double r = (a > 0.f ? a : 1e-6f) / 448.0;
        p->act_scale[l + 1] = (float)ldexp(1.0, (int)ceil(log2(r)));
    }
    if (p->prec != HT_FP32) return ht_pack_tc_weights(p, s);
    return HT_OK;
}

int64_t ht_policy_num_params(const ht_policy *p) { return p ? p->n_w + p->n_b : 0; }

int64_t ht_policy_flops_per_px(const ht_policy *p)
{
    if (!p) return 0;
    int64_t f = 0;
    for (int l = 0; l < p->L; ++l) f += 2 * 9 * (int64_t)p->ch[l] * p->ch[l + 1];
    return f;
}

}  // extern "C"

ht_status ht_policy_ensure_ws(ht_policy *p, size_t bytes)
{
    if (bytes <= p->ws_bytes) return HT_OK;
    if (p->d_ws) {
        HT_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(p->d_ws);
        p->d_ws = nullptr;
        p->ws_bytes = 0;
    }
    HT_CUDA_TRY(cudaMalloc(&p->d_ws, bytes));
    p->ws_bytes = bytes;
    return HT_OK;
}

extern "C" {

ht_status ht_validate_images(const ht_image *imgs, int n, int min_side)
{
    HT_CHECK_ARG(imgs != nullptr && n >= 1, "need at least one image");
    for (int i = 0; i < n; ++i) {
        HT_CHECK_ARG(imgs[i].contone != nullptr, "image %d: null contone", i);
        HT_CHECK_ARG(imgs[i].h >= min_side && imgs[i].w >= min_side && imgs[i].h <= 16384 && imgs[i].w <= 16384,
                     "image %d: size %dx%d outside [%d, 16384]", i, imgs[i].h, imgs[i].w, min_side);
        HT_CHECK_ARG(imgs[i].pitch >= imgs[i].w, "image %d: pitch < width", i);
    }
    return HT_OK;
}

ht_status ht_halftone(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed, uint32_t *const *out_bits,
                      float *const *out_prob, void *stream)
{
    HT_RANGE("ht_halftone");
    HT_CHECK_ARG(p != nullptr, "null policy");
    ht_status st = ht_validate_images(imgs, n, 1);
    if (st != HT_OK) return st;
    HT_CHECK_ARG(mode == HT_MODE_THRESHOLD || mode == HT_MODE_BERNOULLI, "unknown mode %d", mode);
    HT_CHECK_ARG(out_bits != nullptr, "null output array");
    for (int i = 0; i < n; ++i) HT_CHECK_ARG(out_bits[i] != nullptr, "image %d: null bits pointer", i);
    cudaStream_t s = (cudaStream_t)stream;
    if (p->prec != HT_FP32) {
        st = ht_policy_ensure_ws(p, ht_tc_batch_ws_bytes(p, imgs, n));
        if (st != HT_OK) return st;
        return ht_run_tc_batch(p, imgs, n, mode, seed, out_bits, out_prob, s);
    }
    size_t need = 0;
    for (int i = 0; i < n; ++i) {
        const size_t b = ht_fp32_ws_bytes(p, imgs[i].h, imgs[i].w);
        need = b > need ? b : need;
    }
    st = ht_policy_ensure_ws(p, need);
    if (st != HT_OK) return st;
    for (int i = 0; i < n; ++i) {
        float *prob = out_prob ? out_prob[i] : nullptr;
        const size_t half = ht_fp32_ws_bytes(p, imgs[i].h, imgs[i].w) / 2;
        st = ht_run_fp32(p, imgs[i], (uint32_t)i, mode, seed, out_bits[i], prob, (float *)p->d_ws,
                         (float *)((char *)p->d_ws + half), s);
        if (st != HT_OK) return st;
    }
    return HT_OK;
}

static ht_status validate_call(const ht_policy *p, const ht_image *imgs, int n, int mode, uint32_t *const *out_bits)
{
    HT_CHECK_ARG(p != nullptr, "null policy");
    ht_status st = ht_validate_images(imgs, n, 1);
    if (st != HT_OK) return st;
    HT_CHECK_ARG(mode == HT_MODE_THRESHOLD || mode == HT_MODE_BERNOULLI, "unknown mode %d", mode);
    HT_CHECK_ARG(out_bits != nullptr, "null output array");
    for (int i = 0; i < n; ++i) HT_CHECK_ARG(out_bits[i] != nullptr, "image %d: null bits pointer", i);
    return HT_OK;
}

ht_status ht_plan_create(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed, uint32_t *const *out_bits,
                         float *const *out_prob, ht_plan **out)
{
    HT_RANGE("ht_plan_create");
    HT_CHECK_ARG(out != nullptr, "null output pointer");
    *out = nullptr;
    const ht_status st = validate_call(p, imgs, n, mode, out_bits);
    if (st != HT_OK) return st;
    return ht_plan_create_impl(p, imgs, n, mode, seed, out_bits, out_prob, out);
}

ht_status ht_plan_launch(ht_plan *plan, void *stream)
{
    HT_RANGE("ht_plan_launch");
    HT_CHECK_ARG(plan != nullptr, "null plan");
    return ht_plan_launch_impl(plan, (cudaStream_t)stream);
}

ht_status ht_plan_destroy(ht_plan *plan) { return ht_plan_destroy_impl(plan); }

ht_status ht_policy_set_schedule(ht_policy *p, int rows_per_unit, int unit_order, int cta_pair)
{
    HT_CHECK_ARG(p != nullptr, "null policy");
    HT_CHECK_ARG(rows_per_unit >= 3 && rows_per_unit <= 4096, "rows_per_unit must be in [3, 4096]");
    HT_CHECK_ARG(rows_per_unit <= 8 || p->arch != HT_ARCH_RESNET,
                 "streaming strips (rows_per_unit > 8) need the 64-wide plain architecture");
    HT_CHECK_ARG(unit_order == 0 || unit_order == 1, "unit_order must be 0 or 1");
    HT_CHECK_ARG(cta_pair == 0 || cta_pair == 1, "cta_pair must be 0 or 1");
    p->tune_ru = rows_per_unit;
    p->tune_order = unit_order;
    p->tune_pair = cta_pair;
    return HT_OK;
}

ht_status ht_policy_autotune(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed,
                             uint32_t *const *out_bits, float *const *out_prob, int reps, ht_tune_result *results,
                             int max_results, int *n_results, void *stream)
{
    HT_RANGE("ht_policy_autotune");
    ht_status st = validate_call(p, imgs, n, mode, out_bits);
    if (st != HT_OK) return st;
    HT_CHECK_ARG(reps >= 1 && reps <= 1000, "reps must be in [1, 1000]");
    HT_CHECK_ARG(max_results >= 0 && (results || max_results == 0), "bad results array");
    if (n_results) *n_results = 0;
    if (p->prec == HT_FP32) {
        ht_set_error("the autotuner schedules the tensor-core forms (BF16, FP8)");
        return HT_ERR_UNSUPPORTED;
    }
    st = ht_policy_ensure_ws(p, ht_tc_batch_ws_bytes(p, imgs, n));
    if (st != HT_OK) return st;
    return ht_tc_autotune(p, imgs, n, mode, seed, out_bits, out_prob, reps, results, max_results, n_results,
                          (cudaStream_t)stream);
}

ht_status ht_validate_reward_opts(const ht_reward_opts *o)
{
    HT_CHECK_ARG(o != nullptr, "null reward options");
    HT_CHECK_ARG(o->radius >= 1 && o->radius <= 7, "radius must be in [1, 7]");
    HT_CHECK_ARG(o->levels >= 2 && o->levels <= 4, "levels must be in [2, 4]");
    HT_CHECK_ARG(o->sigma_hvs > 0 && o->sigma_ssim > 0, "window sigmas must be positive");
    return HT_OK;
}

ht_status ht_reward(const ht_image *c, const uint32_t *const *bits, int n, const ht_reward_opts *opts, double *out,
                    void *stream)
{
    HT_RANGE("ht_reward");
    ht_status st = ht_validate_reward_opts(opts);
    if (st != HT_OK) return st;
    st = ht_validate_images(c, n, 2 * opts->radius + 1);
    if (st != HT_OK) return st;
    HT_CHECK_ARG(bits && out, "null argument");
    for (int i = 0; i < n; ++i) HT_CHECK_ARG(bits[i] != nullptr, "image %d: null bits", i);
    return ht_reward_launch(c, bits, n, *opts, out, (cudaStream_t)stream);
}

ht_status ht_toggle_delta(const ht_image *c, const uint32_t *const *bits, const float *const *v, int n,
                          const ht_reward_opts *opts, float *const *dR, void *stream)
{
    HT_RANGE("ht_toggle_delta");
    ht_status st = ht_validate_reward_opts(opts);
    if (st != HT_OK) return st;
    st = ht_validate_images(c, n, 2 * opts->radius + 1);
    if (st != HT_OK) return st;
    HT_CHECK_ARG(bits && dR, "null argument");
    HT_CHECK_ARG(opts->levels == 2 || v, "multi-level toggle deltas need the policy outputs v");
    for (int i = 0; i < n; ++i)
        HT_CHECK_ARG(bits[i] && dR[i] && (opts->levels == 2 || v[i]), "image %d: null pointer", i);
    const size_t need = ht_toggle_scratch_floats_batch(c, n, opts->radius);
    cudaStream_t s = (cudaStream_t)stream;
    float *scratch = nullptr;
    HT_CUDA_TRY(cudaMallocAsync((void **)&scratch, need * sizeof(float), s));
    st = ht_toggle_launch(c, bits, v, n, *opts, dR, scratch, need, s);
    cudaFreeAsync(scratch, s);
    return st;
}

ht_status ht_anisotropy_loss(const float *q, int n_patches, int n, int mode, int n_rad, int n_ang, double *out_loss,
                             float *grad, void *stream)
{
    HT_RANGE("ht_anisotropy_loss");
    HT_CHECK_ARG(q && out_loss, "null argument");
    HT_CHECK_ARG(n_patches >= 1, "need at least one patch");
    HT_CHECK_ARG(n >= 8 && n <= 1024 && (n & (n - 1)) == 0, "n must be a power of two in [8, 1024]");
    HT_CHECK_ARG(mode == 0 || mode == 1, "mode must be 0 or 1");
    if (mode == 1) HT_CHECK_ARG(n_rad >= 1 && n_rad <= 256 && n_ang >= 2 && n_ang <= 64, "bad bin counts");
    else {
        n_rad = 1;
        n_ang = 1;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = ht_las_scratch_bytes(n_patches, n, n_rad, n_ang);
    void *scratch = nullptr;
    HT_CUDA_TRY(cudaMallocAsync(&scratch, bytes, s));
    ht_status st = ht_las_launch(q, n_patches, n, mode, n_rad, n_ang, out_loss, grad, scratch, bytes, s);
    cudaFreeAsync(scratch, s);
    return st;
}

ht_status ht_sync(void *stream)
{
    HT_RANGE("ht_sync");
    HT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int *flag = ht_device_error_flag();
    if (!flag) return HT_ERR_CUDA;
    int v[8];
    HT_CUDA_TRY(cudaMemcpy(v, flag, sizeof(v), cudaMemcpyDeviceToHost));
    if (v[0] != 0) {
        cudaMemset(flag, 0, sizeof(v));
        unsigned long long el;
        memcpy(&el, v + 6, sizeof(el));
        ht_set_error("device-side wait expired (error %d): barrier at shared 0x%x, block %d of %d threads, warp %d, "
                     "%d polls, %.3f s",
                     v[0], (unsigned)v[2], v[4], (unsigned)v[3] >> 16, v[3] & 0xFFFF, v[5], (double)el * 1e-9);
        return (ht_status)v[0];
    }
    return HT_OK;
}

}  // extern "C"

void ht_preload_kernels()
{
    static std::once_flag once;
    std::call_once(once, [] {
        ht_preload_conv_tc();
        ht_preload_conv_fp32();
        ht_preload_reward();
        ht_preload_spectrum();
        ht_preload_train();
        ht_preload_train_tc();
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, k_absmax);
        cudaGetLastError();
    });
}
