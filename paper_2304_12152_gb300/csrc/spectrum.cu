// spectrum.cu -- periodogram of constant-gray probability maps and the
// anisotropy-suppressing loss with its gradient (Eqs. psd, rapsd, anis, as;
// Sec. IV, probability-map proxy; Algorithm 1 TRAIN step).
//
//   F = DFT2(q), P(f) = |F(f)|^2 / N                         (Eq. psd)
//   mode 0 (Eq. as): rings of width 1 (rho = round(|f|)), DC excluded, rings
//     with < 2 samples skipped:  L = sum_rho sum_{f in rho} (P(f) - Pbar_rho)^2,
//     dL/dP(f) = 2 (P(f) - Pbar_rho) (the ring-mean term cancels).
//   mode 1 (binned): n_rad radial x n_ang angular bins over 0 < |f| < n/2;
//     per radial bin A = 1/(K-1) sum_k (a_k - m)^2 / m^2 (a_k angular-bin means,
//     m the radial-bin mean, K non-empty angular bins); L = mean of A.
//   dL/dq(x) = (2/N) Re sum_f G(f) F(f) e^{+2 pi i f.x / n},  G = dL/dP.
//
// The 2-D DFT is a radix-2 FFT over rows then columns, one CTA per line with
// the line in shared memory; binning accumulates per-CTA in shared memory
// (FP64 sums) and adds each bin to global memory once per CTA.
#include "ht_internal.cuh"

namespace {

__device__ __forceinline__ int bitrev(int i, int logn) { return (int)(__brev((unsigned)i) >> (32 - logn)); }

// In-place radix-2 FFT of one line held in shared memory (n complex values).
__device__ void fft_line(float2 *s, int n, int logn, float sign)
{
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1;
        for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
            const int grp = t / half, k = t % half;
            const int i = grp * len + k, j = i + half;
            float sn, cs;
            sincospif(sign * 2.0f * (float)k / (float)len, &sn, &cs);
            const float2 a = s[i], b = s[j];
            const float2 bw = make_float2(b.x * cs - b.y * sn, b.x * sn + b.y * cs);
            s[i] = make_float2(a.x + bw.x, a.y + bw.y);
            s[j] = make_float2(a.x - bw.x, a.y - bw.y);
        }
        __syncthreads();
    }
}

// rows: in real (q) or complex (C); out complex C.  grid (n, patches)
__global__ void k_fft_rows(const float *__restrict__ qr, const float2 *__restrict__ qc, float2 *__restrict__ out,
                           int n, int logn, float sign, float *__restrict__ real_out, float real_scale)
{
    extern __shared__ float2 s[];
    const size_t base = ((size_t)blockIdx.y * n + blockIdx.x) * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 v = qr ? make_float2(qr[base + i], 0.f) : qc[base + i];
        s[bitrev(i, logn)] = v;
    }
    __syncthreads();
    fft_line(s, n, logn, sign);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (real_out) real_out[base + i] = s[i].x * real_scale;
        else out[base + i] = s[i];
    }
}

// columns, in place.  grid (n, patches)
__global__ void k_fft_cols(float2 *__restrict__ C, int n, int logn, float sign)
{
    extern __shared__ float2 s[];
    const size_t base = (size_t)blockIdx.y * n * n + blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[bitrev(i, logn)] = C[base + (size_t)i * n];
    __syncthreads();
    fft_line(s, n, logn, sign);
    for (int i = threadIdx.x; i < n; i += blockDim.x) C[base + (size_t)i * n] = s[i];
}

__device__ __forceinline__ int centred(int k, int n) { return k < n / 2 ? k : k - n; }

// Bin of frequency index (a, b); -1 if the sample takes no part.
__device__ __forceinline__ int bin_of(int a, int b, int n, int mode, int n_rad, int n_ang)
{
    const int u = centred(a, n), v = centred(b, n);
    const int m2 = u * u + v * v;
    if (mode == 0) {
        if (m2 == 0) return -1;
        return (int)floor(sqrt((double)m2) + 0.5);      // no ties: sqrt(int) never ends in .5
    }
    const double half = (double)(n / 2);
    const double r = sqrt((double)m2);
    if (m2 == 0 || r >= half) return -1;
    int br = (int)floor(r / half * n_rad);
    if (br >= n_rad) br = n_rad - 1;
    int bt;
    if ((n_ang % 4) == 0 && (u == 0 || v == 0 || u == v || u == -v)) {
        // directions on a bin edge (0, 45, 90, 135 degrees) open their bin
        bt = u == 0 ? 0 : v == 0 ? n_ang / 2 : u == v ? n_ang / 4 : 3 * n_ang / 4;
    } else {
        double th = atan2((double)u, (double)v);
        if (th < 0) th += M_PI;
        if (th >= M_PI) th -= M_PI;
        bt = (int)floor(th / M_PI * n_ang);
        if (bt >= n_ang) bt = n_ang - 1;
    }
    return br * n_ang + bt;
}

// grid (ceil(n*n/256), patches); bins: sums[patch][nb], cnt[patch][nb]
__global__ void k_bin_accum(const float2 *__restrict__ C, int n, int mode, int n_rad, int n_ang, int nb,
                            double *__restrict__ sums, int *__restrict__ cnt)
{
    extern __shared__ unsigned char smem[];
    double *s_sum = (double *)smem;
    int *s_cnt = (int *)(s_sum + nb);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        s_sum[i] = 0.0;
        s_cnt[i] = 0;
    }
    __syncthreads();
    const size_t N = (size_t)n * n;
    const size_t f = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f < N) {
        const int a = (int)(f / n), b = (int)(f % n);
        const int k = bin_of(a, b, n, mode, n_rad, n_ang);
        if (k >= 0) {
            const float2 F = C[(size_t)blockIdx.y * N + f];
            const double P = ((double)F.x * F.x + (double)F.y * F.y) / (double)N;
            atomicAdd(&s_sum[k], P);
            atomicAdd(&s_cnt[k], 1);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        if (s_cnt[i]) {
            atomicAdd(&sums[(size_t)blockIdx.y * nb + i], s_sum[i]);
            atomicAdd(&cnt[(size_t)blockIdx.y * nb + i], s_cnt[i]);
        }
    }
}

// one CTA per patch: per-bin coefficients for G(f) and (mode 1) the loss.
// coef[patch][nb]: mode 0 -> ring mean (NaN when the ring is skipped);
//                  mode 1 -> dL/da_k / n_k ; coefm[patch][n_rad] -> dL/dm / n_rho
// Mode 1: one warp per radial bin (lanes over angular bins), then the loss as an
// ordered sum over radial bins by thread 0.
constexpr int FIN_MAX_RAD = 256;                 // largest n_rad the entry points accept
__global__ void __launch_bounds__(1024) k_bin_finalize(const double *__restrict__ sums, const int *__restrict__ cnt,
                                                       int mode, int n_rad, int n_ang, int nb,
                                                       double *__restrict__ coef, double *__restrict__ coefm,
                                                       double *__restrict__ loss)
{
    const size_t pb = (size_t)blockIdx.x * nb;
    if (mode == 0) {
        for (int i = threadIdx.x; i < nb; i += blockDim.x)
            coef[pb + i] = cnt[pb + i] >= 2 ? sums[pb + i] / cnt[pb + i] : (double)NAN;
        return;
    }
    __shared__ int s_used[FIN_MAX_RAD];
    __shared__ double s_term[FIN_MAX_RAD];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // per radial bin: total, count, occupied angular bins
    for (int br = warp; br < n_rad; br += nw) {
        double tot = 0.0;
        int c = 0, K = 0;
        for (int bt = lane; bt < n_ang; bt += 32) {
            tot += sums[pb + br * n_ang + bt];
            c += cnt[pb + br * n_ang + bt];
            K += cnt[pb + br * n_ang + bt] > 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
            K += __shfl_xor_sync(0xffffffffu, K, o);
        }
        if (lane == 0) s_used[br] = K >= 2 ? 1 : 0;
    }
    __syncthreads();
    int n_used = 0;
    for (int br = 0; br < n_rad; ++br) n_used += s_used[br];
    for (int br = warp; br < n_rad; br += nw) {
        double tot = 0.0;
        int c = 0, K = 0;
        for (int bt = lane; bt < n_ang; bt += 32) {
            tot += sums[pb + br * n_ang + bt];
            c += cnt[pb + br * n_ang + bt];
            K += cnt[pb + br * n_ang + bt] > 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
            K += __shfl_xor_sync(0xffffffffu, K, o);
        }
        if (K < 2) {
            for (int bt = lane; bt < n_ang; bt += 32) coef[pb + br * n_ang + bt] = 0.0;
            if (lane == 0) {
                coefm[(size_t)blockIdx.x * n_rad + br] = 0.0;
                s_term[br] = 0.0;
            }
            continue;
        }
        const double m = tot / c, im = 1.0 / m, iK1 = 1.0 / (K - 1), iu = 1.0 / n_used;
        double A = 0.0, dm = 0.0;
        for (int bt = lane; bt < n_ang; bt += 32) {
            const int j = br * n_ang + bt;
            const int cj = cnt[pb + j];
            double cf = 0.0;
            if (cj > 0) {
                const double ak = sums[pb + j] / cj, d = (ak - m) * im;   // (a_k - m) / m
                A += d * d;
                cf = 2.0 * d * im * iK1 / cj * iu;
                dm += (-2.0 * d * im - 2.0 * d * d * im) * iK1;
            }
            coef[pb + j] = cf;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            A += __shfl_xor_sync(0xffffffffu, A, o);
            dm += __shfl_xor_sync(0xffffffffu, dm, o);
        }
        if (lane == 0) {
            coefm[(size_t)blockIdx.x * n_rad + br] = dm / c * iu;
            s_term[br] = A * iK1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double L = 0.0;
        for (int br = 0; br < n_rad; ++br) L += s_term[br];
        loss[blockIdx.x] = n_used > 0 ? L / n_used : 0.0;
    }
}

// G(f) F(f) into C (in place); mode 0 also accumulates the loss.
__global__ void k_apply_G(float2 *__restrict__ C, int n, int mode, int n_rad, int n_ang, int nb,
                          const double *__restrict__ coef, const double *__restrict__ coefm, double *__restrict__ loss,
                          int want_grad)
{
    const size_t N = (size_t)n * n;
    const size_t f = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double contrib = 0.0;
    if (f < N) {
        const int a = (int)(f / n), b = (int)(f % n);
        const int k = bin_of(a, b, n, mode, n_rad, n_ang);
        const size_t idx = (size_t)blockIdx.y * N + f;
        const float2 F = C[idx];
        double G = 0.0;
        if (k >= 0) {
            if (mode == 0) {
                const double mean = coef[(size_t)blockIdx.y * nb + k];
                if (!isnan(mean)) {
                    const double P = ((double)F.x * F.x + (double)F.y * F.y) / (double)N;
                    const double d = P - mean;
                    contrib = d * d;
                    G = 2.0 * d;
                }
            } else {
                G = coef[(size_t)blockIdx.y * nb + k] + coefm[(size_t)blockIdx.y * n_rad + k / n_ang];
            }
        }
        if (want_grad) C[idx] = make_float2((float)(G * F.x), (float)(G * F.y));
    }
    if (mode == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
        if ((threadIdx.x & 31) == 0 && contrib != 0.0) atomicAdd(&loss[blockIdx.y], contrib);
    }
}

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace

size_t ht_las_scratch_bytes(int n_patches, int n, int n_rad, int n_ang)
{
    const int n_rings = (int)lround(sqrt(2.0) * (n / 2)) + 2;
    const int nb = n_rings > n_rad * n_ang ? n_rings : n_rad * n_ang;
    size_t b = (size_t)n_patches * n * n * sizeof(float2);
    b += (size_t)n_patches * nb * (sizeof(double) * 2 + sizeof(int)) + (size_t)n_patches * n_rad * sizeof(double);
    return b + 1024;
}

ht_status ht_las_launch(const float *q, int n_patches, int n, int mode, int n_rad, int n_ang, double *out_loss,
                        float *grad, void *scratch, size_t scratch_bytes, cudaStream_t s)
{
    const int logn = ilog2(n);
    const int n_rings = (int)lround(sqrt(2.0) * (n / 2)) + 2;
    const int nb = mode == 0 ? n_rings : n_rad * n_ang;
    if (mode == 1 && (n_rad < 1 || n_rad > FIN_MAX_RAD)) {
        ht_set_error("n_rad out of range");
        return HT_ERR_INVALID_ARG;
    }
    if (scratch_bytes < ht_las_scratch_bytes(n_patches, n, n_rad, n_ang)) {
        ht_set_error("spectrum scratch too small");
        return HT_ERR_INVALID_ARG;
    }
    char *p = (char *)scratch;
    float2 *C = (float2 *)p;
    p += (size_t)n_patches * n * n * sizeof(float2);
    double *sums = (double *)p;
    p += (size_t)n_patches * nb * sizeof(double);
    double *coef = (double *)p;
    p += (size_t)n_patches * nb * sizeof(double);
    double *coefm = (double *)p;
    p += (size_t)n_patches * n_rad * sizeof(double);
    int *cnt = (int *)p;

    HT_CUDA_TRY(cudaMemsetAsync(sums, 0, (size_t)n_patches * nb * sizeof(double), s));
    HT_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)n_patches * nb * sizeof(int), s));
    HT_CUDA_TRY(cudaMemsetAsync(out_loss, 0, (size_t)n_patches * sizeof(double), s));
    const int tpb = n / 2 < 32 ? 32 : (n / 2 > 512 ? 512 : n / 2);
    const size_t line_smem = (size_t)n * sizeof(float2);
    k_fft_rows<<<dim3(n, n_patches), tpb, line_smem, s>>>(q, nullptr, C, n, logn, -1.f, nullptr, 0.f);
    HT_LAUNCH_CHECK();
    k_fft_cols<<<dim3(n, n_patches), tpb, line_smem, s>>>(C, n, logn, -1.f);
    HT_LAUNCH_CHECK();
    const unsigned nblk = (unsigned)(((size_t)n * n + 255) / 256);
    const size_t bin_smem = (size_t)nb * (sizeof(double) + sizeof(int));
    k_bin_accum<<<dim3(nblk, n_patches), 256, bin_smem, s>>>(C, n, mode, n_rad, n_ang, nb, sums, cnt);
    HT_LAUNCH_CHECK();
    k_bin_finalize<<<n_patches, 1024, 0, s>>>(sums, cnt, mode, n_rad, n_ang, nb, coef, coefm, out_loss);
    HT_LAUNCH_CHECK();
    k_apply_G<<<dim3(nblk, n_patches), 256, 0, s>>>(C, n, mode, n_rad, n_ang, nb, coef, coefm, out_loss,
                                                    grad != nullptr);
    HT_LAUNCH_CHECK();
    if (grad) {
        k_fft_cols<<<dim3(n, n_patches), tpb, line_smem, s>>>(C, n, logn, +1.f);
        HT_LAUNCH_CHECK();
        k_fft_rows<<<dim3(n, n_patches), tpb, line_smem, s>>>(nullptr, C, nullptr, n, logn, +1.f, grad,
                                                              2.0f / ((float)n * (float)n));
        HT_LAUNCH_CHECK();
    }
    return HT_OK;
}

void ht_preload_spectrum()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_fft_rows);
    cudaFuncGetAttributes(&fa, k_fft_cols);
    cudaFuncGetAttributes(&fa, k_bin_accum);
    cudaFuncGetAttributes(&fa, k_bin_finalize);
    cudaFuncGetAttributes(&fa, k_apply_G);
}
