// reward.cu -- reward R = -MSE(HVS(h), HVS(c)) + w_s CSSIM(h, c) and the toggle
// deltas of the local-expectation gradient.
//
// Reward (Eq. reward, Eq. final_reward, Eq. cssim and the contrast map of
// Sec. V): every window is a normalised Gaussian, applied "valid" (no padding,
// Sec. VI-A).  A 2-D normalised Gaussian is the outer product of the
// normalised 1-D Gaussian, so each window sum runs as a row pass then a column
// pass over a shared-memory tile.  Five window sums per output:
//   HVS(h - c)      -> e = HVS(h) - HVS(c)
//   W(h)            -> mu_h; var_h = mu_h - mu_h^2 (h is binary, h^2 = h)
//   W(c'), W(c'^2)  -> mu_c, var_c   (c' = c - c_ref, c_ref a per-tile constant
//                                     that removes the cancellation in E[c^2]-mu^2)
//   W(h c')         -> cov = E[h c'] - mu_h mu_c'
// SSIM_j = (2 mu_h mu_c + C1)(2 cov + C2) / ((mu_h^2 + mu_c^2 + C1)(var_h + var_c + C2)),
// sigma_j = k sqrt(var_c), CSSIM term = sigma_j SSIM_j + 1 - sigma_j.
// Per-image sums are reduced in FP64 (warp shuffles, then one atomic per block).
//
// Toggle deltas (Eq. le, Eq. marl; Sec. III-C): flipping pixel a by
// delta = 1 - 2 h_a only changes the window sums of the outputs j whose window
// contains a, by delta * g(a - j) (HVS) and delta * w(a - j) (SSIM window):
//   e_j'    = e_j + delta g
//   mu_h'   = mu_h + delta w,   var_h' = mu_h' - mu_h'^2
//   cov'    = cov + delta w (c_a - mu_c)
// so dR_a = R(h_a = 1) - R(h_a = 0) = (1/M) sum_j [ -(2 g e_j + delta g^2)
//            + delta w_s sigma_j (SSIM_j' - SSIM_j) ]  (exact, no approximation).
#include <mutex>

#include "ht_internal.cuh"

namespace {

constexpr int MAXR = 7;
constexpr int RT = 32;                 // reward tile: 32 x 32 valid outputs
constexpr int NQ = 5;

struct Win {
    float g[2 * MAXR + 1];             // HVS 1-D taps (normalised)
    float w[2 * MAXR + 1];             // SSIM window 1-D taps (normalised)
    int r;
    float c1, c2, k, ws;
};

// Up to RW_MAXB images per launch, passed in the kernel parameter (blockIdx.z =
// image); grid x / y cover the largest image, blocks past an image's extent exit.
constexpr int RW_MAXB = 32;
struct RwImg {
    const float *c;
    const uint32_t *bits;     // 1 bit/px (binary) or a 2-bit level index/px (multitone)
    float *maps;              // toggle deltas: NMAP(_LV) moment maps of this image
    float *dR;                // toggle deltas: output
    double *acc;              // reward: 3 FP64 accumulators
    const float *v;           // multitone toggle deltas: the policy output v, [H][W]
    int cpitch, H, W, words;
    int levels;               // 2 binary, else ink levels of the multitone prototype
};
struct RwBatch {
    RwImg im[RW_MAXB];
};

__device__ __forceinline__ float hbit(const uint32_t *bits, int words, int y, int x)
{
    return (float)((bits[(size_t)y * words + (x >> 5)] >> (x & 31)) & 1u);
}
__device__ __forceinline__ int hlevel(const uint32_t *bits, int words, int y, int x)
{
    return (int)((bits[(size_t)y * words + (x >> 4)] >> (2 * (x & 15))) & 3u);
}
// halftone value of pixel (y, x): the bit (binary) or level index / (L - 1) (multitone)
template <bool LV>
__device__ __forceinline__ float hval(const RwImg &I, int y, int x)
{
    if constexpr (LV) return (float)hlevel(I.bits, I.words, y, x) / (float)(I.levels - 1);
    else return hbit(I.bits, I.words, y, x);
}

// Computes the window sums for a 32x32 tile of valid outputs.  Returns, for the
// calling thread's outputs (rows ty, ty+8, ty+16, ty+24; column tx), the
// per-output quantities through the callback-free arrays.  Multi-level
// halftones (LV) add the sixth sum W(h^2) (h^2 != h); its row pass runs after
// the first five, into the contone tile's space (dead by then).
struct Moments {
    float e, muh, muc, varc, cov, eh2;
};

template <bool LV>
__device__ void tile_moments(const RwImg &I, const Win &wn, int vy0, int vx0, float (*s_h)[RT + 2 * MAXR],
                             float (*s_c)[RT + 2 * MAXR], float (*s_row)[RT + 2 * MAXR][RT], Moments out[4],
                             bool valid[4])
{
    const float *__restrict__ c = I.c;
    const int cpitch = I.cpitch, H = I.H, W = I.W;
    const int r = wn.r, span = RT + 2 * r;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const float cref = c[(size_t)min(vy0 + r, H - 1) * cpitch + min(vx0 + r, W - 1)];
    constexpr int MAXSPAN = RT + 2 * MAXR, NPER = (MAXSPAN * MAXSPAN + 255) / 256;
    float hvs[NPER], cvs[NPER];
#pragma unroll
    for (int k = 0; k < NPER; ++k) {          // loads first (one memory latency), then the shared stores
        const int i = tid + 256 * k;
        const int yy = i / span, xx = i % span;
        const int gy = vy0 + yy, gx = vx0 + xx;       // image coords of tile input
        hvs[k] = 0.f;
        cvs[k] = 0.f;
        if (i < span * span && gy < H && gx < W) {
            hvs[k] = hval<LV>(I, gy, gx);
            cvs[k] = __ldg(c + (size_t)gy * cpitch + gx) - cref;
        }
    }
#pragma unroll
    for (int k = 0; k < NPER; ++k) {
        const int i = tid + 256 * k;
        if (i < span * span) {
            s_h[i / span][i % span] = hvs[k];
            s_c[i / span][i % span] = cvs[k];
        }
    }
    __syncthreads();
    // row pass: s_row[q][yy][x] for yy in [0, span), x in [0, 32)
    for (int yy = ty; yy < span; yy += 8) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
        for (int k = 0; k <= 2 * r; ++k) {
            const float hv = s_h[yy][tx + k], cv = s_c[yy][tx + k];
            a0 = fmaf(wn.g[k], hv - (cv + cref), a0);   // h - c (cv holds c - c_ref)
            a1 = fmaf(wn.w[k], hv, a1);
            a2 = fmaf(wn.w[k], cv, a2);
            a3 = fmaf(wn.w[k], cv * cv, a3);
            a4 = fmaf(wn.w[k], hv * cv, a4);
        }
        s_row[0][yy][tx] = a0;
        s_row[1][yy][tx] = a1;
        s_row[2][yy][tx] = a2;
        s_row[3][yy][tx] = a3;
        s_row[4][yy][tx] = a4;
    }
    __syncthreads();
    float(*s_h2)[RT] = reinterpret_cast<float(*)[RT]>(&s_c[0][0]);
    if constexpr (LV) {
        for (int yy = ty; yy < span; yy += 8) {
            float a5 = 0.f;
            for (int k = 0; k <= 2 * r; ++k) {
                const float hv = s_h[yy][tx + k];
                a5 = fmaf(wn.w[k], hv * hv, a5);
            }
            s_h2[yy][tx] = a5;
        }
        __syncthreads();
    }
    const int VH = H - 2 * r, VW = W - 2 * r;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int oy = ty + 8 * t;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
        for (int k = 0; k <= 2 * r; ++k) {
            a0 = fmaf(wn.g[k], s_row[0][oy + k][tx], a0);
            a1 = fmaf(wn.w[k], s_row[1][oy + k][tx], a1);
            a2 = fmaf(wn.w[k], s_row[2][oy + k][tx], a2);
            a3 = fmaf(wn.w[k], s_row[3][oy + k][tx], a3);
            a4 = fmaf(wn.w[k], s_row[4][oy + k][tx], a4);
        }
        Moments m;
        m.e = a0;
        m.muh = a1;
        m.muc = a2 + cref;
        m.varc = fmaxf(a3 - a2 * a2, 0.f);
        m.cov = a4 - a1 * a2;
        m.eh2 = a1;                                      // binary: h^2 = h
        if constexpr (LV) {
            float a5 = 0.f;
            for (int k = 0; k <= 2 * r; ++k) a5 = fmaf(wn.w[k], s_h2[oy + k][tx], a5);
            m.eh2 = a5;
        }
        out[t] = m;
        valid[t] = (vy0 + oy < VH) && (vx0 + tx < VW);
    }
}

__device__ __forceinline__ float ssim_of(float muh, float muc, float varh, float varc, float cov, float c1, float c2)
{
    return ((2.f * muh * muc + c1) * (2.f * cov + c2)) / ((muh * muh + muc * muc + c1) * (varh + varc + c2));
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool LV>
__global__ void __launch_bounds__(256) k_reward_tiles(const __grid_constant__ RwBatch B, const Win wn)
{
    __shared__ float s_h[RT + 2 * MAXR][RT + 2 * MAXR];
    __shared__ float s_c[RT + 2 * MAXR][RT + 2 * MAXR];
    __shared__ float s_row[NQ][RT + 2 * MAXR][RT];
    __shared__ double s_red[3][8];
    const RwImg &I = B.im[blockIdx.z];
    if ((int)blockIdx.y * RT >= I.H - 2 * wn.r || (int)blockIdx.x * RT >= I.W - 2 * wn.r) return;
    double *acc = I.acc;
    Moments m[4];
    bool valid[4];
    tile_moments<LV>(I, wn, blockIdx.y * RT, blockIdx.x * RT, s_h, s_c, s_row, m, valid);
    double se = 0.0, ss = 0.0, sc = 0.0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (!valid[t]) continue;
        const float varh = fmaxf(m[t].eh2 - m[t].muh * m[t].muh, 0.f);
        const float s = ssim_of(m[t].muh, m[t].muc, varh, m[t].varc, m[t].cov, wn.c1, wn.c2);
        const float sig = wn.k * sqrtf(m[t].varc);
        se += (double)m[t].e * (double)m[t].e;
        ss += (double)s;
        sc += (double)(sig * s + (1.f - sig));
    }
    se = warp_sum(se);
    ss = warp_sum(ss);
    sc = warp_sum(sc);
    const int warp = threadIdx.y, lane = threadIdx.x;
    if (lane == 0) {
        s_red[0][warp] = se;
        s_red[1][warp] = ss;
        s_red[2][warp] = sc;
    }
    __syncthreads();
    if (warp == 0 && lane < 3) {
        double v = 0.0;
        for (int i = 0; i < 8; ++i) v += s_red[lane][i];
        atomicAdd(&acc[lane], v);
    }
}

__global__ void k_reward_finalize(const double *__restrict__ acc, int n, const double *__restrict__ inv_m, float ws,
                                  double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double mse = acc[3 * i] * inv_m[i], ssim = acc[3 * i + 1] * inv_m[i], cssim = acc[3 * i + 2] * inv_m[i];
    out[4 * i + 0] = mse;
    out[4 * i + 1] = ssim;
    out[4 * i + 2] = cssim;
    out[4 * i + 3] = -mse + (double)ws * cssim;
}

// Per-output maps for the toggle deltas, valid coords [VH][VW]:
// 0 e, 1 mu_h, 2 mu_c, 3 var_c + C2, 4 cov, 5 sigma, 6 SSIM (+ 7 E[h^2] for
// multi-level halftones).
constexpr int NMAP = 7, NMAP_LV = 8;

template <bool LV>
__global__ void __launch_bounds__(256) k_moment_maps(const __grid_constant__ RwBatch B, const Win wn)
{
    __shared__ float s_h[RT + 2 * MAXR][RT + 2 * MAXR];
    __shared__ float s_c[RT + 2 * MAXR][RT + 2 * MAXR];
    __shared__ float s_row[NQ][RT + 2 * MAXR][RT];
    const RwImg &I = B.im[blockIdx.z];
    const int VH = I.H - 2 * wn.r, VW = I.W - 2 * wn.r;
    const int vy0 = blockIdx.y * RT, vx0 = blockIdx.x * RT;
    if (vy0 >= VH || vx0 >= VW) return;
    float *maps = I.maps;
    Moments m[4];
    bool valid[4];
    tile_moments<LV>(I, wn, vy0, vx0, s_h, s_c, s_row, m, valid);
    const size_t plane = (size_t)VH * VW;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (!valid[t]) continue;
        const size_t k = (size_t)(vy0 + threadIdx.y + 8 * t) * VW + vx0 + threadIdx.x;
        const float varh = fmaxf(m[t].eh2 - m[t].muh * m[t].muh, 0.f);
        if constexpr (LV) maps[7 * plane + k] = m[t].eh2;
        maps[0 * plane + k] = m[t].e;
        maps[1 * plane + k] = m[t].muh;
        maps[2 * plane + k] = m[t].muc;
        maps[3 * plane + k] = m[t].varc + wn.c2;
        maps[4 * plane + k] = m[t].cov;
        maps[5 * plane + k] = wn.k * sqrtf(m[t].varc);
        maps[6 * plane + k] = ssim_of(m[t].muh, m[t].muc, varh, m[t].varc, m[t].cov, wn.c1, wn.c2);
    }
}

constexpr int DTX = 32, DTY = 8;

// Multi-level halftones (LV, the multitoning prototype of Sec. VI-E): the two
// actions of pixel a are the levels lo = floor(v_a (L - 1)) (at most L - 2) and
// lo + 1 around the policy output v_a; dR_a = R(h_a = hi) - R(h_a = lo), as the
// difference of the moment-shift updates for t = (hi - cur) / (L - 1) and
// t = (lo - cur) / (L - 1) (one of them is 0 when the current level is one of
// the pair):  e' = e + t g, mu_h' = mu_h + t w, E[h^2]' = E[h^2] + ((h_a + t)^2 -
// h_a^2) w, cov' = cov + t w (c_a - mu_c).
template <bool LV>
__global__ void __launch_bounds__(DTX *DTY, 3) k_toggle_delta(const __grid_constant__ RwBatch B, const Win wn)
{
    constexpr int SH = DTY + 2 * MAXR, SW = DTX + 2 * MAXR, NM = LV ? NMAP_LV : NMAP;
    __shared__ float s_m[NM][SH][SW];
    const RwImg &I = B.im[blockIdx.z];
    const float *__restrict__ c = I.c;
    const uint32_t *__restrict__ bits = I.bits;
    const float *__restrict__ maps = I.maps;
    float *__restrict__ dR = I.dR;
    const int cpitch = I.cpitch, H = I.H, W = I.W, words = I.words;
    const int r = wn.r;
    const int VH = H - 2 * r, VW = W - 2 * r;
    const size_t plane = (size_t)VH * VW;
    const int ay0 = blockIdx.y * DTY, ax0 = blockIdx.x * DTX;
    if (ay0 >= H || ax0 >= W) return;
    const int tid = threadIdx.y * DTX + threadIdx.x;
    // stage maps for output positions j in [a0 - r, a0 + tile + r) (image coords)
    constexpr int NT = NM * SH * SW, NPER = (NT + DTX * DTY - 1) / (DTX * DTY), NB = (NPER + 1) / 2;
#pragma unroll
    for (int k0 = 0; k0 < NPER; k0 += NB) {   // two batches: loads first, then the shared stores
        float vals[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int i = tid + (k0 + k) * DTX * DTY;
            const int q = i / (SH * SW), rem = i % (SH * SW);
            const int yy = rem / SW, xx = rem % SW;
            const int jy = ay0 - r + yy, jx = ax0 - r + xx;   // image coords of output j
            vals[k] = 0.f;
            if (k0 + k < NPER && i < NT && jy >= r && jy < H - r && jx >= r && jx < W - r)
                vals[k] = __ldg(maps + q * plane + (size_t)(jy - r) * VW + (jx - r));
        }
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int i = tid + (k0 + k) * DTX * DTY;
            if (k0 + k < NPER && i < NT) s_m[i / (SH * SW)][(i % (SH * SW)) / SW][i % SW] = vals[k];
        }
    }
    __syncthreads();
    const int ay = ay0 + threadIdx.y, ax = ax0 + threadIdx.x;
    if (ay >= H || ax >= W) return;
    const float ca = c[(size_t)ay * cpitch + ax];
    if constexpr (LV) {
        const float inv = 1.f / (float)(I.levels - 1);
        const int cur = hlevel(bits, words, ay, ax);
        const int lo = min((int)floorf(I.v[(size_t)ay * W + ax] * (float)(I.levels - 1)), I.levels - 2);
        const float hv = (float)cur * inv;
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {                      // q = 0: hi (+), q = 1: lo (-)
            const int lev = lo + (q == 0 ? 1 : 0);
            if (lev == cur) continue;
            const float t = (float)(lev - cur) * inv, sgn = q == 0 ? 1.f : -1.f;
            const float dh2 = (hv + t) * (hv + t) - hv * hv;
            for (int dy = -r; dy <= r; ++dy) {
                const int jy = ay + dy;
                if (jy < r || jy >= H - r) continue;
                const float gy = wn.g[dy + r], wy = wn.w[dy + r];
                for (int dx = -r; dx <= r; ++dx) {
                    const int jx = ax + dx;
                    if (jx < r || jx >= W - r) continue;
                    const int sy = threadIdx.y + r + dy, sx = threadIdx.x + r + dx;
                    const float g = gy * wn.g[dx + r];
                    const float w = wy * wn.w[dx + r];
                    const float e = s_m[0][sy][sx], muh = s_m[1][sy][sx], muc = s_m[2][sy][sx];
                    const float varc2 = s_m[3][sy][sx], cov = s_m[4][sy][sx], sig = s_m[5][sy][sx];
                    const float ss = s_m[6][sy][sx], eh2 = s_m[7][sy][sx];
                    const float muh2 = muh + t * w;
                    const float varh2 = fmaxf(eh2 + dh2 * w - muh2 * muh2, 0.f);
                    const float cov2 = cov + t * w * (ca - muc);
                    const float s2 = __fdividef((2.f * muh2 * muc + wn.c1) * (2.f * cov2 + wn.c2),
                                                (muh2 * muh2 + muc * muc + wn.c1) * (varh2 + varc2));
                    acc += sgn * (-(2.f * t * g * e + t * t * g * g) + wn.ws * sig * (s2 - ss));
                }
            }
        }
        dR[(size_t)ay * W + ax] = acc / ((float)VH * (float)VW);
        return;
    }
    const float ha = hbit(bits, words, ay, ax);
    const float delta = 1.f - 2.f * ha;
    float acc = 0.f;
    for (int dy = -r; dy <= r; ++dy) {
        const int jy = ay + dy;
        if (jy < r || jy >= H - r) continue;
        const float gy = wn.g[dy + r], wy = wn.w[dy + r];
        for (int dx = -r; dx <= r; ++dx) {
            const int jx = ax + dx;
            if (jx < r || jx >= W - r) continue;
            const int sy = threadIdx.y + r + dy, sx = threadIdx.x + r + dx;
            const float g = gy * wn.g[dx + r];
            const float w = wy * wn.w[dx + r];
            const float e = s_m[0][sy][sx], muh = s_m[1][sy][sx], muc = s_m[2][sy][sx];
            const float varc2 = s_m[3][sy][sx], cov = s_m[4][sy][sx], sig = s_m[5][sy][sx], ss = s_m[6][sy][sx];
            const float muh2 = muh + delta * w;
            const float varh2 = muh2 - muh2 * muh2;
            const float cov2 = cov + delta * w * (ca - muc);
            // the denominator lies in [C1 C2, ~5]: the fast division (2 ulp) is exact enough
            const float s2 = __fdividef((2.f * muh2 * muc + wn.c1) * (2.f * cov2 + wn.c2),
                                        (muh2 * muh2 + muc * muc + wn.c1) * (varh2 + varc2));
            acc += -(2.f * g * e + delta * g * g) + delta * wn.ws * sig * (s2 - ss);
        }
    }
    dR[(size_t)ay * W + ax] = acc / ((float)VH * (float)VW);
}

// Binary toggle deltas for a fixed window radius R (the paper's 11 x 11 windows: R = 5),
// the common case of the training step.  The same exact moment-shift update as
// k_toggle_delta, arranged so that the 121-term window loop runs unrolled and without
// bounds checks:
//   - outside the valid region the staged maps read e = 0, sigma = 0, var_c + C2 = 1
//     (every term there then vanishes and no division sees a zero denominator);
//   - the MSE part splits into -2 sum_j g_{j-a} e_j (in the loop) and -delta S_a, with
//     S_a = sum over valid j of g_{j-a}^2 = (sum of g_y^2 over valid rows) x (sum of
//     g_x^2 over valid columns), the window being a product of 1-D taps;
//   - the 2-D tap products g_y g_x and w_y w_x come precomputed in the kernel parameters;
//   - delta w_sg sigma_j (SSIM' - SSIM_j) is summed as sigma_j (SSIM' - SSIM_j), the
//     factor delta w_s applied once.
template <int R>
struct Win2 {
    float g2[(2 * R + 1) * (2 * R + 1)];
    float w2[(2 * R + 1) * (2 * R + 1)];
};

template <int R>
__global__ void __launch_bounds__(DTX *DTY, 3) k_toggle_delta_r(const __grid_constant__ RwBatch B, const Win wn,
                                                                 const __grid_constant__ Win2<R> w2)
{
    constexpr int SH = DTY + 2 * R, SW = DTX + 2 * R, K = 2 * R + 1;
    // the seven maps interleaved as two float4 per position, (e, mu_h, mu_c, var_c + C2) and
    // (cov, sigma, ss, mu_c^2 + C1): two 16-byte loads per window term, consecutive threads
    // 16 bytes apart (no bank conflicts)
    __shared__ float4 s_p[SH][SW], s_q[SH][SW];
    const RwImg &I = B.im[blockIdx.z];
    const float *__restrict__ c = I.c;
    const float *__restrict__ maps = I.maps;
    const int H = I.H, W = I.W;
    const int VH = H - 2 * R, VW = W - 2 * R;
    const size_t plane = (size_t)VH * VW;
    const int ay0 = blockIdx.y * DTY, ax0 = blockIdx.x * DTX;
    if (ay0 >= H || ax0 >= W) return;
    const int tid = threadIdx.y * DTX + threadIdx.x;
    for (int i = tid; i < NMAP * SH * SW; i += DTX * DTY) {
        const int q = i / (SH * SW), rem = i % (SH * SW);
        const int yy = rem / SW, xx = rem % SW;
        const int jy = ay0 - R + yy, jx = ax0 - R + xx;        // image coords of output j
        float v = q == 3 ? 1.f : 0.f;
        if (jy >= R && jy < H - R && jx >= R && jx < W - R) v = __ldg(maps + q * plane + (size_t)(jy - R) * VW + (jx - R));
        float *dst = q < 4 ? &s_p[yy][xx].x + q : &s_q[yy][xx].x + (q - 4);
        *dst = v;
    }
    __syncthreads();
    for (int i = tid; i < SH * SW; i += DTX * DTY) {
        const float muc = s_p[i / SW][i % SW].z;
        s_q[i / SW][i % SW].w = fmaf(muc, muc, wn.c1);
    }
    __syncthreads();
    const int ay = ay0 + threadIdx.y, ax = ax0 + threadIdx.x;
    if (ay >= H || ax >= W) return;
    const float ca = c[(size_t)ay * I.cpitch + ax];
    const float delta = 1.f - 2.f * hbit(I.bits, I.words, ay, ax);
    float sy = 0.f, sx = 0.f;
#pragma unroll
    for (int d = -R; d <= R; ++d) {
        const float gd = wn.g[d + R] * wn.g[d + R];
        if (ay + d >= R && ay + d < H - R) sy += gd;
        if (ax + d >= R && ax + d < W - R) sx += gd;
    }
    float ge = 0.f, acc = 0.f;
#pragma unroll 1
    for (int dy = 0; dy < K; ++dy) {
#pragma unroll
        for (int dx = 0; dx < K; ++dx) {
            const int sy_ = threadIdx.y + dy, sx_ = threadIdx.x + dx;
            const float4 mp = s_p[sy_][sx_], mq = s_q[sy_][sx_];
            const float e = mp.x, muh = mp.y, muc = mp.z, varc2 = mp.w;
            const float cov = mq.x, sig = mq.y, ss = mq.z, muc2c1 = mq.w;
            ge = fmaf(w2.g2[dy * K + dx], e, ge);
            const float dw = delta * w2.w2[dy * K + dx];
            const float muh2 = muh + dw;
            const float varh2 = fmaf(-muh2, muh2, muh2);
            const float cov2 = fmaf(dw, ca - muc, cov);
            const float num = fmaf(2.f * muh2, muc, wn.c1) * fmaf(2.f, cov2, wn.c2);
            const float den = fmaf(muh2, muh2, muc2c1) * (varh2 + varc2);
            // the denominator lies in [C1 C2, ~5]: the fast division (2 ulp) is exact enough
            acc = fmaf(sig, __fdividef(num, den) - ss, acc);
        }
    }
    const float dr = -2.f * ge - delta * (sy * sx) + delta * wn.ws * acc;
    I.dR[(size_t)ay * W + ax] = dr / ((float)VH * (float)VW);
}

Win make_win(const ht_reward_opts &o)
{
    Win wn;
    wn.r = o.radius;
    double sg = 0, sw = 0, g[2 * MAXR + 1], w[2 * MAXR + 1];
    for (int i = -o.radius; i <= o.radius; ++i) {
        g[i + o.radius] = exp(-(double)(i * i) / (2.0 * o.sigma_hvs * o.sigma_hvs));
        w[i + o.radius] = exp(-(double)(i * i) / (2.0 * o.sigma_ssim * o.sigma_ssim));
        sg += g[i + o.radius];
        sw += w[i + o.radius];
    }
    for (int i = 0; i < 2 * MAXR + 1; ++i) {
        wn.g[i] = i <= 2 * o.radius ? (float)(g[i] / sg) : 0.f;
        wn.w[i] = i <= 2 * o.radius ? (float)(w[i] / sw) : 0.f;
    }
    wn.c1 = o.c1;
    wn.c2 = o.c2;
    wn.k = o.k_contrast;
    wn.ws = o.w_s;
    return wn;
}

}  // namespace

namespace {
RwImg rw_img(const ht_image &c, const uint32_t *bits, int levels)
{
    RwImg I{};
    I.c = c.contone;
    I.bits = bits;
    I.cpitch = c.pitch;
    I.H = c.h;
    I.W = c.w;
    I.levels = levels;
    I.words = ht_bits_row_words(c.w, levels > 2 ? HT_HEAD_MULTITONE : HT_HEAD_SIGMOID);
    return I;
}

// reward window sums of images [base, base + cnt) into acc[3 i] (launch only)
ht_status launch_reward_tiles(const ht_image *c, const uint32_t *const *bits, int base, int cnt, const Win &wn,
                              int levels, double *acc, cudaStream_t s)
{
    RwBatch B{};
    int gx = 1, gy = 1;
    for (int k = 0; k < cnt; ++k) {
        const int i = base + k;
        B.im[k] = rw_img(c[i], bits[i], levels);
        B.im[k].acc = acc + 3 * (size_t)k;
        gx = max(gx, (c[i].w - 2 * wn.r + RT - 1) / RT);
        gy = max(gy, (c[i].h - 2 * wn.r + RT - 1) / RT);
    }
    if (levels > 2) k_reward_tiles<true><<<dim3(gx, gy, cnt), dim3(32, 8), 0, s>>>(B, wn);
    else k_reward_tiles<false><<<dim3(gx, gy, cnt), dim3(32, 8), 0, s>>>(B, wn);
    HT_LAUNCH_CHECK();
    return HT_OK;
}
}  // namespace

ht_status ht_reward_launch(const ht_image *c, const uint32_t *const *bits, int n, const ht_reward_opts &o,
                           double *out, cudaStream_t s)
{
    const Win wn = make_win(o);
    // scratch: 3 accumulators + 1/M per image, staged in `out`'s stream via a small allocation
    double *acc = nullptr;
    HT_CUDA_TRY(cudaMallocAsync((void **)&acc, sizeof(double) * 4 * n, s));
    HT_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * 3 * n, s));
    double *inv_m_h = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i) inv_m_h[i] = 1.0 / ((double)(c[i].h - 2 * o.radius) * (double)(c[i].w - 2 * o.radius));
    cudaError_t ce = cudaMemcpyAsync(acc + 3 * n, inv_m_h, sizeof(double) * n, cudaMemcpyHostToDevice, s);
    free(inv_m_h);
    HT_CUDA_TRY(ce);
    ht_prof_start(HTK_REWARD, s);
    for (int base = 0; base < n; base += RW_MAXB) {
        const ht_status st =
            launch_reward_tiles(c, bits, base, min(RW_MAXB, n - base), wn, o.levels, acc + 3 * (size_t)base, s);
        if (st != HT_OK) return st;
    }
    ht_prof_stop(s);
    k_reward_finalize<<<(n + 127) / 128, 128, 0, s>>>(acc, n, acc + 3 * n, o.w_s, out);
    HT_LAUNCH_CHECK();
    HT_CUDA_TRY(cudaFreeAsync(acc, s));
    return HT_OK;
}

ht_status ht_toggle_launch(const ht_image *c, const uint32_t *const *bits, const float *const *v, int n,
                           const ht_reward_opts &o, float *const *dR, float *scratch, size_t scratch_floats,
                           cudaStream_t s)
{
    const Win wn = make_win(o);
    const bool lv = o.levels > 2;
    const int nmap = lv ? NMAP_LV : NMAP;
    for (int base = 0; base < n; base += RW_MAXB) {
        const int cnt = min(RW_MAXB, n - base);
        RwBatch B{};
        size_t off = 0;
        int gx = 1, gy = 1, tx = 1, ty = 1;
        for (int k = 0; k < cnt; ++k) {
            const int i = base + k;
            const int VH = c[i].h - 2 * o.radius, VW = c[i].w - 2 * o.radius;
            B.im[k] = rw_img(c[i], bits[i], o.levels);
            B.im[k].maps = scratch + off;
            B.im[k].dR = dR[i];
            B.im[k].v = lv ? v[i] : nullptr;
            off += (size_t)nmap * VH * VW;
            gx = max(gx, (VW + RT - 1) / RT);
            gy = max(gy, (VH + RT - 1) / RT);
            tx = max(tx, (c[i].w + DTX - 1) / DTX);
            ty = max(ty, (c[i].h + DTY - 1) / DTY);
        }
        if (off > scratch_floats) {
            ht_set_error("toggle-delta scratch too small");
            return HT_ERR_INVALID_ARG;
        }
        ht_prof_start(HTK_TOGGLE, s);
        if (lv) {
            k_moment_maps<true><<<dim3(gx, gy, cnt), dim3(32, 8), 0, s>>>(B, wn);
            HT_LAUNCH_CHECK();
            k_toggle_delta<true><<<dim3(tx, ty, cnt), dim3(DTX, DTY), 0, s>>>(B, wn);
        } else {
            k_moment_maps<false><<<dim3(gx, gy, cnt), dim3(32, 8), 0, s>>>(B, wn);
            HT_LAUNCH_CHECK();
            if (o.radius == 5) {
                Win2<5> w2;
                for (int i = 0; i < 11; ++i)
                    for (int j = 0; j < 11; ++j) {
                        w2.g2[i * 11 + j] = wn.g[i] * wn.g[j];
                        w2.w2[i * 11 + j] = wn.w[i] * wn.w[j];
                    }
                k_toggle_delta_r<5><<<dim3(tx, ty, cnt), dim3(DTX, DTY), 0, s>>>(B, wn, w2);
            } else {
                k_toggle_delta<false><<<dim3(tx, ty, cnt), dim3(DTX, DTY), 0, s>>>(B, wn);
            }
        }
        ht_prof_stop(s);
        HT_LAUNCH_CHECK();
    }
    return HT_OK;
}

size_t ht_toggle_scratch_floats(int h, int w, int r) { return (size_t)NMAP_LV * (h - 2 * r) * (w - 2 * r); }

size_t ht_toggle_scratch_floats_batch(const ht_image *c, int n, int r)
{
    size_t best = 0;
    for (int base = 0; base < n; base += RW_MAXB) {
        size_t sum = 0;
        for (int i = base; i < n && i < base + RW_MAXB; ++i) sum += ht_toggle_scratch_floats(c[i].h, c[i].w, r);
        best = sum > best ? sum : best;
    }
    return best;
}

// ---------------------------------------------------------------------------
// Allocation-free reward.
//
// Some callers of this library must not allocate device memory while they run:
// a host application whose allocator has reserved the device memory it is
// allowed to use (a further cudaMalloc would fail or push it over its budget),
// or a streaming loop that cannot accept the device-wide synchronisation that
// cudaMalloc / cudaFree may imply.  ht_reward needs a few doubles of scratch per
// image (FP64 accumulators); ht_reward_noalloc keeps them in the file-scope
// device array below instead, which every GPU that loads the library holds
// until the process exits.
//
// Host code only sees the array's host-side stand-in; its device address comes
// from cudaGetSymbolAddress with the calling device current.  It is looked up on
// every call made outside a stream capture (so a device reset, which reloads the
// module at a new address, is followed), and the call caches it per device; a call
// whose stream is capturing uses that cache, so the first call on a device must
// come before any capture.  All calls share the array: the accumulators are
// cleared at the start of every call, and calls whose work overlaps on the GPU
// (different streams, no ordering) race on it.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_reward_noalloc_acc[3 * HT_REWARD_NOALLOC_MAX_IMAGES];

namespace {

std::mutex g_noalloc_mu;
double *g_noalloc_addr[64] = {nullptr};

struct InvM64 {
    double v[64];
};

// out[4 i + ...] for images base .. base + count - 1 (count <= 64)
__global__ void k_reward_finalize_noalloc(const double *__restrict__ acc, int count, InvM64 inv_m, float ws,
                                          double *__restrict__ out)
{
    const int i = threadIdx.x;
    if (i >= count) return;
    const double m = inv_m.v[i];
    const double mse = acc[3 * i] * m, ssim = acc[3 * i + 1] * m, cssim = acc[3 * i + 2] * m;
    out[4 * i + 0] = mse;
    out[4 * i + 1] = ssim;
    out[4 * i + 2] = cssim;
    out[4 * i + 3] = -mse + (double)ws * cssim;
}

}  // namespace

extern "C" ht_status ht_reward_noalloc(const ht_image *c, const uint32_t *const *bits, int n,
                                       const ht_reward_opts *opts, double *out, void *stream)
{
    HT_RANGE("ht_reward_noalloc");
    // the same argument checks as ht_reward, plus the array's capacity
    ht_status st = ht_validate_reward_opts(opts);
    if (st != HT_OK) return st;
    st = ht_validate_images(c, n, 2 * opts->radius + 1);
    if (st != HT_OK) return st;
    HT_CHECK_ARG(n <= HT_REWARD_NOALLOC_MAX_IMAGES, "ht_reward_noalloc takes at most %d images per call (got %d)",
                 HT_REWARD_NOALLOC_MAX_IMAGES, n);
    HT_CHECK_ARG(bits && out, "null argument");
    for (int i = 0; i < n; ++i) HT_CHECK_ARG(bits[i] != nullptr, "image %d: null bits", i);
    const int r = opts->radius;
    int dev = 0;
    HT_CUDA_TRY(cudaGetDevice(&dev));
    HT_CHECK_ARG(dev >= 0 && dev < 64, "device index %d out of range", dev);
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    HT_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
    double *acc = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void *addr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&addr, g_reward_noalloc_acc);
            if (e != cudaSuccess || addr == nullptr) {
                ht_set_error("cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return HT_ERR_CUDA;
            }
            g_noalloc_addr[dev] = (double *)addr;
        } else if (!g_noalloc_addr[dev]) {
            ht_set_error("ht_reward_noalloc: the first call on a device must come before any stream capture");
            return HT_ERR_INVALID_ARG;
        }
        acc = g_noalloc_addr[dev];
    }
    const Win wn = make_win(*opts);
    HT_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * 3 * (size_t)n, s));
    for (int base = 0; base < n; base += RW_MAXB) {
        st = launch_reward_tiles(c, bits, base, min(RW_MAXB, n - base), wn, opts->levels, acc + 3 * (size_t)base, s);
        if (st != HT_OK) return st;
    }
    for (int base = 0; base < n; base += 64) {
        const int count = n - base < 64 ? n - base : 64;
        InvM64 im;
        for (int k = 0; k < count; ++k)
            im.v[k] = 1.0 / ((double)(c[base + k].h - 2 * r) * (double)(c[base + k].w - 2 * r));
        k_reward_finalize_noalloc<<<1, 64, 0, s>>>(acc + 3 * base, count, im, opts->w_s, out + 4 * (size_t)base);
        HT_LAUNCH_CHECK();
    }
    return HT_OK;
}

void ht_preload_reward()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_reward_tiles<false>);
    cudaFuncGetAttributes(&fa, k_reward_tiles<true>);
    cudaFuncGetAttributes(&fa, k_reward_finalize);
    cudaFuncGetAttributes(&fa, k_moment_maps<false>);
    cudaFuncGetAttributes(&fa, k_moment_maps<true>);
    cudaFuncGetAttributes(&fa, k_toggle_delta<false>);
    cudaFuncGetAttributes(&fa, k_toggle_delta<true>);
    cudaFuncGetAttributes(&fa, k_toggle_delta_r<5>);
    cudaFuncGetAttributes(&fa, k_reward_finalize_noalloc);
}
