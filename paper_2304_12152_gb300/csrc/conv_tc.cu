// conv_tc.cu -- tensor-core form of the policy forward on sm_103a.
//
// Policy (Sec. III "State"/"Agents", Sec. VI-A): 3x3 convolutions, zero
// padding 1, ReLU between layers, sigmoid / softmax head.
//
//  k_first_input  per pixel, c and the noise channel z (Philox stream 0), each
//                 as an exact sum of three bf16 parts, two 16-byte chunks (the
//                 training step and the residual policy; the inference forms of
//                 the 64-wide policy build these chunks inside layer 1).
//  k_conv_tc      one pipeline, four kinds: layer 1 (2 -> 64, on the split
//                 input), a hidden 64 -> 64 layer, the last hidden layer with
//                 the 1-logit head's per-tap partials fused into its epilogue,
//                 and the 64 -> 4 softmax head.  Implicit GEMM on tcgen05: an
//                 MMA tile is 128 consecutive pixels of one input row (M = 128)
//                 against the three kernel rows stacked along N; K runs over the
//                 input channels, one shifted descriptor per dx.  Input rows are
//                 staged by bulk async copies into a ring of shared-memory
//                 slots; weights stay resident in shared memory; FP32
//                 accumulators live in TMEM (one block per output row of a unit).
//                 Epilogue: tcgen05.ld -> (dequant) + bias -> ReLU -> bf16 / e4m3
//                 -> global (or head partials, or softmax + level draw + packing).
//  k_head_partials  1-logit head: sum of the 9 partials + bias, sigmoid, Philox
//                 stream 1 draw, bit packing.
//
// Activation layout in HBM ("chunk-planar"): [chunk][H][W][16 bytes], a chunk
// being 8 bf16 channels (8 chunks) or 16 e4m3 channels (4 chunks).  One image
// row of one chunk is contiguous, so a staged row is one bulk copy per chunk,
// and it lands in shared memory in the canonical no-swizzle K-major layout
// that tcgen05 descriptors read: pixels at a 16-byte stride (SBO = 128 B per
// 8-pixel core matrix), chunks ROW_PX * 16 B apart (LBO).  A one-pixel shift of
// the A operand is a 16-byte shift of the descriptor start address.
//
// Warp roles (one persistent CTA per SM): warp 0 = copy producer
// (and TMEM owner), warp 1 = MMA issuer, warps 2-9 = epilogue (two per TMEM
// lane quarter), warp 10 = a second copy producer (the two take the staged rows in
// turn): 352 threads.  Layer 1 with its input built in the kernel: 544 threads,
// warps 0 and 10-16 build the staged rows in place of the copy producers.
// Every mbarrier wait is bounded (globaltimer); on expiry the kernel records
// HT_ERR_TIMEOUT, drains its own copies and MMAs, frees TMEM and returns.
#include <stdlib.h>

#include <vector>

#include "tc_common.cuh"

namespace {

#ifndef HT_CONV_NSLOT
#define HT_CONV_NSLOT 6
#endif
#ifndef HT_FUSED_NIN
#define HT_FUSED_NIN 8                     // layer-1 input warps = its ring depth (even)
#endif
constexpr int NSLOT = HT_CONV_NSLOT;       // CTA-pair form: input-row ring depth (lookahead of the copy engine)
constexpr int NTHREADS = 320;              // producer, MMA issuer, 8 epilogue warps
#ifndef HT_CONV_NPROD
#define HT_CONV_NPROD 2
#endif
#ifndef HT_CONV_NS
#define HT_CONV_NS 8                       // k_conv_tc: input-row ring depth (a multiple of NPROD)
#endif
constexpr int NPROD = HT_CONV_NPROD;       // k_conv_tc: copy producers (warps 0, 10, 11, ...)

// Kernel kinds built from one pipeline: a hidden 64 -> 64 layer, the last
// hidden layer with the 1-logit head's per-tap partials fused into its
// epilogue, and layer 1 (2 -> 64), whose input is the 32-byte-per-pixel
// three-part bf16 split of c and z written by k_first_input (two staged chunks,
// K = 16 per MMA of which 12 carry products), and the
// 64 -> 4 softmax head, whose three dy blocks are 16 columns wide (4 logits with
// bf16 hi weights, the same 4 with the lo parts, 8 zero columns: the weights stay
// exact as hi + lo in one MMA per K step); its epilogue adds the two parts,
// applies softmax, draws the level and packs 2 bits/px.
// Residual policy (Sec. VI-A, CH = 32): KIND_RES is a block's second convolution,
// whose epilogue adds the block input -- read in place from the output buffer
// before it is overwritten -- ahead of the ReLU; KIND_RESHEAD is the last block's,
// which turns its output into the head partials instead of storing it.
enum : int { KIND_HIDDEN = 0, KIND_HEADPART = 1, KIND_FIRST = 2, KIND_HEAD4 = 3, KIND_RES = 4, KIND_RESHEAD = 5 };

template <bool FP8, int KIND, int CH = 64, bool F16 = false>
struct Cfg {
    static constexpr bool FIRST = KIND == KIND_FIRST;
    static constexpr bool HEAD4 = KIND == KIND_HEAD4;
    static constexpr bool RES = KIND == KIND_RES || KIND == KIND_RESHEAD;
    static constexpr bool HEADP = KIND == KIND_HEADPART || KIND == KIND_RESHEAD;   // fused head partials
    static constexpr bool MMA8 = FP8 && !FIRST && !HEAD4;      // e4m3 operands (kind::f8f6f4)
    // FP16 form: binary16 operands (kind::f16, format F16) in every layer but layer 1,
    // whose split input and weights stay bf16 (its output is stored as binary16)
    static constexpr bool F16OP = F16 && !FIRST;
    static constexpr uint32_t AB = (MMA8 || F16OP) ? 0u : 1u;  // instruction-descriptor A/B format
    static constexpr int CO = CH;                              // output channels (all but the 4-logit head)
    static constexpr int NCHUNK = FIRST ? 2 : (MMA8 ? CH / 16 : CH / 8);   // 16-byte chunks per staged pixel
    static constexpr int NCOPY = NCHUNK;                       // chunks staged from HBM per pixel
    static constexpr int NOUT = HEAD4 ? 16 : CH;               // output columns per dy block (= TMEM block stride)
    static constexpr int SLOT_BYTES = NCHUNK * ROW_PX * 16;
    static constexpr int W_BYTES = 3 * NCHUNK * 3 * NOUT * 16; // [dx][chunk][3 dy][NOUT n][16 B]
    static constexpr int KSTEPS = NCHUNK / 2;                  // MMAs per dx (K = 16 / 32 per MMA)
    static constexpr int NS = FIRST ? HT_FUSED_NIN : HT_CONV_NS;   // ring depth (layer 1: one input warp per slot)
    static constexpr int SMEM = W_BYTES + NS * SLOT_BYTES + 1024 /*align*/ + 4096 /*barriers*/ + (FIRST ? NS * 576 : 0);
    static_assert(NS % HT_CONV_NPROD == 0 && SMEM <= 232448, "ring depth");
};

struct ConvParams {
    const ImgDesc *imgs;     // device table of the call's images
    int n_imgs, n_units;
    int in_buf;              // activations are read from act[in_buf], written to act[in_buf ^ 1]
    const void *wpack;       // packed weights of this layer ([dx][chunk][3 dy][n][16 B])
    // per-output-channel epilogue constants, read straight from the kernel's
    // constant bank: acc * scale[n] + bias[n] (scale = input scale x weight
    // scale in the FP8 form, 1 otherwise)
    float scale[64];
    float bias[64];
    float head_w[9 * 64];    // fused 1-logit head: last-layer weights [tap][channel]
    unsigned long long head_w2[64][4];   // the same, taps (0,1) (2,3) (4,5) (6,7) packed per channel
    float out_inv_scale;     // FP8 output: 1 / scale of the next layer's input
    int out_fp8;
    uint64_t seed;           // Philox seed (layer 1: noise channel; 4-logit head: level draw)
    int mode;                // 4-logit head: HT_MODE_*
    int dgrad;               // 1: data-gradient layer (no bias, no ReLU; mask from the table, bf16 out)
    int ru, order;           // unit geometry: rows per unit (<= RU TMEM blocks) and unit order
    int *err;
};

// Fused 1-logit head (Sec. VI-A output layer): the nine per-tap dot products of the
// stored (bf16, or binary16 in the FP16 form) activations, acc[t] = sum_n r(v[n]) *
// w[t][n] in channel order.  Taps 0-7 run as packed pairs (each lane an ordinary
// fmaf, so the per-tap sums are bit-identical to nine scalar chains), tap 8 alone.
template <int CO, bool F16 = false>
__device__ __forceinline__ void head_partials9(const float *v, const ConvParams &P, float *acc)
{
    unsigned long long pr[4] = {0ull, 0ull, 0ull, 0ull};
    float a8 = 0.f;
#pragma unroll
    for (int n = 0; n < CO; ++n) {
        const float a = act_round<F16>(v[n]);
        unsigned long long aa;
        asm("mov.b64 %0, {%1, %1};" : "=l"(aa) : "f"(a));
#pragma unroll
        for (int t = 0; t < 4; ++t) asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(pr[t]) : "l"(aa), "l"(P.head_w2[n][t]));
        a8 = fmaf(a, P.head_w[8 * CO + n], a8);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[2 * t]), "=f"(acc[2 * t + 1]) : "l"(pr[t]));
    acc[8] = a8;
}


// ---------------------------------------------------------------------------
// 64 -> 64 layer on tcgen05
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// 64 -> 64 layer on tcgen05
//
// Work unit = RU (8) consecutive output rows x one 128-pixel column tile.  Its
// RU + 2 input rows are staged one after another; each staged input row r is
// multiplied, for every dx and K step, against the three kernel rows stacked
// along N ([dy=2 | dy=1 | dy=0], N = 192): the three 64-column slices of the
// product are exactly the contributions of row r to output rows r-1, r, r+1,
// and they land in those rows' TMEM accumulator blocks, which sit side by side
// (block j = output row y0 + j).  Edge input rows use N = 64 / 128.  Every
// accumulator block is zeroed by the epilogue after it is drained, so all MMAs
// accumulate.  Per output row: 12-15 MMAs of N = 192 instead of 36 of N = 64.
//
// Row-streaming form (STREAM): a unit is a tall strip (P.ru > 8 output rows) of one column
// tile, so every input row is staged once per strip instead of 1.25 times per 8-row unit.
// The eight TMEM blocks form a ring: the CTA's G-th output row (G counts the output rows of
// all its strips so far) accumulates in block G % 8, guarded by that block's bfull / bfree
// barriers at phase G / 8.  A staged row's window of up to three output rows wraps past
// block 7 for two rows in eight; there the window is issued as two MMAs per K step (blocks
// p .. 7 and 0 ..), so that each output row still accumulates in one block through one chain
// of MMAs, in the same order as in the 8-row units: the two forms give identical bits.
// ---------------------------------------------------------------------------
// Layer-1 input of one pixel: c and z each split exactly into three bf16 parts, laid out as
// the K elements (c0, c0, c1, c0, c1, c2, z0, z0 | z1, z0, z1, z2, 0, 0, 0, 0), two 16-byte
// chunks (the matching weights are described at k_first_input).
__device__ __forceinline__ void first_input_pixel(float c, float z, uint4 &o0, uint4 &o1)
{
    float c0, c1, c2, z0, z1, z2;
    split3_bf16(c, c0, c1, c2);
    split3_bf16(z, z0, z1, z2);
    o0 = make_uint4(pack_bf16x2(c0, c0), pack_bf16x2(c1, c0), pack_bf16x2(c1, c2), pack_bf16x2(z0, z0));
    o1 = make_uint4(pack_bf16x2(z1, z0), pack_bf16x2(z1, z2), 0u, 0u);
}

// Layer 1 with its input built in the kernel (FUSED): warps 0 and 10 .. 8 + NIN_WARPS take
// the producers' place, one per input-ring slot (the kind's ring depth, Cfg::NS).  Eight
// warps (96 registers, no spills) built the rows 15% faster than six (124 registers).
constexpr int NIN_WARPS = HT_FUSED_NIN;
constexpr int NTHREADS_FUSED = NTHREADS + (NIN_WARPS - 1) * 32;
static_assert(NTHREADS_FUSED <= 576, "block size of the layer-1 kernel");
constexpr int NTHREADS_CONV = NTHREADS + (NPROD - 1) * 32;   // k_conv_tc: + the further copy producers

template <bool FP8, int KIND, bool TR = false, int CH = 64, bool F16 = false, bool STREAM = false, bool FUSED = false>
__global__ void __launch_bounds__(FUSED ? NTHREADS_FUSED : NTHREADS_CONV, 1) k_conv_tc(const ConvParams P)
{
    static_assert(!FUSED || (KIND == KIND_FIRST && !TR && CH == 64), "in-kernel input: inference layer 1 only");
    static_assert(!FUSED || Cfg<FP8, KIND, CH, F16>::NS == NIN_WARPS, "one input warp per ring slot");
    using C = Cfg<FP8, KIND, CH, F16>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *s_w = smem;
    uint8_t *s_rows = smem + C::W_BYTES;
    uint64_t *bars = (uint64_t *)(s_rows + C::NS * C::SLOT_BYTES);
    uint64_t *full = bars, *empty = bars + C::NS, *wbar = bars + 2 * C::NS, *bfull = wbar + 1, *bfree = bfull + RU,
             *drain = bfree + RU;
    int2 *s_meta = (int2 *)(drain + 1);                         // (k, nrows) of the row in each slot
    uint32_t *s_tmem = (uint32_t *)(s_meta + C::NS);
    volatile int *s_abort = (volatile int *)(s_tmem + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool input_warp = FUSED && (warp == 0 || warp >= 10);

    if (threadIdx.x == 0) {
        for (int i = 0; i < C::NS; ++i) {
            mbar_init(smem_u32(&full[i]), 1);
            mbar_init(smem_u32(&empty[i]), 1);
        }
        mbar_init(smem_u32(wbar), 1);
        for (int i = 0; i < RU; ++i) {
            mbar_init(smem_u32(&bfull[i]), 1);
            mbar_init(smem_u32(&bfree[i]), 4);
        }
        mbar_init(smem_u32(drain), 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(s_tmem), TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *s_tmem;

    if (input_warp) {
        if constexpr (FUSED) {
        // -------------------- producer: layer-1 input built here --------------------
        // NIN_WARPS (= C::NS) warps build the staged rows from the contone image and the noise
        // channel, warp w the rows of ring slot w, so that up to C::NS rows are in flight: per pixel
        // the two 16-byte chunks of the layer-1 input (first_input_pixel, the values
        // k_first_input stores), zero outside the image.  z is Philox4x32-10 of
        // (g / 4, image, 0, 0), g = y * W + x, lane g % 4: the row's calls (at most 34
        // groups of 4 pixels) are made once, two per lane at most, and shared through the
        // warp's part of shared memory.  The contone values of the warp's next row in the
        // same unit are loaded while it builds this one.
        const int wi = warp == 0 ? 0 : warp - 9;                     // 0 .. C::NS - 1 = ring slot
        uint4 *s_u = (uint4 *)(((uintptr_t)(s_abort + 1) + 15) & ~(uintptr_t)15) + wi * 36;
        if (warp == 0 && lane == 0) {
            mbar_arrive_expect_tx(smem_u32(wbar), C::W_BYTES);
            bulk_g2s(smem_u32(s_w), P.wpack, C::W_BYTES, smem_u32(wbar));
        }
        const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
        uint32_t li = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < P.n_units && ok; u += gridDim.x) {
            const UnitInfo ui = unit_info(P.imgs, P.n_imgs, P.in_buf, u, P.ru, P.order);
            const float *__restrict__ contone = ui.D->contone;
            const int cpitch = ui.D->cpitch;
            const uint32_t image = ui.D->image;
            const int H = ui.H, W = ui.W, x0 = ui.x0, y0 = ui.y0, nrows = ui.nrows;
            const int lo = max(x0 - 1, 0), hi = min(x0 - 1 + ROW_PX, W);       // in-image pixel range
            float cn[5];                                       // contone, pixels x0 - 1 + lane + 32 q
            auto load_row = [&](int yy) {
                const bool in = yy >= 0 && yy < H;
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    const int x = x0 - 1 + lane + 32 * q;
                    cn[q] = (in && x >= lo && x < hi) ? __ldg(contone + (size_t)yy * cpitch + x) : 0.f;
                }
            };
            // first row of this unit that is the warp's
            int r = (int)((uint32_t)(wi - (int)(li % C::NS) + C::NS) % C::NS);
            if (r < nrows + 2) load_row(y0 - 1 + r);
            for (; r < nrows + 2; r += C::NS) {
                const uint32_t lr = li + (uint32_t)r;             // this row's index in the CTA's ring sequence
                const int yy = y0 - 1 + r;
                const bool row_in = (yy >= 0 && yy < H) && hi > lo;
                float cv[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) cv[q] = cn[q];
                if (r + C::NS < nrows + 2) load_row(yy + C::NS);
                const uint64_t G0 = row_in ? ((uint64_t)yy * (uint64_t)W + (uint64_t)lo) >> 2 : 0;
                if (row_in) {
                    const uint32_t ng = (uint32_t)((((uint64_t)yy * (uint64_t)W + (uint64_t)(hi - 1)) >> 2) - G0) + 1u;
                    for (uint32_t t = (uint32_t)lane; t < ng; t += 32)
                        s_u[t] = ht_philox4x32_10(make_uint4((uint32_t)(G0 + t), image, 0u, 0u), key);
                }
                int got = 0;
                if (lane == 0) got = mbar_wait(smem_u32(&empty[wi]), ((lr / C::NS) & 1u) ^ 1u, s_abort, P.err) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, got, 0)) {
                    ok = false;
                    break;
                }
                __syncwarp();
                uint8_t *dst = s_rows + wi * C::SLOT_BYTES;
                // z of pixel x is word g % 4 of the row's Philox group g / 4 - G0, g = yy * W + x:
                // 32-bit word (x - lo) + r0 of s_u, r0 = (yy * W + lo) % 4
                const uint32_t *s_u32 = reinterpret_cast<const uint32_t *>(s_u);
                const uint32_t r0 = (uint32_t)(((uint64_t)yy * (uint64_t)W + (uint64_t)lo) & 3u);
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    const int i = lane + 32 * q;               // pixel x0 - 1 + i of the staged row
                    if (i < ROW_PX) {
                        const int x = x0 - 1 + i;
                        uint4 o0 = make_uint4(0, 0, 0, 0), o1 = make_uint4(0, 0, 0, 0);
                        if (row_in && x >= lo && x < hi) {
                            const uint32_t w = s_u32[(uint32_t)(x - lo) + r0];
                            first_input_pixel(cv[q], (float)(w >> 8) * (1.0f / 16777216.0f), o0, o1);
                        }
                        *reinterpret_cast<uint4 *>(dst + (size_t)i * 16) = o0;
                        *reinterpret_cast<uint4 *>(dst + ((size_t)ROW_PX + i) * 16) = o1;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    s_meta[wi] = make_int2(r, nrows);
                    mbar_arrive(smem_u32(&full[wi]));
                }
                __syncwarp();                                  // s_u is rewritten for the warp's next row
            }
            li += (uint32_t)nrows + 2u;
        }
        if (ok && (int)(li % C::NS) == wi) {
            // end marker (from the warp of the next row's slot): the MMA warp stops at k = -1
            if (lane == 0 && mbar_wait(smem_u32(&empty[wi]), ((li / C::NS) & 1u) ^ 1u, s_abort, P.err)) {
                s_meta[wi] = make_int2(-1, 0);
                mbar_arrive(smem_u32(&full[wi]));
            }
        }
        // the weight copy must have landed before the CTA exits
        if (warp == 0 && lane == 0) mbar_wait(smem_u32(wbar), 0, s_abort, P.err, true);
        }
    } else if (warp == 0 || (warp >= 10 && warp < 9 + NPROD)) {
        // ------------------------- producers -------------------------
        // One input row = NCHUNK contiguous runs of ROW_PX * 16 bytes in HBM (one
        // per channel chunk).  NPROD warps (0, 10, ...) take the CTA's ring rows in turn,
        // producer p the rows li = p mod NPROD (the ring depth is a multiple of NPROD, so each
        // slot always has the same producer): one warp's wait and bookkeeping for a row then
        // overlap another's copies, which a single warp left the copy engine idle through.  In-image
        // pixels arrive by bulk async copies (complete_tx on the slot's barrier); halo
        // pixels outside the image are zero-filled by the warp with shared stores, made
        // visible to the tensor core's async proxy by a proxy fence before the arrive.
        const uint32_t turn = warp == 0 ? 0u : (uint32_t)(warp - 9);
        int last_issued[C::NS];
        for (int i = 0; i < C::NS; ++i) last_issued[i] = -1;
        if (warp == 0 && lane == 0) {
            mbar_arrive_expect_tx(smem_u32(wbar), C::W_BYTES);
            bulk_g2s(smem_u32(s_w), P.wpack, C::W_BYTES, smem_u32(wbar));
        }
        uint32_t li = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < P.n_units && ok; u += gridDim.x) {
            const UnitInfo ui = unit_info(P.imgs, P.n_imgs, P.in_buf, u, P.ru, P.order);
            const int y0 = ui.y0, y1 = ui.y0 + ui.nrows, x0 = ui.x0;
            const int lo = max(x0 - 1, 0), hi = min(x0 - 1 + ROW_PX, ui.W);   // in-image pixel range
            for (int r = 0; r < (y1 - y0) + 2; ++r, ++li) {
                if (li % NPROD != turn) continue;              // another producer's row
                const int slot = (int)(li % C::NS);
                const uint32_t ph = (li / C::NS) & 1u;
                int got = 0;
                if (lane == 0) got = mbar_wait(smem_u32(&empty[slot]), ph ^ 1u, s_abort, P.err) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, got, 0)) {
                    ok = false;
                    break;
                }
                uint8_t *dst = s_rows + slot * C::SLOT_BYTES;
                const int yy = y0 - 1 + r;
                const bool row_in = (yy >= 0 && yy < ui.H);
                bool zeroed = false;
                if (!row_in) {
                    for (int k = lane; k < C::NCOPY * ROW_PX; k += 32)
                        *reinterpret_cast<uint4 *>(dst + (size_t)k * 16) = make_uint4(0, 0, 0, 0);
                    zeroed = true;
                } else if (lo > x0 - 1 || hi < x0 - 1 + ROW_PX) {
                    const int nl = lo - (x0 - 1), nr = (x0 - 1 + ROW_PX) - hi;
                    for (int k = lane; k < C::NCOPY * (nl + nr); k += 32) {
                        const int c = k / (nl + nr), j = k % (nl + nr);
                        const int px = j < nl ? j : (hi - (x0 - 1)) + (j - nl);
                        *reinterpret_cast<uint4 *>(dst + ((size_t)c * ROW_PX + px) * 16) = make_uint4(0, 0, 0, 0);
                    }
                    zeroed = true;
                }
                if (zeroed) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                const uint32_t run = (uint32_t)(hi - lo) * 16u;
                if (lane == 0) {
                    s_meta[slot] = make_int2(r, y1 - y0);
                    if (row_in && hi > lo) mbar_arrive_expect_tx(smem_u32(&full[slot]), run * C::NCOPY);
                    else mbar_arrive(smem_u32(&full[slot]));
                }
                __syncwarp();
                if (row_in && hi > lo && lane < C::NCOPY)        // one bulk copy per chunk, issued together
                    bulk_g2s(smem_u32(dst + ((size_t)lane * ROW_PX + (lo - (x0 - 1))) * 16),
                             ui.in + (((size_t)lane * ui.H + yy) * ui.W + lo) * 16, run, smem_u32(&full[slot]));
                last_issued[slot] = (int)li;
            }
        }
        if (ok && li % NPROD == turn) {
            // end marker (from the warp whose turn it is): the MMA warp stops at a row with k = -1
            const int slot = (int)(li % C::NS);
            int got = 0;
            if (lane == 0) got = mbar_wait(smem_u32(&empty[slot]), ((li / C::NS) & 1u) ^ 1u, s_abort, P.err) ? 1 : 0;
            if (__shfl_sync(0xffffffffu, got, 0)) {
                if (lane == 0) {
                    s_meta[slot] = make_int2(-1, 0);
                    mbar_arrive(smem_u32(&full[slot]));
                }
                last_issued[slot] = (int)li;       // the marker is this slot's newest phase
            }
        }
        // drain: every issued copy must have landed before the CTA exits
        if (lane == 0) {
            for (int s2 = 0; s2 < C::NS; ++s2)
                if (last_issued[s2] >= 0)
                    mbar_wait(smem_u32(&full[s2]), ((uint32_t)last_issued[s2] / C::NS) & 1u, s_abort, P.err, true);
            if (warp == 0) mbar_wait(smem_u32(wbar), 0, s_abort, P.err, true);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------- MMA issuer -------------------------
        // The whole warp runs the schedule (its state stays warp-uniform) and one
        // elected lane issues the MMAs and commits.  Each staged row's (k, nrows)
        // comes from the producer's per-slot record, read only where a unit starts;
        // within a unit k steps by one, so nothing but the barrier checks sits between
        // one row's MMAs and the next.  Descriptors = base descriptor + compile-time /
        // small offsets added to the 14-bit start-address field (addresses stay below
        // 256 KB).
        {
            const uint32_t el = elect_one();
            const uint64_t a_base = sdesc(smem_u32(s_rows), ROW_PX * 16, 128);
            const uint64_t b_base = sdesc(smem_u32(s_w), 3 * C::NOUT * 16, 128);
            bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(wbar), 0, s_abort, P.err));
            uint32_t slot = 0, ph = 0, uit = 0;
            uint32_t g0 = 0;                      // streaming form: output rows of the CTA's strips so far
            int k = 0, nrows = 0;
            bool unit_start = true;
            while (ok) {
                ok = mbar_wait_poll_warp(smem_u32(&full[slot]), ph, s_abort, P.err);
                if (!ok) break;
                if (unit_start) {
                    const volatile int *mv = (const volatile int *)&s_meta[slot];
                    k = __shfl_sync(0xffffffffu, mv[0], 0);
                    nrows = __shfl_sync(0xffffffffu, mv[1], 0);
                    if (k < 0) break;
                    unit_start = false;
                    if (C::MMA8 && !STREAM && nrows == RU && P.ru == RU) {
                        // A full unit (the common case) of an e4m3 layer, unrolled: every row's
                        // N range, TMEM block and weight sub-range is a compile-time constant,
                        // so only the barrier checks and the MMAs (6 per row) remain between
                        // rows.  Measured faster for e4m3 layers and slower for bf16 ones
                        // (12 MMAs per row, twice the unrolled code).
#pragma unroll
                        for (int kk = 0; kk < RU + 2; ++kk) {
                            if (kk > 0) {
                                ok = mbar_wait_poll_warp(smem_u32(&full[slot]), ph, s_abort, P.err);
                                if (!ok) break;
                            }
                            if (kk < RU) {
                                ok = mbar_wait_poll_warp(smem_u32(&bfree[kk]), uit & 1u, s_abort, P.err);
                                if (!ok) break;
                            }
                            tc_fence_after();
                            constexpr int zero = 0;
                            const int jlo = kk - 2 > zero ? kk - 2 : zero, jhi = kk < RU - 1 ? kk : RU - 1;
                            const uint32_t n = (uint32_t)(jhi - jlo + 1) * C::NOUT;
                            const uint32_t idesc = idesc_m128_ab<C::AB>(n);
                            const uint32_t sb = (uint32_t)(2 - kk + jlo);
                            const uint32_t d = tmem_base + (uint32_t)jlo * C::NOUT;
                            const uint64_t a_q = a_base + (uint64_t)((slot * (uint32_t)C::SLOT_BYTES) >> 4);
                            const uint64_t b_q = b_base + (uint64_t)((sb * C::NOUT * 16u) >> 4);
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                                for (int ks = 0; ks < C::KSTEPS; ++ks)
                                    mma_ss_el<C::MMA8>(el, d, a_q + (uint64_t)(((2 * ks * ROW_PX + dx) * 16) >> 4),
                                                    b_q + (uint64_t)((((dx * C::NCHUNK + 2 * ks) * 3) * C::NOUT * 16) >> 4),
                                                    idesc);
                            mma_commit_el(el, smem_u32(&empty[slot]));
                            if (kk >= 2) mma_commit_el(el, smem_u32(&bfull[kk - 2]));
                            if (++slot == (uint32_t)C::NS) {
                                slot = 0;
                                ph ^= 1u;
                            }
                        }
                        if (!ok) break;
                        ++uit;
                        unit_start = true;
                        continue;
                    }
                }
                if constexpr (STREAM) {
                    // Eight staged rows with full windows whose first TMEM block is 0 .. 7,
                    // unrolled, so that every window's blocks, split point and weight sub-range
                    // are compile-time constants (the same waits, MMAs and commits in the same
                    // order as the rolled loop below)
                    if (k >= 2 && ((g0 + (uint32_t)k - 2u) & 7u) == 0 && k + 7 <= nrows - 1) {
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            if (kk > 0) {
                                ok = mbar_wait_poll_warp(smem_u32(&full[slot]), ph, s_abort, P.err);
                                if (!ok) break;
                            }
                            const uint32_t g = g0 + (uint32_t)(k + kk);         // output row entering use
                            ok = mbar_wait_poll_warp(smem_u32(&bfree[(kk + 2) & 7]), (g / 8u) & 1u, s_abort, P.err);
                            if (!ok) break;
                            tc_fence_after();
                            constexpr uint32_t r1c[8] = {3, 3, 3, 3, 3, 3, 2, 1};
                            const uint32_t r1 = r1c[kk], r2 = 3u - r1;
                            const uint32_t idesc1 = idesc_m128_ab<C::AB>(r1 * C::NOUT);
                            const uint32_t idesc2 = idesc_m128_ab<C::AB>((r2 ? r2 : 1u) * C::NOUT);
                            const uint64_t a_q = a_base + (uint64_t)((slot * (uint32_t)C::SLOT_BYTES) >> 4);
                            const uint64_t b_q2 = b_base + (uint64_t)((r1 * C::NOUT * 16u) >> 4);
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                                for (int ks = 0; ks < C::KSTEPS; ++ks) {
                                    const uint64_t a_k = a_q + (uint64_t)(((2 * ks * ROW_PX + dx) * 16) >> 4);
                                    const uint64_t b_k =
                                        (uint64_t)((((dx * C::NCHUNK + 2 * ks) * 3) * C::NOUT * 16) >> 4);
                                    mma_ss_el<C::MMA8>(el, tmem_base + (uint32_t)kk * C::NOUT, a_k, b_base + b_k, idesc1);
                                    if (r2) mma_ss_el<C::MMA8>(el, tmem_base, a_k, b_q2 + b_k, idesc2);
                                }
                            mma_commit_el(el, smem_u32(&empty[slot]));
                            mma_commit_el(el, smem_u32(&bfull[kk]));      // output row k + kk - 2 complete
                            if (++slot == (uint32_t)C::NS) {
                                slot = 0;
                                ph ^= 1u;
                            }
                        }
                        if (!ok) break;
                        k += 8;
                        continue;
                    }
                }
                if (k < nrows) {                                                   // block of row k enters use
                    if constexpr (STREAM) {
                        const uint32_t g = g0 + (uint32_t)k;
                        ok = mbar_wait_poll_warp(smem_u32(&bfree[g % 8u]), (g / 8u) & 1u, s_abort, P.err);
                    } else {
                        ok = mbar_wait_poll_warp(smem_u32(&bfree[k]), uit & 1u, s_abort, P.err);
                    }
                    if (!ok) break;
                }
                tc_fence_after();
                const int jlo = max(0, k - 2), jhi = min(nrows - 1, k);
                const uint32_t sb = (uint32_t)(2 - k + jlo);                       // first stacked dy block
                const uint32_t a_off = (slot * (uint32_t)C::SLOT_BYTES) >> 4;
                if constexpr (STREAM) {
                    // ring block of row jlo; rows past block 7 go to a second MMA at block 0
                    const uint32_t p = (g0 + (uint32_t)jlo) % 8u;
                    const uint32_t r = (uint32_t)(jhi - jlo + 1);
                    const uint32_t r1 = min(r, 8u - p), r2 = r - r1;
                    const uint32_t idesc1 = idesc_m128_ab<C::AB>(r1 * C::NOUT);
                    const uint32_t idesc2 = idesc_m128_ab<C::AB>((r2 ? r2 : 1u) * C::NOUT);
                    const uint64_t a_q = a_base + (uint64_t)a_off;
                    const uint64_t b_q1 = b_base + (uint64_t)((sb * C::NOUT * 16u) >> 4);
                    const uint64_t b_q2 = b_base + (uint64_t)(((sb + r1) * C::NOUT * 16u) >> 4);
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                        for (int ks = 0; ks < C::KSTEPS; ++ks) {
                            const uint64_t a_k = a_q + (uint64_t)(((2 * ks * ROW_PX + dx) * 16) >> 4);
                            const uint64_t b_k = (uint64_t)((((dx * C::NCHUNK + 2 * ks) * 3) * C::NOUT * 16) >> 4);
                            mma_ss_el<C::MMA8>(el, tmem_base + p * C::NOUT, a_k, b_q1 + b_k, idesc1);
                            if (r2) mma_ss_el<C::MMA8>(el, tmem_base, a_k, b_q2 + b_k, idesc2);
                        }
                } else {
                    const uint32_t n = (uint32_t)(jhi - jlo + 1) * C::NOUT;
                    const uint32_t idesc = idesc_m128_ab<C::AB>(n);
                    const uint32_t d = tmem_base + (uint32_t)jlo * C::NOUT;
                    const uint64_t a_q = a_base + (uint64_t)a_off;
                    const uint64_t b_q = b_base + (uint64_t)((sb * C::NOUT * 16u) >> 4);
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                        for (int ks = 0; ks < C::KSTEPS; ++ks)
                            mma_ss_el<C::MMA8>(el, d, a_q + (uint64_t)(((2 * ks * ROW_PX + dx) * 16) >> 4),
                                            b_q + (uint64_t)((((dx * C::NCHUNK + 2 * ks) * 3) * C::NOUT * 16) >> 4),
                                            idesc);
                }
                mma_commit_el(el, smem_u32(&empty[slot]));
                if (k >= 2)                                                 // output row k-2 complete
                    mma_commit_el(el, smem_u32(&bfull[STREAM ? (g0 + (uint32_t)k - 2u) % 8u : (uint32_t)(k - 2)]));
                if (++slot == (uint32_t)C::NS) {
                    slot = 0;
                    ph ^= 1u;
                }
                if (STREAM && k == nrows + 1) {
                    g0 += (uint32_t)nrows;                // the ring continues with the next strip
                    unit_start = true;
                } else if (k == nrows + 1) {
                    // Blocks a short unit leaves unused still go through one full/free round per
                    // unit, so that every block's barriers stay in step.  Wait until the epilogue
                    // has released the block from the previous unit before signalling it: a parity
                    // wait cannot tell phase k from phase k + 2, so no barrier may run two phases
                    // ahead of its consumer (two short units in a row would otherwise do that).
                    for (int j = nrows; j < P.ru && ok; ++j) {
                        ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&bfree[j]), uit & 1u, s_abort, P.err));
                        if (ok) mma_commit_el(el, smem_u32(&bfull[j]));
                    }
                    ++uit;
                    unit_start = true;
                } else {
                    ++k;
                }
            }
            // drain: all issued MMAs complete before TMEM is released
            mma_commit_el(el, smem_u32(drain));
            mbar_wait(smem_u32(drain), 0, s_abort, P.err, true);
        }
    } else {
        // ------------------------- epilogue -------------------------
        // Eight warps: two per TMEM lane quarter; group g drains blocks g, g+2, ...  (8-row
        // units: block j holds row j; streaming form: block (G0 + j) % 8 holds row j, so a
        // group still owns the blocks of its parity)
        const int quarter = warp & 3;                 // TMEM lanes 32*quarter .. +31
        const int grp = (warp - 2) >> 2;              // 0 or 1
        const int px = quarter * 32 + lane;           // pixel within the tile
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        const int nblk = STREAM ? 8 : P.ru;
        // accumulators start at zero (TMEM is undefined after allocation)
        for (int j = grp; j < nblk; j += 2)
            for (int c = 0; c < C::NOUT; c += 16) tmem_zero16(lane_base + j * C::NOUT + c);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0)
            for (int j = grp; j < nblk; j += 2) mbar_arrive(smem_u32(&bfree[j]));
        uint32_t uit = 0;
        uint32_t g0 = 0;                              // streaming form: the CTA's output rows so far
        bool ok = true;
        for (int u = blockIdx.x; u < P.n_units && ok; u += gridDim.x, ++uit) {
            const UnitInfo ui = unit_info(P.imgs, P.n_imgs, P.in_buf, u, P.ru, P.order);
            const int y0 = ui.y0, nrows = ui.nrows;
            const int x = ui.x0 + px;
            const int jbeg = STREAM ? (int)((g0 + (uint32_t)grp) & 1u) : grp;
            const int jend = STREAM ? nrows : P.ru;
            const uint32_t g_unit = g0;
            if (STREAM) g0 += (uint32_t)nrows;
            for (int j = jbeg; j < jend; j += 2) {
                const uint32_t blk = STREAM ? (g_unit + (uint32_t)j) % 8u : (uint32_t)j;
                const uint32_t par = STREAM ? ((g_unit + (uint32_t)j) / 8u) & 1u : uit & 1u;
                int got = 0;
                if (lane == 0) got = mbar_wait(smem_u32(&bfull[blk]), par, s_abort, P.err) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if constexpr (C::HEAD4) {
                    // 4-logit head: softmax, level draw, 2-bit packing (whole warp, 32 pixels)
                    float v[16];
                    if (j < nrows) {
                        const uint32_t taddr = lane_base + blk * C::NOUT;
                        tmem_ld16(taddr, v);
                        tmem_wait_ld();
                        tmem_zero16(taddr);
                        tmem_wait_st();
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&bfree[blk]));
                    if (j < nrows) {
                        float z[4];
#pragma unroll
                        for (int k2 = 0; k2 < 4; ++k2)                 // (hi + lo parts) x weight scale + bias
                            z[k2] = fmaf(v[k2] + v[k2 + 4], P.scale[k2], P.bias[k2]);
                        const ImgDesc *D = ui.D;
                        ht_head_emit(z, 4, HT_HEAD_SOFTMAX, P.mode, P.seed, D->image, ui.x0 + quarter * 32, y0 + j,
                                     ui.H, ui.W, D->bits, D->words, D->prob);
                    }
                    continue;
                }
                float v[C::CO];
                if (j < nrows) {
                    const uint32_t taddr = lane_base + blk * (uint32_t)C::NOUT;
#pragma unroll
                    for (int c = 0; c < C::CO; c += 16) tmem_ld16(taddr + c, v + c);
                    tmem_wait_ld();
                    for (int c = 0; c < C::CO; c += 16) tmem_zero16(taddr + c);
                    tmem_wait_st();
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bfree[blk]));
                if (j < nrows && x < ui.W) {
                    const size_t o = (size_t)(y0 + j) * ui.W + x;
                    if (TR && P.dgrad) {
                        // data gradient: mask by the ReLU of the layer this gradient flows into
                        const uint2 m = __ldg(ui.D->mask + o);
#pragma unroll
                        for (int n = 0; n < C::CO; ++n)
                            if (!(((n < 32 ? m.x : m.y) >> (n & 31)) & 1u)) v[n] = 0.f;
                        store_pixel<C::CO>(v, ui.out, 0, 1.f, ui.H, ui.W, y0 + j, x);
                        continue;
                    }
                    if constexpr ((KIND == KIND_HIDDEN || KIND == KIND_FIRST) && !TR && CH == 64) {
                        if (!P.out_fp8) {
                            store_pixel_bias_relu_bf16<F16>(v, P.scale, P.bias, ui.out, ui.H, ui.W, y0 + j, x);
                        } else {
                            store_pixel_bias_relu_e4m3(v, P.scale, P.bias, P.out_inv_scale, ui.out, ui.H, ui.W, y0 + j,
                                                       x);
                        }
                        continue;
                    }
#pragma unroll
                    for (int n = 0; n < C::CO; ++n) v[n] = fmaf(v[n], P.scale[n], P.bias[n]);
                    if constexpr (C::RES) {
                        // identity shortcut: the block input, stored (bf16) where this output goes
#pragma unroll
                        for (int c = 0; c < C::CO / 8; ++c) {
                            const uint4 q = *reinterpret_cast<const uint4 *>(
                                ui.out + (((size_t)c * ui.H + y0 + j) * ui.W + x) * 16);
                            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                v[8 * c + 2 * h] += __uint_as_float(w4[h] << 16);
                                v[8 * c + 2 * h + 1] += __uint_as_float(w4[h] & 0xFFFF0000u);
                            }
                        }
                    }
#pragma unroll
                    for (int n = 0; n < C::CO; ++n) v[n] = fmaxf(v[n], 0.f);
                    if (TR && ui.D->mask) {
                        // training forward: which stored (bf16) activations are positive
                        uint2 m = make_uint2(0u, 0u);
#pragma unroll
                        for (int n = 0; n < 32; ++n) {
                            m.x |= (bf16_round(v[n]) > 0.f ? 1u : 0u) << n;
                            if (C::CO > 32) m.y |= (bf16_round(v[(n + 32) % C::CO]) > 0.f ? 1u : 0u) << n;
                        }
                        ui.D->mask[o] = m;
                    }
                    if constexpr (C::HEADP) {
                        // fused C -> 1 head: per-tap dot products of the bf16-rounded activations
                        const size_t plane = (size_t)ui.H * ui.W;
                        float *partials = ui.D->part ? ui.D->part : (float *)ui.out;
                        float acc[9];
                        head_partials9<C::CO, F16>(v, P, acc);
#pragma unroll
                        for (int t = 0; t < 9; ++t) partials[t * plane + o] = acc[t];
                        if (TR && ui.D->save) store_pixel<C::CO>(v, ui.D->save, 0, 1.f, ui.H, ui.W, y0 + j, x);
                    } else if constexpr (F16 && CH == 64) {
                        store_pixel_f16(v, ui.out, ui.H, ui.W, y0 + j, x);
                    } else {
                        store_pixel<C::CO>(v, ui.out, P.out_fp8, P.out_inv_scale, ui.H, ui.W, y0 + j, x);
                    }
                }
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

// ---------------------------------------------------------------------------
// CTA-pair form of the 64 -> 64 layer (hidden, and the last hidden layer with
// the fused head partials): tcgen05 cta_group::2, M = 256.
//
// A cluster of two CTAs works on one unit = RU output rows x one 256-pixel
// column tile; CTA r stages and stores pixels [x0 + 128 r, x0 + 128 r + 128).
// The first CTA's MMA warp issues every MMA of the unit: A = both CTAs' staged
// rows (each 128 x K at the same shared offset), B = the dy-stacked weights
// split by N between the CTAs, D = each CTA's own TMEM blocks.  A single-CTA
// MMA (M = 128) re-fetches its 128-row A tile from shared memory for every
// instruction; with a pair each SM still supplies 128 rows of A but only half
// of B, and the instruction stream runs at the tensor pipe's own rate.
//
// Weights (this CTA's half): per (dx, K step) one group of PV_ROWS rows x 32 B
// holding, for each N range an MMA of a unit can cover, the CTA's n/2 rows
// (variant v: stacked columns [start, start + n) of [dy=2 | dy=1 | dy=0]).
//
// Hand-offs between the CTAs: the second CTA's warp 1 relays "my row landed"
// and "my weights landed" to the first CTA (remote mbarrier arrive on pfull /
// pwbar); the second CTA's epilogue warps release accumulator blocks on the
// first CTA's bfree; the MMA warp's commits arrive on both CTAs' barriers
// (multicast).  The producer passes (k, nrows) of every staged row, and an end
// marker, through s_meta, so the MMA warp needs no image-table lookups.
// ---------------------------------------------------------------------------
constexpr int PV_ROWS = 320;                    // 96 + 32 + 64 + 64 + 32 + 32
constexpr int PV_GROUP_BYTES = PV_ROWS * 32;    // two 16-byte K chunks per row
__host__ __device__ constexpr int pv_start(int v) { return v == 1 ? 128 : (v == 2 || v == 5) ? 64 : 0; }
__host__ __device__ constexpr int pv_n(int v) { return v == 0 ? 192 : (v == 2 || v == 3) ? 128 : 64; }
__host__ __device__ constexpr int pv_row(int v)
{
    return v == 0 ? 0 : v == 1 ? 96 : v == 2 ? 128 : v == 3 ? 192 : v == 4 ? 256 : 288;
}
// variant of an MMA that starts at dy block sb (0 = dy 2) and covers n columns
__device__ __forceinline__ int pv_of(int sb, int n)
{
    return n == 192 ? 0 : n == 128 ? (sb == 1 ? 2 : 3) : (sb == 2 ? 1 : sb == 0 ? 4 : 5);
}

template <bool FP8>
struct Cfg2 {
    static constexpr int NCHUNK = FP8 ? 4 : 8;                  // 16-byte chunks per staged pixel
    static constexpr int KSTEPS = NCHUNK / 2;                   // MMAs per dx (K = 16 bf16 / 32 e4m3)
    static constexpr int SLOT_BYTES = NCHUNK * ROW_PX * 16;
    static constexpr int W_BYTES = 3 * KSTEPS * PV_GROUP_BYTES; // this CTA's weight image
    static constexpr int SMEM = W_BYTES + NSLOT * SLOT_BYTES + 1024 /*align*/ + 4096 /*barriers, meta*/;
};

template <bool FP8, int KIND>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1) k_conv_tc2(const ConvParams P)
{
    using C = Cfg2<FP8>;
    constexpr bool HEADP = KIND == KIND_HEADPART;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *s_w = smem;
    uint8_t *s_rows = smem + C::W_BYTES;
    uint64_t *bars = (uint64_t *)(s_rows + NSLOT * C::SLOT_BYTES);
    uint64_t *full = bars, *pfull = bars + NSLOT, *empty = bars + 2 * NSLOT, *wbar = bars + 3 * NSLOT,
             *pwbar = wbar + 1, *bfull = wbar + 2, *bfree = bfull + RU, *drain = bfree + RU;
    int2 *s_meta = (int2 *)(drain + 1);                         // (k, nrows) of the row in each slot
    uint32_t *s_tmem = (uint32_t *)(s_meta + NSLOT);
    volatile int *s_abort = (volatile int *)(s_tmem + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int pair_id = (int)blockIdx.x >> 1, n_pairs = (int)gridDim.x >> 1;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NSLOT; ++i) {
            mbar_init(smem_u32(&full[i]), 1);
            mbar_init(smem_u32(&pfull[i]), 1);
            mbar_init(smem_u32(&empty[i]), 1);
        }
        mbar_init(smem_u32(wbar), 1);
        mbar_init(smem_u32(pwbar), 1);
        for (int i = 0; i < RU; ++i) {
            mbar_init(smem_u32(&bfull[i]), 1);
            mbar_init(smem_u32(&bfree[i]), 8);                 // 4 epilogue warps in each CTA
        }
        mbar_init(smem_u32(drain), 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    cluster_sync_all();          // both CTAs' barriers exist before any remote arrive or multicast commit
    if (warp == 0) tmem_alloc_pair(smem_u32(s_tmem), TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem_base = *s_tmem;
    const uint32_t peer_abort = mapa_rank(smem_u32((const void *)s_abort), rank ^ 1u);

    if (warp == 0) {
        // ------------------------- producer (both CTAs) -------------------------
        int last_issued[NSLOT];
        for (int i = 0; i < NSLOT; ++i) last_issued[i] = -1;
        if (lane == 0) {
            mbar_arrive_expect_tx(smem_u32(wbar), C::W_BYTES);
            bulk_g2s(smem_u32(s_w), (const uint8_t *)P.wpack + (size_t)rank * C::W_BYTES, C::W_BYTES, smem_u32(wbar));
        }
        uint32_t li = 0;
        bool ok = true;
        for (int u = pair_id; u < P.n_units && ok; u += n_pairs) {
            const UnitInfo ui = unit_info<true>(P.imgs, P.n_imgs, P.in_buf, u, P.ru, P.order);
            const int y0 = ui.y0, nrows = ui.nrows, x0 = ui.x0 + TILE_M * (int)rank;
            const int lo = max(x0 - 1, 0), hi = min(x0 - 1 + ROW_PX, ui.W);   // in-image pixel range
            for (int r = 0; r < nrows + 2; ++r, ++li) {
                const int slot = (int)(li % NSLOT);
                const uint32_t ph = (li / NSLOT) & 1u;
                int got = 0;
                if (lane == 0) got = mbar_wait_cl(smem_u32(&empty[slot]), ph ^ 1u, s_abort, peer_abort, P.err) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, got, 0)) {
                    ok = false;
                    break;
                }
                uint8_t *dst = s_rows + slot * C::SLOT_BYTES;
                const int yy = y0 - 1 + r;
                const bool any = (yy >= 0 && yy < ui.H && hi > lo);
                bool zeroed = false;
                if (!any) {
                    for (int k = lane; k < C::NCHUNK * ROW_PX; k += 32)
                        *reinterpret_cast<uint4 *>(dst + (size_t)k * 16) = make_uint4(0, 0, 0, 0);
                    zeroed = true;
                } else if (lo > x0 - 1 || hi < x0 - 1 + ROW_PX) {
                    const int nl = lo - (x0 - 1), nr = (x0 - 1 + ROW_PX) - hi;   // both in [0, ROW_PX)
                    for (int k = lane; k < C::NCHUNK * (nl + nr); k += 32) {
                        const int c = k / (nl + nr), j = k % (nl + nr);
                        const int px = j < nl ? j : (hi - (x0 - 1)) + (j - nl);
                        *reinterpret_cast<uint4 *>(dst + ((size_t)c * ROW_PX + px) * 16) = make_uint4(0, 0, 0, 0);
                    }
                    zeroed = true;
                }
                if (zeroed) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    s_meta[slot] = make_int2(r, nrows);
                    if (any) {
                        const uint32_t run = (uint32_t)(hi - lo) * 16u;
                        mbar_arrive_expect_tx(smem_u32(&full[slot]), run * C::NCHUNK);
                        for (int c = 0; c < C::NCHUNK; ++c)
                            bulk_g2s(smem_u32(dst + ((size_t)c * ROW_PX + (lo - (x0 - 1))) * 16),
                                     ui.in + (((size_t)c * ui.H + yy) * ui.W + lo) * 16, run, smem_u32(&full[slot]));
                    } else {
                        mbar_arrive(smem_u32(&full[slot]));
                    }
                }
                last_issued[slot] = (int)li;
            }
        }
        if (ok) {
            // end marker: the consumers stop at a row with k = -1
            const int slot = (int)(li % NSLOT);
            int got = 0;
            if (lane == 0)
                got = mbar_wait_cl(smem_u32(&empty[slot]), ((li / NSLOT) & 1u) ^ 1u, s_abort, peer_abort, P.err) ? 1 : 0;
            if (__shfl_sync(0xffffffffu, got, 0)) {
                if (lane == 0) {
                    s_meta[slot] = make_int2(-1, 0);
                    mbar_arrive(smem_u32(&full[slot]));
                }
                // the marker is this slot's newest phase: the drain below waits for it
                // (its parity), which implies the slot's earlier copies have landed
                last_issued[slot] = (int)li;
            }
        }
        // drain: every issued copy must have landed before the CTA exits
        if (lane == 0) {
            for (int s2 = 0; s2 < NSLOT; ++s2)
                if (last_issued[s2] >= 0)
                    mbar_wait(smem_u32(&full[s2]), ((uint32_t)last_issued[s2] / NSLOT) & 1u, s_abort, P.err, true);
            mbar_wait(smem_u32(wbar), 0, s_abort, P.err, true);
        }
        __syncwarp();
    } else if (warp == 1 && leader) {
        // ------------------------- MMA issuer (first CTA, whole warp, elected lane issues) ----------
        {
            const uint32_t el = elect_one();
            const uint64_t a_base = sdesc(smem_u32(s_rows), ROW_PX * 16, 128);
            const uint32_t w_addr = smem_u32(s_w);
            auto wait1 = [&](uint32_t bar, uint32_t par) -> bool {
                return __all_sync(0xffffffffu, mbar_wait_cl(bar, par, s_abort, peer_abort, P.err));
            };
            bool ok = wait1(smem_u32(wbar), 0) && wait1(smem_u32(pwbar), 0);
            uint32_t slot = 0, ph = 0, uit = 0;
            int k = 0, nrows = 0;
            bool unit_start = true;
            while (ok) {
                ok = wait1(smem_u32(&full[slot]), ph) && wait1(smem_u32(&pfull[slot]), ph);
                if (!ok) break;
                if (unit_start) {
                    const volatile int *mv = (const volatile int *)&s_meta[slot];
                    k = __shfl_sync(0xffffffffu, mv[0], 0);
                    nrows = __shfl_sync(0xffffffffu, mv[1], 0);
                    if (k < 0) break;
                    unit_start = false;
                }
                if (k < nrows) {
                    ok = wait1(smem_u32(&bfree[k]), uit & 1u);     // block k enters use
                    if (!ok) break;
                }
                tc_fence_after();
                const int jlo = max(0, k - 2), jhi = min(nrows - 1, k);
                const uint32_t n = (uint32_t)(jhi - jlo + 1) * 64u;
                const int sb = 2 - k + jlo;                                  // first stacked dy block
                const int v = pv_of(sb, (int)n);
                const uint64_t b_q = sdesc(w_addr + (uint32_t)pv_row(v) * 32u, (uint32_t)(pv_n(v) / 2) * 16u, 128u);
                const uint32_t idesc = idesc_m256<FP8>(n);
                const uint32_t d = tmem_base + (uint32_t)jlo * 64u;
                const uint64_t a_q = a_base + (uint64_t)((slot * (uint32_t)C::SLOT_BYTES) >> 4);
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                    for (int ks = 0; ks < C::KSTEPS; ++ks)
                        mma_ss_pair_el<FP8>(el, d, a_q + (uint64_t)(((2 * ks * ROW_PX + dx) * 16) >> 4),
                                         b_q + (uint64_t)(((dx * C::KSTEPS + ks) * PV_GROUP_BYTES) >> 4), idesc);
                mma_commit_pair_el(el, smem_u32(&empty[slot]));
                if (k >= 2) mma_commit_pair_el(el, smem_u32(&bfull[k - 2]));       // output row k-2 complete
                if (++slot == (uint32_t)NSLOT) {
                    slot = 0;
                    ph ^= 1u;
                }
                if (k == nrows + 1) {
                    // blocks this unit leaves unused still go through one full/free round
                    for (int j = nrows; j < P.ru && ok; ++j) {
                        ok = wait1(smem_u32(&bfree[j]), uit & 1u);
                        if (ok) mma_commit_pair_el(el, smem_u32(&bfull[j]));
                    }
                    ++uit;
                    unit_start = true;
                } else {
                    ++k;
                }
            }
            // drain: every issued MMA completes before TMEM is released
            mma_commit_pair_el(el, smem_u32(drain));
            mbar_wait_cl(smem_u32(drain), 0, s_abort, 0u, P.err, true);
        }
    } else if (warp == 1) {
        // ------------------------- relay (second CTA, lane 0) -------------------------
        if (lane == 0) {
            bool ok = mbar_wait_cl(smem_u32(wbar), 0, s_abort, peer_abort, P.err);
            if (ok) mbar_arrive_cluster(mapa_rank(smem_u32(pwbar), 0u));
            for (uint32_t q = 0; ok; ++q) {
                const int slot = (int)(q % NSLOT);
                ok = mbar_wait_cl(smem_u32(&full[slot]), (q / NSLOT) & 1u, s_abort, peer_abort, P.err);
                if (!ok) break;
                const int k = ((const volatile int *)&s_meta[slot])[0];
                mbar_arrive_cluster(mapa_rank(smem_u32(&pfull[slot]), 0u));
                if (k < 0) break;
            }
            // the first CTA's last MMAs read this CTA's shared memory and write its TMEM
            mbar_wait_cl(smem_u32(drain), 0, s_abort, 0u, P.err, true);
        }
    } else {
        // ------------------------- epilogue (both CTAs) -------------------------
        const int quarter = warp & 3;                 // TMEM lanes 32*quarter .. +31
        const int grp = (warp - 2) >> 2;              // 0 or 1
        const int px = quarter * 32 + lane;           // pixel within this CTA's 128-pixel half
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        auto release = [&](int j) {
            if (leader) mbar_arrive(smem_u32(&bfree[j]));
            else mbar_arrive_cluster(mapa_rank(smem_u32(&bfree[j]), 0u));
        };
        for (int j = grp; j < P.ru; j += 2)
            for (int c = 0; c < 64; c += 16) tmem_zero16(lane_base + j * 64 + c);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0)
            for (int j = grp; j < P.ru; j += 2) release(j);
        uint32_t uit = 0;
        bool ok = true;
        for (int u = pair_id; u < P.n_units && ok; u += n_pairs, ++uit) {
            const UnitInfo ui = unit_info<true>(P.imgs, P.n_imgs, P.in_buf, u, P.ru, P.order);
            const int y0 = ui.y0, nrows = ui.nrows;
            const int x = ui.x0 + TILE_M * (int)rank + px;
            for (int j = grp; j < P.ru; j += 2) {
                int got = 0;
                if (lane == 0) got = mbar_wait_cl(smem_u32(&bfull[j]), uit & 1u, s_abort, peer_abort, P.err) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                float v[64];
                if (j < nrows) {
                    const uint32_t taddr = lane_base + j * 64u;
#pragma unroll
                    for (int c = 0; c < 64; c += 16) tmem_ld16(taddr + c, v + c);
                    tmem_wait_ld();
                    for (int c = 0; c < 64; c += 16) tmem_zero16(taddr + c);
                    tmem_wait_st();
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) release(j);
                if (j < nrows && x < ui.W) {
                    const size_t o = (size_t)(y0 + j) * ui.W + x;
                    if (!HEADP && !P.out_fp8) {
                        store_pixel_bias_relu_bf16(v, P.scale, P.bias, ui.out, ui.H, ui.W, y0 + j, x);
                        continue;
                    }
#pragma unroll
                    for (int n = 0; n < 64; ++n) v[n] = fmaxf(fmaf(v[n], P.scale[n], P.bias[n]), 0.f);
                    if constexpr (HEADP) {
                        const size_t plane = (size_t)ui.H * ui.W;
                        float *partials = ui.D->part ? ui.D->part : (float *)ui.out;
                        float acc[9];
                        head_partials9<64>(v, P, acc);
#pragma unroll
                        for (int t = 0; t < 9; ++t) partials[t * plane + o] = acc[t];
                    } else {
                        store_pixel<64>(v, ui.out, P.out_fp8, P.out_inv_scale, ui.H, ui.W, y0 + j, x);
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync_all();          // neither CTA frees TMEM or exits while the pair's MMAs may touch it
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// Layer-1 input: per pixel, c and z each split exactly into three bf16 parts
// v = v0 + v1 + v2 (split3_bf16), laid out as the K elements
//   (c0, c0, c1, c0, c1, c2, z0, z0 | z1, z0, z1, z2, 0, 0, 0, 0)
// in two 16-byte chunks of the chunk-planar layout (chunk 0 in act[1], chunk 1
// H*W*16 bytes after it).  The packed layer-1 weights hold the matching
// (w0, w1, w0, w2, w1, w0) per input channel, so one bf16 MMA forms
// v0 w0 + v0 w1 + v1 w0 + v0 w2 + v1 w1 + v2 w0: every product whose size is
// above 2^-24 |v w| (the terms left out are below 2^-25 |v w|), i.e. the
// layer-1 sums carry float32-level error, as a float32 convolution would.
// z comes from Philox4x32-10 with one call per aligned group of 4 indices g.
// ---------------------------------------------------------------------------
// A block covers 256 groups (1 024 pixels).  Where they all belong to one image, the
// outputs are staged in shared memory and written back with consecutive threads on
// consecutive pixels; a block that straddles two images writes pixel by pixel.
__global__ void __launch_bounds__(256) k_first_input(const ImgDesc *__restrict__ imgs, int n_imgs, int n_groups,
                                                     uint64_t seed)
{
    __shared__ uint4 s_out[2][1024];
    const int t = threadIdx.x;
    const int gb = blockIdx.x * 256;                            // the block's first 4-group
    const int gi = gb + t;                                      // this thread's 4-group
    const int im = find_image(n_imgs, gi < n_groups ? gi : n_groups - 1,
                              [&](int i) { return __ldg(&imgs[i].pre_begin); });
    const int imb = find_image(n_imgs, gb, [&](int i) { return __ldg(&imgs[i].pre_begin); });
    const bool one_image = __syncthreads_and(gi >= n_groups || im == imb);
    const ImgDesc *D = imgs + im;
    const int W = __ldg(&D->W), cpitch = __ldg(&D->cpitch);
    const uint64_t npx = (uint64_t)__ldg(&D->H) * (uint64_t)W;
    const uint64_t g0 = (uint64_t)(gi - __ldg(&D->pre_begin)) * 4;
    const bool active = gi < n_groups && g0 < npx;
    uint4 o0[4] = {}, o1[4] = {};
    if (active) {
        const uint4 r = ht_philox4x32_10(make_uint4((uint32_t)(g0 >> 2), __ldg(&D->image), 0u, 0u),
                                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        const uint32_t lanes[4] = {r.x, r.y, r.z, r.w};
        uint64_t y = g0 / (uint64_t)W;
        int x = (int)(g0 - y * (uint64_t)W);
        const float *__restrict__ contone = D->contone;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const float c = g0 + l < npx ? __ldg(contone + (size_t)y * cpitch + x) : 0.f;
            const float z = (float)(lanes[l] >> 8) * (1.0f / 16777216.0f);
            first_input_pixel(c, z, o0[l], o1[l]);
            if (++x == W) {
                x = 0;
                ++y;
            }
        }
    }
    uint4 *out = reinterpret_cast<uint4 *>(D->act[1]);
    if (one_image) {
        // 16-byte slot idx is stored at idx ^ ((idx >> 3) & 3): for the writes (idx = 4t + l)
        // eight consecutive threads then hit eight different slots modulo 8 (no bank
        // conflict), and the reads (consecutive idx) stay a permutation within 64 bytes
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int q = 4 * t + (l ^ ((t >> 1) & 3));
            s_out[0][q] = o0[l];
            s_out[1][q] = o1[l];
        }
        __syncthreads();
        const uint64_t gB = (uint64_t)(gb - __ldg(&imgs[imb].pre_begin)) * 4;   // the block's first pixel
        const uint64_t npxb = (uint64_t)__ldg(&imgs[imb].H) * (uint64_t)__ldg(&imgs[imb].W);
        uint4 *outb = reinterpret_cast<uint4 *>(imgs[imb].act[1]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int idx = t + 256 * k;
            const int q = idx ^ ((idx >> 3) & 3);
            const uint64_t g = gB + (uint64_t)idx;
            if (gb + idx / 4 < n_groups && g < npxb) {
                outb[g] = s_out[0][q];
                outb[npxb + g] = s_out[1][q];
            }
        }
    } else if (active) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            if (g0 + l >= npx) break;
            out[g0 + l] = o0[l];
            out[npx + g0 + l] = o1[l];
        }
    }
}


// ---------------------------------------------------------------------------
// 1-logit head from the per-tap partials written by the last conv layer:
// z(y,x) = b + sum_{dy,dx} d_{dy,dx}(y+dy-1, x+dx-1) (zero outside the image),
// then the sigmoid (or the multitoning prototype's level), the action and the packed
// output.  A block is a 128 x 8 tile: warp w takes row y0 + w, lane l the four pixels
// x0 + 4l .. x0 + 4l + 3.  Where W is a multiple of 4 (and the partials are 16-byte
// aligned) the four pixels are one aligned Philox group g = 4m: one Philox call gives their
// four uniforms, and each tap row is one float4 load, its neighbouring columns taken from
// the adjacent lanes.  Otherwise the pixels are read and drawn one by one.  The taps are
// summed in the same order either way (dy, then dx), a tap outside the image adding 0.
// ---------------------------------------------------------------------------
constexpr int HQ_W = 128;

__global__ void __launch_bounds__(HT_X *HT_Y) k_head_partials(const ImgDesc *__restrict__ imgs, int n_imgs, int buf,
                                                              float bias, int mode, uint64_t seed, int head, int levels)
{
    const int lane = threadIdx.x, warp = threadIdx.y;           // block (32, 8): one warp per row
    const int im = find_image(n_imgs, (int)blockIdx.x, [&](int i) { return __ldg(&imgs[i].hq_begin); });
    const ImgDesc *D = imgs + im;
    const int lt = (int)blockIdx.x - __ldg(&D->hq_begin);
    const int H = __ldg(&D->H), W = __ldg(&D->W);
    const int hx = (W + HQ_W - 1) / HQ_W;
    const int x0 = (lt % hx) * HQ_W, y = (lt / hx) * HT_Y + warp;
    if (y >= H) return;                                          // the whole warp
    const float *__restrict__ part = D->part ? D->part : (const float *)D->act[buf];
    const size_t plane = (size_t)H * W;
    const int xb = x0 + 4 * lane;
    const bool vec = (W & 3) == 0 && (((uintptr_t)part) & 15u) == 0;
    float z[4] = {bias, bias, bias, bias};
    if (vec) {
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const int yy = y + dy - 1;
            if (yy < 0 || yy >= H) continue;                     // uniform over the warp
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const float *row = part + (size_t)(dy * 3 + dx) * plane + (size_t)yy * W;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (xb < W) v = __ldg(reinterpret_cast<const float4 *>(row + xb));
                if (dx == 0) {
                    float left = __shfl_up_sync(0xffffffffu, v.w, 1);
                    if (lane == 0) left = x0 > 0 ? __ldg(row + x0 - 1) : 0.f;
                    z[0] += left;
                    z[1] += v.x;
                    z[2] += v.y;
                    z[3] += v.z;
                } else if (dx == 1) {
                    z[0] += v.x;
                    z[1] += v.y;
                    z[2] += v.z;
                    z[3] += v.w;
                } else {
                    float right = __shfl_down_sync(0xffffffffu, v.x, 1);
                    if (lane == 31) right = x0 + HQ_W < W ? __ldg(row + x0 + HQ_W) : 0.f;
                    z[0] += v.y;
                    z[1] += v.z;
                    z[2] += v.w;
                    z[3] += right;
                }
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int x = xb + c;
            if (x >= W) continue;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
                if (yy >= 0 && yy < H && xx >= 0 && xx < W) z[c] += __ldg(part + t * plane + (size_t)yy * W + xx);
            }
        }
    }
    // uniforms of the action draw (Philox stream 1), 0.5 where unused
    const uint32_t image = __ldg(&D->image);
    float u[4] = {0.5f, 0.5f, 0.5f, 0.5f};
    if (mode == HT_MODE_BERNOULLI) {
        const uint64_t g = (uint64_t)y * (uint64_t)W + (uint64_t)xb;
        if (vec) {
            if (xb < W) {
                const uint4 r = ht_philox4x32_10(make_uint4((uint32_t)(g >> 2), image, 1u, 0u),
                                                 make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
                u[0] = (float)(r.x >> 8) * (1.0f / 16777216.0f);
                u[1] = (float)(r.y >> 8) * (1.0f / 16777216.0f);
                u[2] = (float)(r.z >> 8) * (1.0f / 16777216.0f);
                u[3] = (float)(r.w >> 8) * (1.0f / 16777216.0f);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (xb + c < W) u[c] = ht_uniform24(seed, image, 1u, g + (uint64_t)c);
        }
    }
    float pv[4];
    uint32_t code = 0;                                           // this lane's 4 or 8 output bits
    const int words = __ldg(&D->words);
    uint32_t *bits = D->bits + (size_t)y * words;
    if (head == HT_HEAD_SIGMOID) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            pv[c] = 1.f / (1.f + expf(-z[c]));
            const bool hbit = (xb + c < W) && (mode == HT_MODE_BERNOULLI ? (u[c] < pv[c]) : (pv[c] > 0.5f));
            code |= (hbit ? 1u : 0u) << c;
        }
        // word x0 / 32 + l / 8 holds lanes l .. l + 7 (4 bits each, LSB first)
        uint32_t wv = code << (4 * (lane & 7));
        wv |= __shfl_xor_sync(0xffffffffu, wv, 1);
        wv |= __shfl_xor_sync(0xffffffffu, wv, 2);
        wv |= __shfl_xor_sync(0xffffffffu, wv, 4);
        if ((lane & 7) == 0 && xb < W) bits[(x0 >> 5) + (lane >> 3)] = wv;
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float v = 1.f / (1.f + expf(-z[c]));
            const float t = v * (float)(levels - 1);
            const int k = min((int)floorf(t), levels - 2);
            const float frac = t - (float)k;
            const int lev = k + ((mode == HT_MODE_BERNOULLI ? (u[c] < frac) : (frac > 0.5f)) ? 1 : 0);
            pv[c] = v;
            if (xb + c < W) code |= (uint32_t)lev << (2 * c);
        }
        // word x0 / 16 + l / 4 holds lanes l .. l + 3 (8 bits each, LSB first)
        uint32_t wv = code << (8 * (lane & 3));
        wv |= __shfl_xor_sync(0xffffffffu, wv, 1);
        wv |= __shfl_xor_sync(0xffffffffu, wv, 2);
        if ((lane & 3) == 0 && xb < W) bits[(x0 >> 4) + (lane >> 2)] = wv;
    }
    float *prob = D->prob;
    if (prob) {
        float *pr = prob + (size_t)y * W;
        if (vec && (((uintptr_t)prob) & 15u) == 0) {
            if (xb < W) *reinterpret_cast<float4 *>(pr + xb) = make_float4(pv[0], pv[1], pv[2], pv[3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (xb + c < W) pr[xb + c] = pv[c];
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <bool FP8, int KIND, bool TR = false, int CH = 64, bool F16 = false, bool STREAM = false, bool FUSED = false>
ht_status ensure_attr()
{
    static bool attr_set = false;
    if (!attr_set) {
        HT_CUDA_TRY(cudaFuncSetAttribute(k_conv_tc<FP8, KIND, TR, CH, F16, STREAM, FUSED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<FP8, KIND, CH, F16>::SMEM));
        attr_set = true;
    }
    return HT_OK;
}

template <bool FP8, int KIND>
ht_status ensure_attr2()
{
    static bool attr_set = false;
    if (!attr_set) {
        HT_CUDA_TRY(cudaFuncSetAttribute(k_conv_tc2<FP8, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg2<FP8>::SMEM));
        attr_set = true;
    }
    return HT_OK;
}

// CTA pairs that can be resident at once (1 CTA per SM; a pair needs two SMs of one GPC)
int max_pairs()
{
    static int n = 0;
    if (!n) {
        int clusters = 0;
        if (ensure_attr2<false, KIND_HIDDEN>() == HT_OK) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(2 * (num_sms() / 2), 1, 1);
            cfg.blockDim = dim3(NTHREADS, 1, 1);
            cfg.dynamicSmemBytes = Cfg2<false>::SMEM;
            if (cudaOccupancyMaxActiveClusters(&clusters, k_conv_tc2<false, KIND_HIDDEN>, &cfg) != cudaSuccess)
                clusters = 0;
        }
        cudaGetLastError();
        n = clusters > 0 ? clusters : (num_sms() / 2 > 0 ? num_sms() / 2 : 1);
    }
    return n;
}

// every kernel attribute set before a stream capture records the launches
ht_status ensure_all_attrs()
{
    ht_status st;
    if ((st = ensure_attr2<false, KIND_HIDDEN>()) != HT_OK || (st = ensure_attr2<false, KIND_HEADPART>()) != HT_OK ||
        (st = ensure_attr2<true, KIND_HIDDEN>()) != HT_OK || (st = ensure_attr2<true, KIND_HEADPART>()) != HT_OK)
        return st;
    max_pairs();
    if ((st = ensure_attr<false, KIND_HIDDEN>()) != HT_OK || (st = ensure_attr<false, KIND_HEADPART>()) != HT_OK ||
        (st = ensure_attr<false, KIND_FIRST>()) != HT_OK || (st = ensure_attr<false, KIND_HEAD4>()) != HT_OK ||
        (st = ensure_attr<true, KIND_HIDDEN>()) != HT_OK || (st = ensure_attr<true, KIND_HEADPART>()) != HT_OK ||
        (st = ensure_attr<true, KIND_FIRST>()) != HT_OK || (st = ensure_attr<false, KIND_HIDDEN, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_HEADPART, true>()) != HT_OK || (st = ensure_attr<false, KIND_FIRST, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_FIRST, false, 32>()) != HT_OK ||
        (st = ensure_attr<false, KIND_HIDDEN, false, 32>()) != HT_OK ||
        (st = ensure_attr<false, KIND_RES, false, 32>()) != HT_OK ||
        (st = ensure_attr<false, KIND_RESHEAD, false, 32>()) != HT_OK ||
        (st = ensure_attr<false, KIND_FIRST, false, 64, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_HIDDEN, false, 64, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_HEADPART, false, 64, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_HEAD4, false, 64, true>()) != HT_OK)
        return st;
    if ((st = ensure_attr<false, KIND_HIDDEN, false, 64, false, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_HEADPART, false, 64, false, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_FIRST, false, 64, false, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_HEAD4, false, 64, false, true>()) != HT_OK ||
        (st = ensure_attr<true, KIND_HIDDEN, false, 64, false, true>()) != HT_OK ||
        (st = ensure_attr<true, KIND_HEADPART, false, 64, false, true>()) != HT_OK ||
        (st = ensure_attr<true, KIND_FIRST, false, 64, false, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_FIRST, false, 64, true, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_HIDDEN, false, 64, true, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_HEADPART, false, 64, true, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_HEAD4, false, 64, true, true>()) != HT_OK)
        return st;
    if ((st = ensure_attr<false, KIND_FIRST, false, 64, false, false, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_FIRST, false, 64, false, true, true>()) != HT_OK ||
        (st = ensure_attr<true, KIND_FIRST, false, 64, false, false, true>()) != HT_OK ||
        (st = ensure_attr<true, KIND_FIRST, false, 64, false, true, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_FIRST, false, 64, true, false, true>()) != HT_OK ||
        (st = ensure_attr<false, KIND_FIRST, false, 64, true, true, true>()) != HT_OK)
        return st;
    return HT_OK;
}

template <bool FP8, int KIND, bool TR, int CH, bool F16, bool STREAM, bool FUSED = false>
ht_status launch_conv_k(const ConvParams &P, cudaStream_t s)
{
    const ht_status st = ensure_attr<FP8, KIND, TR, CH, F16, STREAM, FUSED>();
    if (st != HT_OK) return st;
    const int grid = P.n_units < num_sms() ? P.n_units : num_sms();
    ht_prof_start(KIND == KIND_FIRST ? HTK_FIRST_TC : KIND == KIND_HEAD4 ? HTK_HEAD_TC
                  : FP8 ? HTK_CONV_TC_FP8 : F16 ? HTK_CONV_TC_FP16 : HTK_CONV_TC_BF16, s);
    k_conv_tc<FP8, KIND, TR, CH, F16, STREAM, FUSED>
        <<<grid, FUSED ? NTHREADS_FUSED : NTHREADS_CONV, Cfg<FP8, KIND, CH, F16>::SMEM, s>>>(P);
    ht_prof_stop(s);
    HT_LAUNCH_CHECK();
    return HT_OK;
}

// Units of more than RU rows run as streaming strips (inference forms of the 64-wide
// architecture only); the 8-row form holds at most RU rows per unit.
template <bool FP8, int KIND, bool TR = false, int CH = 64, bool F16 = false>
ht_status launch_conv(const ConvParams &P, cudaStream_t s)
{
    if (P.ru < 1) return HT_ERR_INVALID_ARG;
    if (P.ru > RU) {
        if constexpr (!TR && CH == 64) return launch_conv_k<FP8, KIND, false, 64, F16, true>(P, s);
        return HT_ERR_INVALID_ARG;
    }
    return launch_conv_k<FP8, KIND, TR, CH, F16, false>(P, s);
}

// Layer 1 of the inference forms with its input built in the kernel (no input pass).
template <bool FP8, bool F16>
ht_status launch_first_fused(const ConvParams &P, cudaStream_t s)
{
    if (P.ru < 1) return HT_ERR_INVALID_ARG;
    if (P.ru > RU) return launch_conv_k<FP8, KIND_FIRST, false, 64, F16, true, true>(P, s);
    return launch_conv_k<FP8, KIND_FIRST, false, 64, F16, false, true>(P, s);
}

// CTA-pair form: P.n_units counts 256-pixel units (ImgDesc::unit2_begin), P.wpack
// holds both CTAs' weight images (CTA r at r * Cfg2::W_BYTES).
template <bool FP8, int KIND>
ht_status launch_conv2(const ConvParams &P, cudaStream_t s)
{
    const ht_status st = ensure_attr2<FP8, KIND>();
    if (st != HT_OK) return st;
    if (P.n_units <= 0) return HT_OK;
    const int pairs = P.n_units < max_pairs() ? P.n_units : max_pairs();
    ht_prof_start(FP8 ? HTK_CONV_TC_FP8 : HTK_CONV_TC_BF16, s);
    k_conv_tc2<FP8, KIND><<<2 * pairs, NTHREADS, Cfg2<FP8>::SMEM, s>>>(P);
    ht_prof_stop(s);
    HT_LAUNCH_CHECK();
    return HT_OK;
}

// Packs P.head_w ([9 taps][co]) into the tap-pair layout the fused head reads.
void fill_head_w2(ConvParams &P, int co)
{
    for (int n = 0; n < co; ++n)
        for (int t = 0; t < 4; ++t) {
            uint32_t lo, hi;
            memcpy(&lo, &P.head_w[(2 * t) * co + n], 4);
            memcpy(&hi, &P.head_w[(2 * t + 1) * co + n], 4);
            P.head_w2[n][t] = (unsigned long long)lo | ((unsigned long long)hi << 32);
        }
}

uint16_t f32_to_bf16_rne(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// round-to-nearest-even to OCP E4M3 (saturating), returns the encoded byte
uint8_t f64_to_e4m3_rne(double x)
{
    const uint8_t sign = x < 0 ? 0x80 : 0;
    double ax = fabs(x);
    if (ax == 0.0) return sign;
    double q;
    if (ax < ldexp(1.0, -6)) {
        q = ldexp(1.0, -9);
    } else {
        int e;
        frexp(ax, &e);
        q = ldexp(1.0, e - 4);
    }
    double r = nearbyint(ax / q) * q;
    if (r > 448.0) r = 448.0;
    if (r < ldexp(1.0, -6)) {                      // subnormal (or rounded up to the min normal below)
        const int m = (int)nearbyint(r / ldexp(1.0, -9));
        if (m < 8) return sign | (uint8_t)m;
    }
    int e;
    const double fr = frexp(r, &e);                // r = fr * 2^e, fr in [0.5, 1)
    const int exp_field = e - 1 + 7;
    const int mant = (int)nearbyint((fr * 2.0 - 1.0) * 8.0);
    return sign | (uint8_t)(exp_field << 3) | (uint8_t)mant;
}

}  // namespace

uint16_t f32_to_f16_rne_host(float f)
{
    const __half h = __float2half_rn(f);
    uint16_t b;
    memcpy(&b, &h, 2);
    return b;
}
float f16_to_f32_host(uint16_t b)
{
    __half h;
    memcpy(&h, &b, 2);
    return __half2float(h);
}

ht_status ht_pack_tc_weights(ht_policy *p, cudaStream_t s)
{
    const bool fp8 = (p->prec == HT_FP8_E4M3);
    const bool f16 = (p->prec == HT_FP16);
    const int CH = p->width;                                   // hidden width (64, or 32 for the residual policy)
    const int cpc = fp8 ? 16 : 8, nchunk = CH / cpc;
    const size_t layer_bytes = (size_t)9 * nchunk * CH * 16;
    const int n_inner = p->L - 2;
    p->wpack_layer_bytes = layer_bytes;
    if (!p->d_wpack) HT_CUDA_TRY(cudaMalloc(&p->d_wpack, layer_bytes * n_inner));
    if (fp8 && !p->d_wscale) HT_CUDA_TRY(cudaMalloc((void **)&p->d_wscale, sizeof(float) * 64 * n_inner));
    // pull the current fp32 weights of the inner layers to the host
    const size_t nw = (size_t)CH * CH * 9;
    float *hw = (float *)malloc(sizeof(float) * nw * n_inner);
    uint8_t *hp = (uint8_t *)malloc(layer_bytes * n_inner);
    float *hs = (float *)malloc(sizeof(float) * 64 * n_inner);
    if (!hw || !hp || !hs) {
        free(hw);
        free(hp);
        free(hs);
        return HT_ERR_OOM;
    }
    cudaError_t e = cudaMemcpyAsync(hw, p->d_w + p->w_off[1], sizeof(float) * nw * n_inner, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free(hw);
        free(hp);
        free(hs);
        HT_CUDA_TRY(e);
    }
    for (int l = 0; l < n_inner; ++l) {
        const float *W = hw + nw * l;     // [n][c][3][3]
        uint8_t *dst = hp + layer_bytes * l;
        for (int n = 0; n < CH; ++n) {
            double sc = 1.0;
            if (fp8) {
                double amax = 0.0;
                for (int k = 0; k < CH * 9; ++k) amax = fmax(amax, fabs((double)W[(size_t)n * CH * 9 + k]));
                sc = amax > 0.0 ? amax / 448.0 : 1.0;
                hs[64 * l + n] = (float)sc;
            }
            for (int tap = 0; tap < 9; ++tap)
                for (int c = 0; c < CH; ++c) {
                    const float wv = W[((size_t)n * CH + c) * 9 + tap];
                    const int dy = tap / 3, dx = tap % 3;
                    const size_t off = ((((size_t)dx * nchunk + c / cpc) * 3 + (2 - dy)) * CH + n) * 16;
                    if (fp8) {
                        dst[off + (c % cpc)] = f64_to_e4m3_rne((double)wv / sc);
                    } else if (f16) {
                        const uint16_t b = f32_to_f16_rne_host(wv);
                        memcpy(dst + off + 2 * (c % cpc), &b, 2);
                    } else {
                        const uint16_t b = f32_to_bf16_rne(wv);
                        memcpy(dst + off + 2 * (c % cpc), &b, 2);
                    }
                }
        }
    }
    {
        // layer 1: B = [dx][chunk 2][3 dy][CH n][8 bf16]; per tap, K elements
        // k = 6 ci + j (ci = 0 for c, 1 for z) hold (w0, w1, w0, w2, w1, w0) of the exact
        // three-part bf16 split w = w0 + w1 + w2, k = 12..15 zero (the pairing of
        // k_first_input's (v0, v0, v1, v0, v1, v2))
        float w0[64 * 2 * 9];
        e = cudaMemcpyAsync(w0, p->d_w + p->w_off[0], sizeof(float) * CH * 2 * 9, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        uint16_t pk[3 * 2 * 3 * 64 * 8];
        memset(pk, 0, sizeof(pk));
        for (int n = 0; n < CH; ++n)
            for (int tap = 0; tap < 9; ++tap)
                for (int ci = 0; ci < 2; ++ci) {
                    const int dy = tap / 3, dx = tap % 3;
                    const float w = w0[(n * 2 + ci) * 9 + tap];
                    uint16_t part[3];
                    float rest = w;
                    for (int q = 0; q < 3; ++q) {            // exact: each remainder fits float32
                        part[q] = f32_to_bf16_rne(rest);
                        const uint32_t b32 = (uint32_t)part[q] << 16;
                        float pf;
                        memcpy(&pf, &b32, 4);
                        rest -= pf;
                    }
                    const uint16_t six[6] = {part[0], part[1], part[0], part[2], part[1], part[0]};
                    for (int j = 0; j < 6; ++j) {
                        const int k = 6 * ci + j;
                        pk[(((dx * 2 + k / 8) * 3 + (2 - dy)) * CH + n) * 8 + k % 8] = six[j];
                    }
                }
        if (e == cudaSuccess && !p->d_w1pack) e = cudaMalloc(&p->d_w1pack, sizeof(pk));
        if (e == cudaSuccess) e = cudaMemcpy(p->d_w1pack, pk, sizeof(pk), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free(hw);
            free(hp);
            free(hs);
            HT_CUDA_TRY(e);
        }
    }
    // biases and (1-logit head) last-layer weights, host side, for the kernel parameters
    e = cudaMemcpyAsync(p->h_b, p->d_b, sizeof(float) * p->n_b, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && p->K == 1)
        e = cudaMemcpyAsync(p->h_headw, p->d_w + p->w_off[p->L - 1], sizeof(float) * CH * 9, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free(hw);
        free(hp);
        free(hs);
        HT_CUDA_TRY(e);
    }
    if (p->K == 1) {
        float tmp[9 * 64];
        memcpy(tmp, p->h_headw, sizeof(float) * 9 * CH);      // [c][tap] -> [tap][c]
        for (int c = 0; c < CH; ++c)
            for (int t = 0; t < 9; ++t) p->h_headw[t * CH + c] = tmp[c * 9 + t];
        p->head_bias = p->h_b[p->b_off[p->L - 1]];
    }
    if (fp8) memcpy(p->h_wscale, hs, sizeof(float) * 64 * n_inner);
    if (p->K == 4) {
        float wl[4 * 64 * 9];
        e = cudaMemcpyAsync(wl, p->d_w + p->w_off[p->L - 1], sizeof(wl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        const size_t part = (size_t)3 * 8 * 3 * 16 * 8;          // 16-bit elements
        std::vector<uint16_t> pk(part, 0);
        // FP16 form: binary16 hi / lo parts of w x 2^k, with 2^k putting the largest |w| near
        // 2^14 (the parts stay normal binary16 numbers); the logits are multiplied by 2^-k
        float wsc = 1.f;
        p->head4_inv_scale = 1.f;
        if (f16) {
            float amax = 0.f;
            for (int k = 0; k < 4 * 64 * 9; ++k) amax = fmaxf(amax, fabsf(wl[k]));
            int k2 = amax > 0.f ? (int)floor(log2(16384.0 / amax)) : 0;
            k2 = k2 < -14 ? -14 : k2 > 24 ? 24 : k2;
            wsc = ldexpf(1.f, k2);
            p->head4_inv_scale = ldexpf(1.f, -k2);
        }
        for (int n = 0; n < 4; ++n)
            for (int c = 0; c < 64; ++c)
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap % 3;
                    const float w = wl[(n * 64 + c) * 9 + tap] * wsc;
                    uint16_t hi, lo;
                    if (f16) {
                        hi = f32_to_f16_rne_host(w);
                        lo = f32_to_f16_rne_host(w - f16_to_f32_host(hi));
                    } else {
                        hi = f32_to_bf16_rne(w);
                        uint32_t hb32 = (uint32_t)hi << 16;
                        float hf;
                        memcpy(&hf, &hb32, 4);
                        lo = f32_to_bf16_rne(w - hf);
                    }
                    // columns n (hi part) and 4 + n (lo part) of the 16-column dy block
                    const size_t off = ((((size_t)dx * 8 + c / 8) * 3 + (2 - dy)) * 16 + n) * 8 + (c % 8);
                    pk[off] = hi;
                    pk[off + 4 * 8] = lo;
                }
        if (e == cudaSuccess && !p->d_wpack4) e = cudaMalloc(&p->d_wpack4, pk.size() * 2);
        if (e == cudaSuccess) e = cudaMemcpy(p->d_wpack4, pk.data(), pk.size() * 2, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free(hw);
            free(hp);
            free(hs);
            HT_CUDA_TRY(e);
        }
    }
    e = cudaMemcpyAsync(p->d_wpack, hp, layer_bytes * n_inner, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && fp8) e = cudaMemcpyAsync(p->d_wscale, hs, sizeof(float) * 64 * n_inner, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && CH == 64 && n_inner > 0 && !f16) {
        // CTA-pair images (BF16 and FP8 forms): for CTA r, per (dx, K step) group, variant v's rows
        // [r n/2, (r+1) n/2) of its stacked column range, both 16-byte K chunks
        const int ksteps = nchunk / 2;
        const size_t wb = (size_t)3 * ksteps * PV_GROUP_BYTES;     // one CTA's image of one layer
        p->wpack2_layer_bytes = 2 * wb;
        std::vector<uint8_t> h2(p->wpack2_layer_bytes * n_inner);
        for (int l = 0; l < n_inner; ++l)
            for (int r = 0; r < 2; ++r)
                for (int dx = 0; dx < 3; ++dx)
                    for (int ks = 0; ks < ksteps; ++ks)
                        for (int v = 0; v < 6; ++v) {
                            const int half = pv_n(v) / 2;
                            for (int c = 0; c < 2; ++c)
                                for (int row = 0; row < half; ++row) {
                                    const int col = pv_start(v) + r * half + row;    // in [dy=2 | dy=1 | dy=0]
                                    const size_t src = layer_bytes * l +
                                        ((((size_t)dx * nchunk + 2 * ks + c) * 3 + col / 64) * CH + col % 64) * 16;
                                    const size_t dst = p->wpack2_layer_bytes * l + wb * r +
                                        (size_t)(dx * ksteps + ks) * PV_GROUP_BYTES + (size_t)pv_row(v) * 32 +
                                        (size_t)c * half * 16 + (size_t)row * 16;
                                    memcpy(&h2[dst], hp + src, 16);
                                }
                        }
        if (!p->d_wpack2) e = cudaMalloc(&p->d_wpack2, h2.size());
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_wpack2, h2.data(), h2.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    free(hw);
    free(hp);
    free(hs);
    HT_CUDA_TRY(e);
    ++p->version;
    return HT_OK;
}

size_t ht_tc_ws_bytes(const ht_policy *p, int h, int w)
{
    (void)p;
    // two ping-pong buffers of 64 bf16 channels (the FP8 form stores e4m3 in the same space)
    return 2 * (size_t)h * w * 64 * 2;
}

namespace {
// Activation workspace of one group of images: HT_WS_BUDGET_GB if set, else a quarter of
// the device's memory (at least 16 GB), so that large uneven batches run as one group of
// persistent launches instead of several, each with its own partial last wave.
size_t ws_budget()
{
    static size_t b = 0;
    if (!b) {
        const char *e = getenv("HT_WS_BUDGET_GB");
        double gb = 16.0;
        if (e) {
            gb = atof(e);
        } else {
            int dev = 0;
            size_t total = 0;
            if (cudaGetDevice(&dev) == cudaSuccess) {
                cudaDeviceProp prop;
                if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) total = prop.totalGlobalMem;
            }
            cudaGetLastError();
            const double quarter = (double)total / 4.0 / 1073741824.0;
            gb = quarter > gb ? quarter : gb;
        }
        b = (size_t)((gb > 0.5 ? gb : 0.5) * 1073741824.0);
    }
    return b;
}
}  // namespace

size_t img_ws_slot(const ht_policy *p, const ht_image &img)
{
    return (ht_tc_ws_bytes(p, img.h, img.w) + 255) / 256 * 256;
}

size_t ht_tc_batch_ws_bytes(const ht_policy *p, const ht_image *imgs, int n)
{
    size_t maxg = 0, cur = 0;
    for (int i = 0; i < n; ++i) {
        const size_t b = img_ws_slot(p, imgs[i]);
        if (cur > 0 && cur + b > ws_budget()) {      // same grouping rule as ht_run_tc_batch
            maxg = cur > maxg ? cur : maxg;
            cur = 0;
        }
        cur += b;
    }
    maxg = cur > maxg ? cur : maxg;
    return maxg + (size_t)n * sizeof(ImgDesc) + 1024;
}

// Loads every kernel of this file (see ht_preload_kernels).
void ht_preload_conv_tc()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HIDDEN>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HEADPART>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_FIRST>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HEAD4>);
    cudaFuncGetAttributes(&fa, k_conv_tc<true, KIND_HIDDEN>);
    cudaFuncGetAttributes(&fa, k_conv_tc<true, KIND_HEADPART>);
    cudaFuncGetAttributes(&fa, k_conv_tc<true, KIND_FIRST>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HIDDEN, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HEADPART, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_FIRST, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_FIRST, false, 32>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HIDDEN, false, 32>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_RES, false, 32>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_RESHEAD, false, 32>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_FIRST, false, 64, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HIDDEN, false, 64, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HEADPART, false, 64, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HEAD4, false, 64, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HIDDEN, false, 64, false, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HEADPART, false, 64, false, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_FIRST, false, 64, false, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HEAD4, false, 64, false, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<true, KIND_HIDDEN, false, 64, false, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<true, KIND_HEADPART, false, 64, false, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<true, KIND_FIRST, false, 64, false, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_FIRST, false, 64, true, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HIDDEN, false, 64, true, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HEADPART, false, 64, true, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_HEAD4, false, 64, true, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_FIRST, false, 64, false, false, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_FIRST, false, 64, false, true, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<true, KIND_FIRST, false, 64, false, false, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<true, KIND_FIRST, false, 64, false, true, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_FIRST, false, 64, true, false, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc<false, KIND_FIRST, false, 64, true, true, true>);
    cudaFuncGetAttributes(&fa, k_conv_tc2<false, KIND_HIDDEN>);
    cudaFuncGetAttributes(&fa, k_conv_tc2<false, KIND_HEADPART>);
    cudaFuncGetAttributes(&fa, k_conv_tc2<true, KIND_HIDDEN>);
    cudaFuncGetAttributes(&fa, k_conv_tc2<true, KIND_HEADPART>);
    cudaFuncGetAttributes(&fa, k_first_input);
    cudaFuncGetAttributes(&fa, k_head_partials);
    ensure_all_attrs();
}

ht_status ht_tc_conv(const ht_tc_layer &a, cudaStream_t s)
{
    int *err = ht_device_error_flag();
    if (!err) return HT_ERR_CUDA;
    ConvParams P{};
    P.imgs = (const ImgDesc *)a.table;
    P.n_imgs = a.n_imgs;
    P.n_units = a.n_units;
    P.in_buf = a.in_buf;
    P.wpack = a.wpack;
    for (int c = 0; c < 64; ++c) {
        P.scale[c] = a.scale ? a.scale[c] : 1.f;
        P.bias[c] = a.bias ? a.bias[c] : 0.f;
    }
    if (a.head_w) {
        memcpy(P.head_w, a.head_w, sizeof(P.head_w));
        fill_head_w2(P, 64);
    }
    P.out_inv_scale = 1.f;
    P.out_fp8 = 0;
    P.seed = a.seed;
    P.dgrad = a.dgrad;
    P.ru = RU;
    P.order = 0;
    P.err = err;
    switch (a.kind) {
    case KIND_HIDDEN: return launch_conv<false, KIND_HIDDEN, true>(P, s);
    case KIND_HEADPART: return launch_conv<false, KIND_HEADPART, true>(P, s);
    case KIND_FIRST: return launch_conv<false, KIND_FIRST, true>(P, s);
    default: ht_set_error("ht_tc_conv: bad kind %d", a.kind); return HT_ERR_INVALID_ARG;
    }
}

ht_status ht_tc_first_input(const void *table, int n_imgs, int n_groups, uint64_t seed, cudaStream_t s)
{
    ht_prof_start(HTK_FIRST_INPUT, s);
    if (n_groups <= 0) return HT_OK;
    k_first_input<<<(n_groups + 255) / 256, 256, 0, s>>>((const ImgDesc *)table, n_imgs, n_groups, seed);
    ht_prof_stop(s);
    HT_LAUNCH_CHECK();
    return HT_OK;
}

ht_status ht_tc_head_partials(const void *table, int n_imgs, int n_tiles, int buf, float bias, int mode,
                              uint64_t seed, cudaStream_t s)
{
    ht_prof_start(HTK_HEAD_TC, s);
    k_head_partials<<<n_tiles, dim3(HT_X, HT_Y), 0, s>>>((const ImgDesc *)table, n_imgs, buf, bias, mode, seed,
                                                         HT_HEAD_SIGMOID, 2);
    ht_prof_stop(s);
    HT_LAUNCH_CHECK();
    return HT_OK;
}

namespace {
// One group of a call's images: their activation buffers fit the workspace
// budget together; each group is one launch per layer over all its images.
struct TcGroup {
    int g0, ng, units, hd, pre;
    int units2;                 // conv units of the CTA-pair form (256-pixel tiles)
    int hq;                     // 128 x 8 tiles of k_head_partials
};

// Host side of a call: the image tables (into `tab`, one entry per image, in call
// order) and the groups.  Activations of every group start at `ws`.
void tc_make_groups(const ht_policy *p, const ht_image *imgs, int n, uint8_t *ws, int ru, uint32_t *const *bits,
                    float *const *prob, std::vector<ImgDesc> &tab, std::vector<TcGroup> &groups)
{
    tab.assign(n, ImgDesc{});
    groups.clear();
    int g0 = 0;
    while (g0 < n) {
        TcGroup G{};
        G.g0 = g0;
        int g1 = g0;
        size_t off = 0;
        while (g1 < n) {
            const size_t b = ht_tc_ws_bytes(p, imgs[g1].h, imgs[g1].w);
            if (g1 > g0 && off + img_ws_slot(p, imgs[g1]) > ws_budget()) break;
            ImgDesc &D = tab[g1];
            D.contone = imgs[g1].contone;
            D.cpitch = imgs[g1].pitch;
            D.H = imgs[g1].h;
            D.W = imgs[g1].w;
            D.act[0] = ws + off;
            D.act[1] = D.act[0] + b / 2;
            off += img_ws_slot(p, imgs[g1]);
            D.bits = bits[g1];
            D.prob = prob ? prob[g1] : nullptr;
            D.words = ht_bits_row_words(D.W, p->head);
            D.image = (uint32_t)g1;
            if (p->arch == HT_ARCH_RESNET)   // 32-wide buffers use half of each 128 B/px slot
                D.part = (float *)(D.act[1] + (size_t)D.H * D.W * 64);
            set_begins(D, G.units, G.hd, G.pre, ru, &G.units2, &G.hq);
            ++g1;
        }
        G.ng = g1 - g0;
        groups.push_back(G);
        g0 = g1;
    }
}

// Device side of a call: per group, layer 1 (input pass + pipeline), the 64 -> 64
// layers and the head.  Kernel launches only (no copies, no allocation), so the
// sequence can be captured into a CUDA graph.
ht_status tc_launch_groups(ht_policy *p, const ImgDesc *d_table, const std::vector<TcGroup> &groups, int mode,
                           uint64_t seed, int ru, int order, int pair, int *err, cudaStream_t s)
{
    const bool fp8 = (p->prec == HT_FP8_E4M3);
    const bool f16 = (p->prec == HT_FP16);
    pair = pair && p->d_wpack2 && p->arch != HT_ARCH_RESNET && !f16 && ru <= RU;
    const int n_inner = p->L - 2;
    for (const TcGroup &G : groups) {
        const ImgDesc *dt = d_table + G.g0;
        const int ng = G.ng;
        if (p->arch == HT_ARCH_RESNET) {           // the 64-wide layer 1 builds its input itself
            ht_prof_start(HTK_FIRST_INPUT, s);
            k_first_input<<<(G.pre + 255) / 256, 256, 0, s>>>(dt, ng, G.pre, seed);
            ht_prof_stop(s);
            HT_LAUNCH_CHECK();
        }
        auto base = [&](ConvParams &P, int in_buf) {
            P.imgs = dt;
            P.n_imgs = ng;
            P.n_units = G.units;
            P.in_buf = in_buf;
            P.ru = ru;
            P.order = order;
            P.seed = seed;
            P.mode = mode;
            P.err = err;
        };
        {
            const bool o8 = fp8 && n_inner > 0;
            ConvParams P{};
            base(P, 1);                            // writes act[0] (the residual form reads the split input in act[1])
            P.wpack = p->d_w1pack;
            for (int c = 0; c < 64; ++c) {
                P.bias[c] = p->h_b[p->b_off[0] + c];
                P.scale[c] = 1.f;
            }
            P.out_inv_scale = o8 ? 1.f / p->act_scale[1] : 1.f;
            P.out_fp8 = o8 ? 1 : 0;
            const ht_status st = p->arch == HT_ARCH_RESNET ? launch_conv<false, KIND_FIRST, false, 32>(P, s)
                                 : fp8                      ? launch_first_fused<true, false>(P, s)
                                 : f16                      ? launch_first_fused<false, true>(P, s)
                                                            : launch_first_fused<false, false>(P, s);
            if (st != HT_OK) return st;
        }
        if (p->arch == HT_ARCH_RESNET) {
            // residual blocks: conv1 x (act[0]) -> t (act[1]); conv2 t -> y, shortcut x, in place in act[0]
            const int nb = n_inner / 2;
            for (int b = 0; b < nb; ++b) {
                for (int half = 0; half < 2; ++half) {
                    const int l = 1 + 2 * b + half;
                    ConvParams P{};
                    base(P, half);
                    P.wpack = (const uint8_t *)p->d_wpack + p->wpack_layer_bytes * (l - 1);
                    for (int c = 0; c < 32; ++c) {
                        P.bias[c] = p->h_b[p->b_off[l] + c];
                        P.scale[c] = 1.f;
                    }
                    P.out_inv_scale = 1.f;
                    ht_status st;
                    if (half == 0) {
                        st = launch_conv<false, KIND_HIDDEN, false, 32>(P, s);
                    } else if (b + 1 < nb) {
                        st = launch_conv<false, KIND_RES, false, 32>(P, s);
                    } else {
                        memcpy(P.head_w, p->h_headw, sizeof(float) * 9 * 32);
                        fill_head_w2(P, 32);
                        st = launch_conv<false, KIND_RESHEAD, false, 32>(P, s);
                    }
                    if (st != HT_OK) return st;
                }
            }
            ht_prof_start(HTK_HEAD_TC, s);
            k_head_partials<<<G.hq, dim3(HT_X, HT_Y), 0, s>>>(dt, ng, 0, p->head_bias, mode, seed, p->head, p->levels);
            ht_prof_stop(s);
            HT_LAUNCH_CHECK();
            continue;
        }
        int cur = 0;
        for (int l = 1; l <= n_inner; ++l) {
            const bool out8 = fp8 && (l < n_inner);
            const bool fuse_head = (l == n_inner) && p->K == 1;
            ConvParams P{};
            base(P, cur);
            P.wpack = (const uint8_t *)p->d_wpack + p->wpack_layer_bytes * (l - 1);
            for (int c = 0; c < 64; ++c) {
                P.bias[c] = p->h_b[p->b_off[l] + c];
                P.scale[c] = fp8 ? p->act_scale[l] * p->h_wscale[64 * (l - 1) + c] : 1.f;
            }
            if (fuse_head) {
                memcpy(P.head_w, p->h_headw, sizeof(P.head_w));
                fill_head_w2(P, 64);
            }
            P.out_inv_scale = out8 ? 1.f / p->act_scale[l + 1] : 1.f;
            P.out_fp8 = out8 ? 1 : 0;
            if (pair) {
                P.n_units = G.units2;
                P.wpack = (const uint8_t *)p->d_wpack2 + p->wpack2_layer_bytes * (l - 1);
                const ht_status st =
                    fp8 ? (fuse_head ? launch_conv2<true, KIND_HEADPART>(P, s) : launch_conv2<true, KIND_HIDDEN>(P, s))
                        : (fuse_head ? launch_conv2<false, KIND_HEADPART>(P, s) : launch_conv2<false, KIND_HIDDEN>(P, s));
                if (st != HT_OK) return st;
                cur ^= 1;
                continue;
            }
            const ht_status st =
                fp8   ? (fuse_head ? launch_conv<true, KIND_HEADPART>(P, s) : launch_conv<true, KIND_HIDDEN>(P, s))
                : f16 ? (fuse_head ? launch_conv<false, KIND_HEADPART, false, 64, true>(P, s)
                                   : launch_conv<false, KIND_HIDDEN, false, 64, true>(P, s))
                      : (fuse_head ? launch_conv<false, KIND_HEADPART>(P, s) : launch_conv<false, KIND_HIDDEN>(P, s));
            if (st != HT_OK) return st;
            cur ^= 1;
        }
        if (p->K == 1) {
            ht_prof_start(HTK_HEAD_TC, s);
            k_head_partials<<<G.hq, dim3(HT_X, HT_Y), 0, s>>>(dt, ng, cur, p->head_bias, mode, seed, p->head,
                                                              p->levels);
            ht_prof_stop(s);
            HT_LAUNCH_CHECK();
        } else {
            ConvParams P{};
            base(P, cur);
            P.wpack = p->d_wpack4;
            for (int c = 0; c < 64; ++c) {
                P.bias[c] = c < 4 ? p->h_b[p->b_off[p->L - 1] + c] : 0.f;
                P.scale[c] = c < 4 ? p->head4_inv_scale : 1.f;
            }
            P.out_inv_scale = 1.f;
            P.out_fp8 = 0;
            const ht_status st = f16 ? launch_conv<false, KIND_HEAD4, false, 64, true>(P, s)
                                     : launch_conv<false, KIND_HEAD4>(P, s);
            if (st != HT_OK) return st;
        }
    }
    return HT_OK;
}
}  // namespace

// All images of a call: grouped so that a group's activation buffers fit the
// workspace budget; per group one launch of layer 1, one per 64 -> 64 layer and
// one of the head, each over the whole group (persistent tile index space).
ht_status ht_run_tc_batch(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed,
                          uint32_t *const *bits, float *const *prob, cudaStream_t s)
{
    int *err = ht_device_error_flag();
    if (!err) return HT_ERR_CUDA;
    // table slots after the activation region (one slot per image, never reused within a call)
    const size_t need = ht_tc_batch_ws_bytes(p, imgs, n);
    if (need > p->ws_bytes) {
        ht_set_error("workspace too small");
        return HT_ERR_INVALID_ARG;
    }
    ImgDesc *d_table = (ImgDesc *)((uint8_t *)p->d_ws + (need - (size_t)n * sizeof(ImgDesc) - 512) / 256 * 256);
    std::vector<ImgDesc> tab;
    std::vector<TcGroup> groups;
    tc_make_groups(p, imgs, n, (uint8_t *)p->d_ws, p->tune_ru, bits, prob, tab, groups);
    HT_CUDA_TRY(cudaMemcpyAsync(d_table, tab.data(), sizeof(ImgDesc) * n, cudaMemcpyHostToDevice, s));
    return tc_launch_groups(p, d_table, groups, mode, seed, p->tune_ru, p->tune_order, p->tune_pair, err, s);
}

// ---------------------------------------------------------------------------
// Plans: one call's launch sequence captured once into a CUDA graph.
// ---------------------------------------------------------------------------
struct ht_plan {
    ht_policy *p = nullptr;
    int n = 0, mode = 0, ru = RU, order = 0, pair = 0;
    uint64_t seed = 0;
    uint64_t version = 0;                 // policy weight version the graph was captured with
    std::vector<ht_image> imgs;
    std::vector<uint32_t *> bits;
    std::vector<float *> prob;
    void *ws = nullptr;                   // plan-owned activations and image table
    ImgDesc *d_table = nullptr;
    std::vector<TcGroup> groups;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {
void plan_release_graph(ht_plan *pl)
{
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    pl->exec = nullptr;
    pl->graph = nullptr;
}

ht_status plan_capture(ht_plan *pl)
{
    plan_release_graph(pl);
    int *err = ht_device_error_flag();
    if (!err) return HT_ERR_CUDA;
    ht_status st = ensure_all_attrs();
    if (st != HT_OK) return st;
    cudaStream_t cs = nullptr;
    HT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = tc_launch_groups(pl->p, pl->d_table, pl->groups, pl->mode, pl->seed, pl->ru, pl->order, pl->pair, err, cs);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &pl->graph);
        if (st == HT_OK && e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && st == HT_OK) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    cudaStreamDestroy(cs);
    if (st != HT_OK) {
        plan_release_graph(pl);
        return st;
    }
    if (e != cudaSuccess) {
        plan_release_graph(pl);
        HT_CUDA_TRY(e);
    }
    pl->version = pl->p->version;
    return HT_OK;
}
}  // namespace

ht_status ht_plan_create_impl(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed,
                              uint32_t *const *bits, float *const *prob, ht_plan **out)
{
    if (p->prec == HT_FP32) {
        ht_set_error("plans capture the tensor-core forms (BF16, FP8)");
        return HT_ERR_UNSUPPORTED;
    }
    ht_plan *pl = new ht_plan();
    pl->p = p;
    pl->n = n;
    pl->mode = mode;
    pl->seed = seed;
    pl->ru = p->tune_ru;
    pl->order = p->tune_order;
    pl->pair = p->tune_pair;
    pl->imgs.assign(imgs, imgs + n);
    pl->bits.assign(bits, bits + n);
    if (prob) pl->prob.assign(prob, prob + n);
    const size_t need = ht_tc_batch_ws_bytes(p, imgs, n);
    cudaError_t e = cudaMalloc(&pl->ws, need);
    if (e != cudaSuccess) {
        delete pl;
        ht_set_error("plan workspace: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? HT_ERR_OOM : HT_ERR_CUDA;
    }
    pl->d_table = (ImgDesc *)((uint8_t *)pl->ws + (need - (size_t)n * sizeof(ImgDesc) - 512) / 256 * 256);
    std::vector<ImgDesc> tab;
    tc_make_groups(p, imgs, n, (uint8_t *)pl->ws, pl->ru, pl->bits.data(), prob ? pl->prob.data() : nullptr, tab,
                   pl->groups);
    e = cudaMemcpy(pl->d_table, tab.data(), sizeof(ImgDesc) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        ht_plan_destroy_impl(pl);
        HT_CUDA_TRY(e);
    }
    const ht_status st = plan_capture(pl);
    if (st != HT_OK) {
        ht_plan_destroy_impl(pl);
        return st;
    }
    *out = pl;
    return HT_OK;
}

ht_status ht_plan_launch_impl(ht_plan *pl, cudaStream_t s)
{
    if (pl->version != pl->p->version) {            // weights, scales or biases changed: capture again
        const ht_status st = plan_capture(pl);
        if (st != HT_OK) return st;
    }
    HT_CUDA_TRY(cudaGraphLaunch(pl->exec, s));
    return HT_OK;
}

ht_status ht_plan_destroy_impl(ht_plan *pl)
{
    if (!pl) return HT_OK;
    plan_release_graph(pl);
    cudaFree(pl->ws);
    delete pl;
    return HT_OK;
}

// Autotuner: times every unit geometry on the caller's own call and keeps the fastest.
ht_status ht_tc_autotune(ht_policy *p, const ht_image *imgs, int n, int mode, uint64_t seed, uint32_t *const *bits,
                         float *const *prob, int reps, ht_tune_result *out, int max_out, int *n_out, cudaStream_t s)
{
    // 8-row units (8, 6, 4 rows), streaming strips (32, 64, 128 rows; 64-wide architecture),
    // CTA pairs (64-wide architecture with a pair weight image)
    static const int cand[][3] = {{8, 0, 0},  {8, 1, 0},  {6, 0, 0},  {6, 1, 0},  {4, 0, 0}, {4, 1, 0},
                                  {32, 0, 0}, {32, 1, 0}, {64, 0, 0}, {64, 1, 0}, {128, 0, 0}, {128, 1, 0},
                                  {8, 0, 1},  {8, 1, 1},  {6, 0, 1},  {6, 1, 1},  {4, 0, 1}, {4, 1, 1}};
    const bool plain = p->arch != HT_ARCH_RESNET;
    int idx[18], nc = 0;
    for (int c = 0; c < 18; ++c)
        if ((cand[c][0] <= RU || plain) && (!cand[c][2] || (plain && p->d_wpack2))) idx[nc++] = c;
    cudaEvent_t e0, e1;
    HT_CUDA_TRY(cudaEventCreate(&e0));
    HT_CUDA_TRY(cudaEventCreate(&e1));
    const int keep_ru = p->tune_ru, keep_order = p->tune_order, keep_pair = p->tune_pair;
    float best = 1e30f;
    int bi = 0, k_out = 0;
    ht_status st = HT_OK;
    for (int ci = 0; ci < nc && st == HT_OK; ++ci) {
        const int c = idx[ci];
        p->tune_ru = cand[c][0];
        p->tune_order = cand[c][1];
        p->tune_pair = cand[c][2];
        st = ht_run_tc_batch(p, imgs, n, mode, seed, bits, prob, s);       // warm-up
        if (st != HT_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == HT_OK; ++r) st = ht_run_tc_batch(p, imgs, n, mode, seed, bits, prob, s);
        cudaEventRecord(e1, s);
        if (st != HT_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = HT_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
        if (out && k_out < max_out) {
            out[k_out].rows_per_unit = cand[c][0];
            out[k_out].unit_order = cand[c][1];
            out[k_out].cta_pair = cand[c][2];
            out[k_out].ms = ms;
            ++k_out;
        }
        if (ms < best) {
            best = ms;
            bi = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HT_OK) {
        p->tune_ru = keep_ru;
        p->tune_order = keep_order;
        p->tune_pair = keep_pair;
        return st;
    }
    p->tune_ru = cand[bi][0];
    p->tune_order = cand[bi][1];
    p->tune_pair = cand[bi][2];
    if (n_out) *n_out = k_out;
    return HT_OK;
}
