// tc_common.cuh -- pieces shared by the tcgen05 kernels (forward conv
// pipeline, weight-gradient pipeline): inline-PTX wrappers for mbarriers, bulk
// async copies, TMEM and tcgen05.mma; bf16 / e4m3 packing; the chunk-planar
// activation store; the per-call image-descriptor table.
#pragma once

#include "head.cuh"

namespace {

constexpr int TILE_M = 128;                // pixels per MMA tile (one row segment)
constexpr int ROW_PX = TILE_M + 2;         // staged pixels per input row (halo of 1 each side)
constexpr int RU = 8;                      // output rows per work unit
constexpr int TMEM_COLS = 512;
constexpr int HT_X = 32, HT_Y = 8;         // head tile: one warp per tile row (the bit-packing granule)
constexpr unsigned long long kTimeoutNs = 2000000000ull;   // 2 s per wait

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// As mbar_try_wait, but a thread whose phase is not complete is suspended (for
// up to suspend_ns) until it completes, instead of returning at once: a waiting
// warp then takes no issue slots from the warps it shares a sub-partition with.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity, uint32_t suspend_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(suspend_ns)
        : "memory");
    return ok != 0;
}
constexpr uint32_t kSuspendNs = 1000;      // per suspended try: the abort flag and the deadline are checked in between

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait.  Returns false on timeout (which it records) or when another
// role has already aborted (unless ignore_abort).  Inlined: a call in an MMA
// issue loop (even one not taken) forces register traffic that starves the
// tensor pipe between rows.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err, bool ignore_abort = false)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_sleep(bar, parity, kSuspendNs)) return true;
        if ((it & 3u) == 0) {
            if (!ignore_abort && *abort_flag) return false;
            const uint64_t el = globaltimer_ns() - t0;
            if (el > kTimeoutNs || it > (1u << 28)) {
                *abort_flag = 1;
                atomicExch(err, (int)HT_ERR_TIMEOUT);
                if (atomicCAS(err + 1, 0, 1) == 0) {        // first expiry: where, and after how long
                    err[2] = (int)bar;
                    err[3] = (int)((blockDim.x << 16) | (threadIdx.x >> 5));
                    err[4] = (int)blockIdx.x;
                    err[5] = (int)it;
                    *reinterpret_cast<unsigned long long *>(err + 6) = el;
                }
                return false;
            }
        }
    }
}

// Non-blocking test of a phase (never suspends the thread).
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the MMA-issuing warp: polls without suspending, so the warp
// resumes issuing as soon as the phase completes; the same expiry record as mbar_wait.
__device__ __forceinline__ bool mbar_wait_poll(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err)
{
    if (mbar_test_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_test_wait(bar, parity)) return true;
        if ((it & 63u) == 0) {
            if (*abort_flag) return false;
            const uint64_t el = globaltimer_ns() - t0;
            if (el > kTimeoutNs || it > (1u << 30)) {
                *abort_flag = 1;
                atomicExch(err, (int)HT_ERR_TIMEOUT);
                if (atomicCAS(err + 1, 0, 1) == 0) {
                    err[2] = (int)bar;
                    err[3] = (int)((blockDim.x << 16) | (threadIdx.x >> 5));
                    err[4] = (int)blockIdx.x;
                    err[5] = (int)it;
                    *reinterpret_cast<unsigned long long *>(err + 6) = el;
                }
                return false;
            }
        }
    }
}

// mbar_wait_poll by every lane of a warp, with a warp-uniform result.
__device__ __forceinline__ bool mbar_wait_poll_warp(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err)
{
    return __all_sync(0xffffffffu, mbar_wait_poll(bar, parity, abort_flag, err));
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: canonical K-major layout without swizzle.
// start >> 4 in [0,14), LBO >> 4 in [16,30), SBO >> 4 in [32,46), version 1 at
// bit 46, base offset 0, swizzle 0.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor: D = F32 (bit 4), A/B format at bits 7/10 (kind::f16:
// F16 = 0, BF16 = 1; kind::f8f6f4: E4M3 = 0), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.  AB is the A/B format code (A and B always share it).
template <uint32_t AB>
__host__ __device__ constexpr uint32_t idesc_m128_ab(uint32_t n)
{
    return (1u << 4) | (AB << 7) | (AB << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}
template <bool FP8>
__host__ __device__ constexpr uint32_t idesc_m128(uint32_t n)
{
    return idesc_m128_ab<FP8 ? 0u : 1u>(n);
}

// Warp-wide issuing: the whole warp runs the MMA schedule, so its state (slot, row,
// descriptors) is warp-uniform, and the one lane chosen by elect_one() issues each MMA
// and commit under a predicate, with no divergent branch around them.  Every MMA here
// accumulates (D += A B; the enable-input-d operand is the constant 1): accumulators
// are zeroed by the epilogue after it drains them, never by the MMA.  A commit arrives
// on the barrier once every MMA issued so far by this thread has completed.
__device__ __forceinline__ uint32_t elect_one()
{
    uint32_t e;
    asm volatile("{\n\t.reg .pred p;\n\telect.sync _|p, 0xffffffff;\n\tselp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(e));
    return e;
}
template <bool FP8>
__device__ __forceinline__ void mma_ss_el(uint32_t el, uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc)
{
    if constexpr (FP8) {
        asm volatile(
            "{\n\t.reg .pred e;\n\tsetp.ne.b32 e, %4, 0;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, 1;\n\t}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(el)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred e;\n\tsetp.ne.b32 e, %4, 0;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n\t}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(el)
            : "memory");
    }
}
__device__ __forceinline__ void mma_commit_el(uint32_t el, uint32_t bar)
{
    asm volatile("{\n\t.reg .pred e;\n\tsetp.ne.b32 e, %1, 0;\n\t"
                 "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}\n" ::"r"(bar),
                 "r"(el)
                 : "memory");
}

// ---------------------------------------------------------------------------
// CTA pairs (cluster of 2, tcgen05 cta_group::2).  Both CTAs allocate and free
// TMEM together (one warp in each); only the pair's first CTA issues MMAs,
// whose M = 256 rows are the two CTAs' 128-row A tiles and whose B operand is
// split by N: the first CTA holds rows [0, N/2), the second [N/2, N), at the
// same shared-memory offset.  Each CTA's TMEM receives its own 128 rows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
// Arrive on a barrier of another CTA of the cluster.  Default semantics
// (release at CTA scope): the data the arrival publishes is either this CTA's
// shared memory filled by the async proxy (bulk copies, observed complete on
// this CTA's own barrier first) or TMEM reads already waited for, so no
// cluster-scope fence is needed; a cluster-scope release here costs a full
// memory barrier per arrival.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr, uint32_t v)
{
    asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}
// Bounded wait on a barrier that the peer CTA may arrive on (default acquire
// semantics, as for mbar_wait).  On expiry it records the timeout like mbar_wait
// and also raises the peer's abort flag (peer_abort: shared::cluster address,
// 0 = none).
__device__ __forceinline__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, volatile int *abort_flag, uint32_t peer_abort, int *err,
                             bool ignore_abort = false)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_sleep(bar, parity, kSuspendNs)) return true;
        if ((it & 3u) == 0) {
            if (!ignore_abort && *abort_flag) return false;
            const uint64_t el = globaltimer_ns() - t0;
            if (el > kTimeoutNs || it > (1u << 28)) {
                *abort_flag = 1;
                if (peer_abort) st_cluster_u32(peer_abort, 1u);
                atomicExch(err, (int)HT_ERR_TIMEOUT);
                if (atomicCAS(err + 1, 0, 1) == 0) {
                    err[2] = (int)bar;
                    err[3] = (int)((blockDim.x << 16) | (threadIdx.x >> 5));
                    err[4] = (int)blockIdx.x;
                    err[5] = (int)it;
                    *reinterpret_cast<unsigned long long *>(err + 6) = el;
                }
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tmem_alloc_pair(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
template <bool FP8>
__host__ __device__ constexpr uint32_t idesc_m256(uint32_t n)
{
    return (1u << 4) | ((FP8 ? 0u : 1u) << 7) | ((FP8 ? 0u : 1u) << 10) | ((n >> 3) << 17) | ((256u >> 4) << 24);
}
// CTA-pair forms (cta_group::2, issued by the pair's first CTA): M = 256, A rows from
// both CTAs, the commit arriving on the barrier at this shared offset in both CTAs.
template <bool FP8>
__device__ __forceinline__ void mma_ss_pair_el(uint32_t el, uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc)
{
    if constexpr (FP8) {
        asm volatile(
            "{\n\t.reg .pred e;\n\tsetp.ne.b32 e, %4, 0;\n\t"
            "@e tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, 1;\n\t}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(el)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred e;\n\tsetp.ne.b32 e, %4, 0;\n\t"
            "@e tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, 1;\n\t}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(el)
            : "memory");
    }
}
__device__ __forceinline__ void mma_commit_pair_el(uint32_t el, uint32_t bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\tsetp.ne.b32 e, %2, 0;\n\t"
        "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n\t}\n" ::"r"(bar),
        "h"((uint16_t)3), "r"(el)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_zero16(uint32_t taddr)
{
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d)
{
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return (lo & 0xFFFFu) | (hi << 16);
}
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float f16_round(float v) { return __half2float(__float2half_rn(v)); }
__device__ __forceinline__ uint32_t pack_f16x2(float a, float b)
{
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}
// rounding of a stored activation: bf16, or IEEE binary16 in the FP16 form
template <bool F16>
__device__ __forceinline__ float act_round(float v)
{
    if constexpr (F16) return f16_round(v);
    else return bf16_round(v);
}
// v = a + b + c exactly for a float32 v: a = bf16(v) holds its top 8 significant bits,
// v - a (exact in float32) has at most 16 significant bits, b = bf16(v - a) the next 8,
// and the remainder v - a - b has at most 8, so c = bf16(v - a - b) is exact.
__device__ __forceinline__ void split3_bf16(float v, float &a, float &b, float &c)
{
    a = bf16_round(v);
    const float r = v - a;
    b = bf16_round(r);
    c = bf16_round(r - b);
}

// Stores CO channel values of one pixel into the chunk-planar layout.
// out_fp8: e4m3(bf16(v) * inv_scale) (16 channels per chunk), else bf16 (8 per chunk).
template <int CO = 64>
__device__ __forceinline__ void store_pixel(const float *v, void *out, int out_fp8, float inv_scale, int H, int W,
                                            int y, int x)
{
    if (out_fp8) {
        uint8_t *o = (uint8_t *)out;
#pragma unroll
        for (int c = 0; c < CO / 16; ++c) {
            uint4 q;
            q.x = pack_e4m3x4(bf16_round(v[16 * c + 0]) * inv_scale, bf16_round(v[16 * c + 1]) * inv_scale,
                              bf16_round(v[16 * c + 2]) * inv_scale, bf16_round(v[16 * c + 3]) * inv_scale);
            q.y = pack_e4m3x4(bf16_round(v[16 * c + 4]) * inv_scale, bf16_round(v[16 * c + 5]) * inv_scale,
                              bf16_round(v[16 * c + 6]) * inv_scale, bf16_round(v[16 * c + 7]) * inv_scale);
            q.z = pack_e4m3x4(bf16_round(v[16 * c + 8]) * inv_scale, bf16_round(v[16 * c + 9]) * inv_scale,
                              bf16_round(v[16 * c + 10]) * inv_scale, bf16_round(v[16 * c + 11]) * inv_scale);
            q.w = pack_e4m3x4(bf16_round(v[16 * c + 12]) * inv_scale, bf16_round(v[16 * c + 13]) * inv_scale,
                              bf16_round(v[16 * c + 14]) * inv_scale, bf16_round(v[16 * c + 15]) * inv_scale);
            *reinterpret_cast<uint4 *>(o + (((size_t)c * H + y) * W + x) * 16) = q;
        }
    } else {
        uint8_t *o = (uint8_t *)out;
#pragma unroll
        for (int c = 0; c < CO / 8; ++c) {
            uint4 q;
            q.x = pack_bf16x2(v[8 * c + 0], v[8 * c + 1]);
            q.y = pack_bf16x2(v[8 * c + 2], v[8 * c + 3]);
            q.z = pack_bf16x2(v[8 * c + 4], v[8 * c + 5]);
            q.w = pack_bf16x2(v[8 * c + 6], v[8 * c + 7]);
            *reinterpret_cast<uint4 *>(o + (((size_t)c * H + y) * W + x) * 16) = q;
        }
    }
}

// Stores 64 channel values of one pixel as IEEE binary16 (8 per chunk).
__device__ __forceinline__ void store_pixel_f16(const float *v, void *out, int H, int W, int y, int x)
{
    uint8_t *o = (uint8_t *)out;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint4 q;
        q.x = pack_f16x2(v[8 * c + 0], v[8 * c + 1]);
        q.y = pack_f16x2(v[8 * c + 2], v[8 * c + 3]);
        q.z = pack_f16x2(v[8 * c + 4], v[8 * c + 5]);
        q.w = pack_f16x2(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4 *>(o + (((size_t)c * H + y) * W + x) * 16) = q;
    }
}

// Epilogue of a bf16-output layer (F16: binary16 output): v * scale + bias (per
// channel), ReLU, rounding, into the chunk-planar layout.  Two channels per
// instruction: a packed FP32 FMA (each lane an ordinary fmaf) and one convert that
// rounds to nearest even and clamps negatives to zero (the same value as rounding
// max(x, 0)).
template <bool F16 = false>
__device__ __forceinline__ void store_pixel_bias_relu_bf16(const float *v, const float *scale, const float *bias,
                                                          void *out, int H, int W, int y, int x)
{
    uint8_t *o = (uint8_t *)out;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint32_t w4[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int n = 8 * c + 2 * h;
            unsigned long long vv, ss, bb, rr;
            asm("mov.b64 %0, {%1, %2};" : "=l"(vv) : "f"(v[n]), "f"(v[n + 1]));
            asm("mov.b64 %0, {%1, %2};" : "=l"(ss) : "f"(scale[n]), "f"(scale[n + 1]));
            asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(bias[n]), "f"(bias[n + 1]));
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rr) : "l"(vv), "l"(ss), "l"(bb));
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(rr));
            if constexpr (F16) asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(w4[h]) : "f"(hi), "f"(lo));
            else asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(w4[h]) : "f"(hi), "f"(lo));
        }
        *reinterpret_cast<uint4 *>(o + (((size_t)c * H + y) * W + x) * 16) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
}

// Epilogue of an e4m3-output layer (FP8 form): v * scale + bias, ReLU, bf16 (the
// activations' storage rounding), times the next layer's inverse input scale (a power
// of two: exact), e4m3 with saturation (round to nearest even), 16 channels per chunk.
// Packed over channel pairs (fma.rn.f32x2, cvt.rn.relu.bf16x2.f32, mul.rn.f32x2,
// cvt.rn.satfinite.e4m3x2.f32): the same values as the per-channel sequence.
__device__ __forceinline__ void store_pixel_bias_relu_e4m3(const float *v, const float *scale, const float *bias,
                                                          float inv_scale, void *out, int H, int W, int y, int x)
{
    uint8_t *o = (uint8_t *)out;
    unsigned long long ii;
    asm("mov.b64 %0, {%1, %1};" : "=l"(ii) : "f"(inv_scale));
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t w4[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint16_t e[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int n = 16 * c + 4 * h + 2 * q;
                unsigned long long vv, ss, bb, rr;
                asm("mov.b64 %0, {%1, %2};" : "=l"(vv) : "f"(v[n]), "f"(v[n + 1]));
                asm("mov.b64 %0, {%1, %2};" : "=l"(ss) : "f"(scale[n]), "f"(scale[n + 1]));
                asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(bias[n]), "f"(bias[n + 1]));
                asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rr) : "l"(vv), "l"(ss), "l"(bb));
                float lo, hi;
                asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(rr));
                uint32_t b2;
                asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(b2) : "f"(hi), "f"(lo));
                asm("mov.b64 %0, {%1, %2};" : "=l"(vv) : "f"(__uint_as_float(b2 << 16)), "f"(__uint_as_float(b2 & 0xFFFF0000u)));
                asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(rr) : "l"(vv), "l"(ii));
                asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(rr));
                asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(e[q]) : "f"(hi), "f"(lo));
            }
            w4[h] = (uint32_t)e[0] | ((uint32_t)e[1] << 16);
        }
        *reinterpret_cast<uint4 *>(o + (((size_t)c * H + y) * W + x) * 16) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
}

// One image of a batched call.  Every kernel of the tensor-core form walks a
// flattened index space (conv units, layer-1 tiles, head tiles) over all images
// of the call and finds its image through the *_begin prefix sums.
struct ImgDesc {
    const float *contone;
    uint8_t *act[2];          // chunk-planar activation buffers (input / output by in_buf)
    uint32_t *bits;
    float *prob;              // nullable
    uint2 *mask;              // nullable: 64-bit ReLU mask per pixel of the layer's output
                              // (written by a forward layer, applied by a data-gradient layer)
    uint8_t *save;            // nullable: last hidden layer with fused head partials also
                              // stores its activations here (training forward)
    float *part;              // nullable: where the fused head partials go (else act[out])
    int cpitch, H, W, words;
    uint32_t image;           // Philox image index (position in the call)
    int xtiles;               // ceil(W / 128)
    int unit_begin;           // first conv unit (xtiles * ceil(H / RU) units per image)
    int hd_begin;             // first head tile (ceil(W / 32) * ceil(H / 8))
    int pre_begin;            // first layer-1 input group of 4 pixels (ceil(H * W / 4))
    int xtiles2;              // ceil(W / 256): column tiles of a CTA pair
    int unit2_begin;          // first conv unit of the CTA-pair form (xtiles2 * ceil(H / RU) units per image)
    int hq_begin;             // first 128 x 8 tile of k_head_partials (ceil(W / 128) * ceil(H / 8))
};

// largest i with begin(i) <= u (images sorted by their begin offsets)
template <typename F>
__device__ __forceinline__ int find_image(int n, int u, F begin)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin(mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct UnitInfo {
    const ImgDesc *D;
    const uint8_t *in;
    uint8_t *out;
    int H, W, x0, y0, nrows;
};

// Unit u of a call: ru (<= RU) rows x one 128-pixel column tile of one image
// (PAIR: one 256-pixel tile, the two 128-pixel halves of a CTA pair).  order 0
// walks an image's units row band by row band, order 1 column tile by column tile.
template <bool PAIR = false>
__device__ __forceinline__ UnitInfo unit_info(const ImgDesc *imgs, int n_imgs, int in_buf, int u, int ru = RU,
                                              int order = 0)
{
    const int im = find_image(n_imgs, u, [&](int i) { return PAIR ? __ldg(&imgs[i].unit2_begin) : __ldg(&imgs[i].unit_begin); });
    const ImgDesc *D = imgs + im;
    const int lu = u - (PAIR ? __ldg(&D->unit2_begin) : __ldg(&D->unit_begin));
    const int xt = PAIR ? __ldg(&D->xtiles2) : __ldg(&D->xtiles);
    constexpr int TW = PAIR ? 2 * TILE_M : TILE_M;
    UnitInfo ui;
    ui.D = D;
    ui.H = __ldg(&D->H);
    ui.W = __ldg(&D->W);
    if (order == 0) {
        ui.x0 = (lu % xt) * TW;
        ui.y0 = (lu / xt) * ru;
    } else {
        const int nb = (ui.H + ru - 1) / ru;
        ui.x0 = (lu / nb) * TW;
        ui.y0 = (lu % nb) * ru;
    }
    ui.nrows = min(ui.H, ui.y0 + ru) - ui.y0;
    ui.in = (const uint8_t *)D->act[in_buf];
    ui.out = D->act[in_buf ^ 1];
    return ui;
}

// Work-index layout of one image inside a call's table: conv units, head tiles,
// layer-1 input groups (prefix sums over the images in table order).
inline void set_begins(ImgDesc &D, int &units, int &hd, int &pre, int ru = RU, int *units2 = nullptr,
                       int *hq = nullptr)
{
    D.xtiles = (D.W + TILE_M - 1) / TILE_M;
    D.unit_begin = units;
    D.hd_begin = hd;
    D.pre_begin = pre;
    D.xtiles2 = (D.W + 2 * TILE_M - 1) / (2 * TILE_M);
    D.unit2_begin = units2 ? *units2 : 0;
    if (units2) *units2 += D.xtiles2 * ((D.H + ru - 1) / ru);
    D.hq_begin = hq ? *hq : 0;
    if (hq) *hq += D.xtiles * ((D.H + HT_Y - 1) / HT_Y);
    units += D.xtiles * ((D.H + ru - 1) / ru);
    hd += ((D.W + HT_X - 1) / HT_X) * ((D.H + HT_Y - 1) / HT_Y);
    pre += (int)(((size_t)D.H * D.W + 3) / 4);
}

int num_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace
