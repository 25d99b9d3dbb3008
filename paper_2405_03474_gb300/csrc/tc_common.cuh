// Device helpers shared by the tcgen05 kernel products (kz_tc.cu, kz_sym.cu):
// bounded mbarrier waits, bulk copies, tcgen05 descriptors / MMA / TMEM loads,
// fp16/bf16 packing and the 2^-x kernel values on the MUFU.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "common.cuh"

namespace ld {
namespace tc {

constexpr long long WAIT_BUDGET = 4000000000ll;  // ~2 s at 2 GHz

enum { ERR_TIMEOUT = 1 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait with a suspend-time hint (ns): while the phase is incomplete the thread
// is parked until the phase completes or the hint runs out, instead of spinning
// and taking issue slots from the warps that compute.
constexpr uint32_t SUSPEND_HINT_NS = 1000000;
__device__ __forceinline__ bool mbar_try_wait_parked(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(SUSPEND_HINT_NS)
        : "memory");
    return ok != 0;
}
// Bounded wait (budget in SM cycles); false on timeout.
__device__ __forceinline__ bool mbar_wait_budget(uint64_t *bar, uint32_t parity, long long budget) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait_parked(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    return mbar_wait_budget(bar, parity, WAIT_BUDGET);
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout with
// core matrices of 8 rows x 16 bytes; lbo = byte step between core matrices
// along K, sbo = byte step between 8-row groups.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor, kind::f16: D fp32, A/B fp16 (ab = 0) or bf16 (ab = 1),
// both K-major, shape M x N.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N, uint32_t ab, uint32_t a_mn_major = 0) {
    return (1u << 4) | (ab << 7) | (ab << 10) | (a_mn_major << 15) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}
template <bool BF16>
__device__ __forceinline__ float2 unpack2(uint32_t u) {
    if (BF16) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
        return __bfloat1622float2(h);
    } else {
        __half2 h = *reinterpret_cast<__half2 *>(&u);
        return __half22float2(h);
    }
}

// hi/lo split of two kernel values for the fp16 x3 products: hi = f with its 13 low
// mantissa bits cleared (11 significant bits, exact in fp16 over its normal range),
// lo = f - hi (exact in fp32, |lo| < 2^-10 |f|), both packed to fp16.  Masking takes
// the ALU pipe instead of a round trip fp32 -> fp16 -> fp32 on the FMA pipe.
__device__ __forceinline__ void split_f16(float2 f, uint32_t &hi, uint32_t &lo) {
    const float2 h = make_float2(__uint_as_float(__float_as_uint(f.x) & 0xFFFFE000u),
                                 __uint_as_float(__float_as_uint(f.y) & 0xFFFFE000u));
    const float2 l = __ffma2_rn(h, make_float2(-1.f, -1.f), f);
    hi = pack2<false>(h.x, h.y);
    lo = pack2<false>(l.x, l.y);
}

// ---- raw MUFU ops (one instruction each; packed f32x2 arithmetic uses the
// sm_100 float2 builtins __fadd2_rn / __ffma2_rn / __fmul2_rn)
__device__ __forceinline__ float mufu_ex2_neg(float x) {  // 2^-x
    float r;
    asm("{\n .reg .f32 t;\n neg.f32 t, %1;\n ex2.approx.ftz.f32 %0, t;\n}" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float mufu_sqrt(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Kernel values are produced scaled by KSCALE = 2^15 (the products' epilogues multiply
// by KSCALE_INV with the variance).  Unit-variance values lie in [0, 1]; scaled they
// lie in [0, 2^15], inside fp16's range, and fp16 keeps its full 11 significant bits
// down to k = 2^-14 / 2^15 ~ 1.9e-9 instead of 6.1e-5, so the hi/lo split represents
// k to ~2^-21 relative (and to ~1e-12 absolute below that) rather than losing the lo
// part of every k < 0.06 to fp16 subnormals.  Powers of two: the scaling is exact.
constexpr int KSCALE_LOG2 = 15;
constexpr float KSCALE = 32768.0f;
constexpr float KSCALE_INV = 1.0f / 32768.0f;

// Coordinate of the padding points past n: every kernel value with them is exactly
// 0 (2^-x underflows), and squared distances to them (< 1e26 for the at most 8
// dimensions, coordinates of real points far below 1e12) keep the scaled Matern
// polynomial finite in fp32.
constexpr float PAD_COORD = 1e12f;

// KSCALE times the unit-variance kernel values of two pairs from their squared scaled
// distances.  The coordinates carry an extra log2(e) factor (Matern) or sqrt(log2 e)
// (RBF), so the exponential is a bare 2^-x:
//   Matern: u' = u log2 e,  k = (1 + u' ln2 + u'^2 ln2^2 / 3) 2^-u'
//   RBF:    u2' = u2 log2 e, k = 2^-u2'
constexpr float LN2 = 0.69314718055994531f;
constexpr float LN2SQ_3 = 0.16015100463940035f;  // (ln 2)^2 / 3

template <int KIND>
__device__ __forceinline__ float2 kval2(float2 u2) {
    if (KIND == LD_RBF)
        return __fmul2_rn(make_float2(mufu_ex2_neg(u2.x), mufu_ex2_neg(u2.y)), make_float2(KSCALE, KSCALE));
    const float2 u = make_float2(mufu_sqrt(u2.x), mufu_sqrt(u2.y));
    const float2 e = make_float2(mufu_ex2_neg(u.x), mufu_ex2_neg(u.y));
    // the polynomial's coefficients carry KSCALE
    const float2 poly = __ffma2_rn(__ffma2_rn(u, make_float2(LN2SQ_3 * KSCALE, LN2SQ_3 * KSCALE),
                                              make_float2(LN2 * KSCALE, LN2 * KSCALE)),
                                   u, make_float2(KSCALE, KSCALE));
    return __fmul2_rn(poly, e);
}

}  // namespace tc
}  // namespace ld
