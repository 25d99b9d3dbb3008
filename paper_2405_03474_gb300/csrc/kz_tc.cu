// Tensor-core kernel product W = (K(X, X) + noise I) V for sm_103a (tcgen05).
//
// The O(n^2) step of Algorithm 1 (Section 2, complexity paragraph) evaluated
// matrix-free: each CTA owns 128 rows i and sweeps all points j in tiles of 64.
//   * 8 "eval" warps compute k(x_i, x_j) on the CUDA cores (fp32 differences,
//     MUFU rsqrt/ex2), round to fp16 (or bf16), optionally split hi/lo, and
//     store the 128 x 64 tile into shared memory in the canonical no-swizzle
//     K-major UMMA layout;
//   * 1 producer warp streams point tiles X_j and the pre-converted operand
//     image of V_j into shared memory with cp.async.bulk (mbarrier tx counts);
//   * 1 MMA warp issues tcgen05.mma (M=128, N=c, K=16) accumulating D = K V in
//     tensor memory (fp32), and releases each stage with tcgen05.commit;
//   * at the end the eval warps read D with tcgen05.ld, undo the column
//     scaling, add noise * V and store W.
// Every mbarrier wait is bounded (clock64 budget); on timeout the CTA records
// an error word, drains what it issued (again bounded), frees TMEM and exits.
//
// Precisions: LD_F16_TC (K, V in fp16), LD_BF16_TC (bf16), LD_F16X3_TC
// (K = Kh + Kl, V = Vh + Vl in fp16; D += Kh Vh + Kh Vl + Kl Vh).  V columns are
// scaled by powers of two so |V| <= 1 before rounding; K is computed with unit
// variance and the variance is applied in the epilogue.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace ld {

namespace {

constexpr int TM = 128;        // rows per CTA (MMA M)
constexpr int TJ = 64;         // j per tile (4 MMA K-steps of 16)
constexpr int NEVAL = 8;       // eval warps
constexpr int NTHREADS = (NEVAL + 2) * 32;
constexpr int A_BYTES = TM * TJ * 2;  // one 128 x 64 half tile
constexpr int MAX_N = 256;
constexpr int KCH = 8;          // j-tiles accumulated in TMEM before a drain
constexpr int DRAIN_MAX_N = 128;
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
// Bounded wait; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > WAIT_BUDGET) return false;
    }
    return true;
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
__host__ __device__ constexpr uint32_t make_idesc(int M, int N, uint32_t ab) {
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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

// unit-variance kernel value from squared scaled distance
template <int KIND>
__device__ __forceinline__ float kval_fast(float u2) {
    if (KIND == LD_RBF) return exp2f(-1.4426950408889634f * u2);
    float uu = fmaxf(u2, 1e-30f);
    float u = uu * rsqrtf(uu);
    float e = exp2f(-1.4426950408889634f * u);
    return fmaf(fmaf(u, 1.0f / 3.0f, 1.0f), u, 1.0f) * e;
}

struct TcParams {
    const float *Xp;        // padded points, ntiles*64 x d
    const uint8_t *img;     // operand image: per tile, nprod x (N x 64) halves
    const float *V;         // original V (n x c, row-major)
    const float *colinv;    // 1 / column scale (N)
    float *W;
    int64_t n;
    int d, c, c0, N, ncols_tmem;
    int ntiles;             // ceil(n / 64)
    float variance, noise;
    int *err;
};

// Dynamic shared memory layout (per stage s): A hi/lo | B hi/lo | X tile
struct Layout {
    int stages, nprod_a, nprod_b, a_bytes, b_bytes, x_bytes, stage_bytes, total;
};

__host__ __device__ inline Layout make_layout(int N, int d, int nprod, int stages) {
    Layout L;
    L.stages = stages;
    L.nprod_a = nprod == 3 ? 2 : 1;
    L.nprod_b = nprod == 3 ? 2 : 1;
    L.a_bytes = L.nprod_a * A_BYTES;
    L.b_bytes = L.nprod_b * N * TJ * 2;
    L.x_bytes = ((TJ * d * 4 + 127) / 128) * 128;
    L.stage_bytes = ((L.a_bytes + L.b_bytes + L.x_bytes + 1023) / 1024) * 1024;
    L.total = 1024 + stages * L.stage_bytes + 1024;  // barriers + alignment slack
    if (nprod == 3 && N <= DRAIN_MAX_N) L.total += TM * (N + 1) * 4;  // drained partial sums
    return L;
}

template <int KIND, int DC, int NPROD, bool BF16, bool DRAIN>
__global__ void __launch_bounds__(NTHREADS, 1) kz_tc_kernel(TcParams p, Layout L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);          // [stages] loads landed
    uint64_t *afull = full + 8;                                   // [stages] A tile written
    uint64_t *empty = afull + 8;                                  // [stages] MMA done with stage
    uint64_t *done = empty + 8;                                   // final accumulate done
    uint64_t *cfull = done + 1;                                   // [2] chunk accumulated in TMEM buffer
    uint64_t *cempty = cfull + 2;                                 // [2] TMEM buffer drained
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(cempty + 2);
    int *s_err = reinterpret_cast<int *>(tmem_slot + 1);
    uint8_t *stage0 = smem + 1024;
    // fp32 partial sums drained from TMEM (DRAIN only): 128 rows x (N + 1)
    float *sacc = reinterpret_cast<float *>(stage0 + (size_t)L.stages * L.stage_bytes);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int dd = DC > 0 ? DC : p.d;
    const int64_t row0 = (int64_t)blockIdx.x * TM;
    const int S = L.stages;
    const int T = p.ntiles;
    const int ldacc = p.N + 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&afull[s], NEVAL * 32);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        mbar_init(&cfull[0], 1);
        mbar_init(&cfull[1], 1);
        mbar_init(&cempty[0], NEVAL * 32);
        mbar_init(&cempty[1], NEVAL * 32);
        *s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (DRAIN)
        for (int e = threadIdx.x; e < TM * ldacc; e += NTHREADS) sacc[e] = 0.f;
    if (warp == NEVAL) {  // MMA warp owns TMEM
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(p.ncols_tmem)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == NEVAL + 1) {
        // ---------------- producer: X tile and operand image of V per j-tile
        if (lane == 0) {
            const uint32_t xb = (uint32_t)(TJ * dd * 4);
            const uint32_t bb = (uint32_t)L.b_bytes;
            int t = 0;
            for (; t < T; ++t) {
                const int s = t % S;
                if (t >= S && !mbar_wait(&empty[s], ((t / S) - 1) & 1)) {
                    atomicOr(s_err, ERR_TIMEOUT);
                    break;
                }
                uint8_t *st = stage0 + (size_t)s * L.stage_bytes;
                mbar_expect_tx(&full[s], xb + bb);
                bulk_g2s(st + L.a_bytes + L.b_bytes, p.Xp + (size_t)t * TJ * dd, xb, &full[s]);
                bulk_g2s(st + L.a_bytes, p.img + (size_t)t * bb, bb, &full[s]);
            }
            // drain: every issued copy must land before the CTA may exit
            for (int u = std::max(0, t - S); u < t; ++u) {
                if (!mbar_wait(&full[u % S], (u / S) & 1)) atomicOr(s_err, ERR_TIMEOUT);
            }
        }
    } else if (warp == NEVAL) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = make_idesc(TM, p.N, BF16 ? 1u : 0u);
            const uint32_t lbo = 128, sbo = 1024;
            const uint32_t bhalf = (uint32_t)(p.N * TJ * 2);
            bool ok = true;
            int t = 0;
            for (; t < T && ok; ++t) {
                const int s = t % S;
                const int k = t / KCH;
                const bool first = DRAIN ? (t % KCH == 0) : (t == 0);
                const uint32_t dt = tmem + (DRAIN ? (uint32_t)((k & 1) * p.N) : 0u);
                if (DRAIN && first && k >= 2 && !mbar_wait(&cempty[k & 1], ((k - 2) >> 1) & 1)) {
                    ok = false;
                    break;
                }
                if (!mbar_wait(&afull[s], (t / S) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(stage0 + (size_t)s * L.stage_bytes);
                const uint32_t b0 = a0 + (uint32_t)L.a_bytes;
#pragma unroll
                for (int ks = 0; ks < TJ / 16; ++ks) {
                    const uint32_t koff = (uint32_t)ks * 256u;
                    const uint64_t ah = make_desc(a0 + koff, lbo, sbo);
                    const uint64_t bh = make_desc(b0 + koff, lbo, sbo);
                    mma_f16(dt, ah, bh, idesc, (first && ks == 0) ? 0u : 1u);
                    if (NPROD == 3) {
                        const uint64_t al = make_desc(a0 + (uint32_t)A_BYTES + koff, lbo, sbo);
                        const uint64_t bl = make_desc(b0 + bhalf + koff, lbo, sbo);
                        mma_f16(dt, ah, bl, idesc, 1u);
                        mma_f16(dt, al, bh, idesc, 1u);
                    }
                }
                mma_commit(&empty[s]);
                if (DRAIN && (t % KCH == KCH - 1 || t == T - 1)) mma_commit(&cfull[k & 1]);
            }
            if (!ok) atomicOr(s_err, ERR_TIMEOUT);
            mma_commit(done);  // arrives once all issued MMAs completed
        }
    } else {
        // ---------------- eval warps: K tile into shared memory
        const int e = threadIdx.x;          // 0 .. 255
        const int rp = e & 63;              // rows rp and rp + 64
        const int jq = e >> 6;              // j range [16 jq, 16 jq + 16)
        const int quad = warp & 3;          // TMEM lane quadrant of this warp
        const int halfc = warp >> 2;        // column half handled in drains/epilogue
        const int ncol_half = p.N / 2;
        float xi0[8], xi1[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            xi0[q] = q < dd ? p.Xp[(row0 + rp) * dd + q] : 0.f;
            xi1[q] = q < dd ? p.Xp[(row0 + rp + 64) * dd + q] : 0.f;
        }
        // move chunk k's TMEM buffer into the fp32 partial sums (round to nearest)
        auto drain = [&](int k) -> bool {
            if (!mbar_wait(&cfull[k & 1], (k >> 1) & 1)) return false;
            tc_fence_after();
            const int row = quad * 32 + lane;
            for (int c8 = halfc * ncol_half; c8 < (halfc + 1) * ncol_half; c8 += 8) {
                float v[8];
                tmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)((k & 1) * p.N + c8), v);
#pragma unroll
                for (int q = 0; q < 8; ++q) sacc[row * ldacc + c8 + q] += v[q];
            }
            tc_fence_before();
            mbar_arrive(&cempty[k & 1]);
            return true;
        };
        const int C = (T + KCH - 1) / KCH;  // chunks
        int drained = 0;                     // chunks already drained
        bool ok = true;
        for (int t = 0; t < T; ++t) {
            const int s = t % S;
            if (DRAIN && t % KCH == KCH / 2 && t >= KCH + KCH / 2) {
                // chunk t / KCH - 1 finished half a chunk ago
                if (!drain(drained)) {
                    ok = false;
                    break;
                }
                ++drained;
            }
            if (!mbar_wait(&full[s], (t / S) & 1)) {
                ok = false;
                break;
            }
            uint8_t *st = stage0 + (size_t)s * L.stage_bytes;
            const float *xs = reinterpret_cast<const float *>(st + L.a_bytes + L.b_bytes);
            const int64_t jbase = (int64_t)t * TJ;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kq = jq * 2 + h;  // core-matrix column (8 j values)
                float k0[8], k1[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int jj = kq * 8 + q;
                    float u0 = 0.f, u1 = 0.f;
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        if (a < dd) {
                            const float xj = xs[jj * dd + a];
                            const float d0 = xi0[a] - xj, d1 = xi1[a] - xj;
                            u0 = fmaf(d0, d0, u0);
                            u1 = fmaf(d1, d1, u1);
                        }
                    }
                    const bool valid = jbase + jj < p.n;
                    k0[q] = valid ? kval_fast<KIND>(u0) : 0.f;
                    k1[q] = valid ? kval_fast<KIND>(u1) : 0.f;
                }
                uint4 h0, h1;
                h0.x = pack2<BF16>(k0[0], k0[1]); h0.y = pack2<BF16>(k0[2], k0[3]);
                h0.z = pack2<BF16>(k0[4], k0[5]); h0.w = pack2<BF16>(k0[6], k0[7]);
                h1.x = pack2<BF16>(k1[0], k1[1]); h1.y = pack2<BF16>(k1[2], k1[3]);
                h1.z = pack2<BF16>(k1[4], k1[5]); h1.w = pack2<BF16>(k1[6], k1[7]);
                const int r0i = rp, r1i = rp + 64;
                const size_t off0 = (size_t)(r0i >> 3) * 1024 + (size_t)kq * 128 + (size_t)(r0i & 7) * 16;
                const size_t off1 = (size_t)(r1i >> 3) * 1024 + (size_t)kq * 128 + (size_t)(r1i & 7) * 16;
                *reinterpret_cast<uint4 *>(st + off0) = h0;
                *reinterpret_cast<uint4 *>(st + off1) = h1;
                if (NPROD == 3) {
                    uint4 l0, l1;
                    uint32_t *hp0 = &h0.x, *hp1 = &h1.x, *lp0 = &l0.x, *lp1 = &l1.x;
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        float2 f0 = unpack2<BF16>(hp0[w]);
                        float2 f1 = unpack2<BF16>(hp1[w]);
                        lp0[w] = pack2<BF16>(k0[2 * w] - f0.x, k0[2 * w + 1] - f0.y);
                        lp1[w] = pack2<BF16>(k1[2 * w] - f1.x, k1[2 * w + 1] - f1.y);
                    }
                    *reinterpret_cast<uint4 *>(st + A_BYTES + off0) = l0;
                    *reinterpret_cast<uint4 *>(st + A_BYTES + off1) = l1;
                }
            }
            fence_async_smem();
            mbar_arrive(&afull[s]);
        }
        // ---------------- epilogue
        const bool got = ok && mbar_wait(done, 0);
        tc_fence_after();
        if (got && DRAIN) {
            for (; drained < C; ++drained)
                if (!drain(drained)) {
                    ok = false;
                    break;
                }
        }
        if (!got || !ok) {
            atomicOr(s_err, ERR_TIMEOUT);
        } else {
            const int64_t i = row0 + quad * 32 + lane;
            for (int c8 = halfc * ncol_half; c8 < (halfc + 1) * ncol_half; c8 += 8) {
                float v[8];
                if (DRAIN) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = sacc[(quad * 32 + lane) * ldacc + c8 + q];
                } else {
                    tmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c8, v);
                }
                if (i < p.n) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int col = p.c0 + c8 + q;
                        if (c8 + q < p.N && col < p.c) {
                            const float vin = p.V[i * p.c + col];
                            p.W[i * p.c + col] = v[q] * p.variance * p.colinv[c8 + q] + p.noise * vin;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == NEVAL) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.ncols_tmem)
                     : "memory");
    }
    if (threadIdx.x == 0 && *s_err) atomicOr(p.err, *s_err);
}

// ------------------------------------------------------------ prep kernels
// per-column max |V| over rows, partials per block
__global__ void colmax_kernel(const float *V, int64_t n, int c, int c0, int N, float *part) {
    // block handles a row range; thread t handles column t (t < N)
    const int col = threadIdx.x;
    const int nb = gridDim.x;
    const int64_t per = (n + nb - 1) / nb;
    const int64_t r0 = blockIdx.x * per, r1 = min(n, r0 + per);
    float m = 0.f;
    if (col < N && c0 + col < c)
        for (int64_t i = r0; i < r1; ++i) m = fmaxf(m, fabsf(V[i * c + c0 + col]));
    if (col < N) part[(size_t)blockIdx.x * N + col] = m;
}

__global__ void colscale_kernel(const float *part, int nb, int N, float *scale, float *colinv) {
    const int col = threadIdx.x;
    if (col >= N) return;
    float m = 0.f;
    for (int b = 0; b < nb; ++b) m = fmaxf(m, part[(size_t)b * N + col]);
    // power of two with m * s <= 1 (exact rescaling)
    int e = 0;
    if (m > 0.f) {
        frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
    }
    const float s = ldexpf(1.0f, -e);
    scale[col] = s;
    colinv[col] = 1.0f / s;
}

// Operand image of V: per j-tile t, per product half (hi, lo), N rows (columns of V)
// x 64 K values in the canonical K-major no-swizzle layout:
// byte offset (col/8)*1024 + (jj/8)*128 + (col%8)*16 + (jj%8)*2.
template <bool BF16, int NPROD>
__global__ void image_kernel(const float *V, int64_t n, int c, int c0, int N, int ntiles,
                             const float *scale, uint8_t *img) {
    // one thread per (t, col, jj-chunk of 8)
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per_tile = (int64_t)N * 8;
    if (idx >= per_tile * ntiles) return;
    const int64_t t = idx / per_tile;
    const int rem = (int)(idx % per_tile);
    const int cr = rem & 7;              // col % 8
    const int kq = (rem >> 3) & 7;       // jj / 8
    const int g = rem >> 6;              // col / 8
    const int col = g * 8 + cr;
    const float s = scale[col];
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t j = t * TJ + kq * 8 + q;
        v[q] = (j < n && col < N && c0 + col < c) ? V[j * c + c0 + col] * s : 0.f;
    }
    uint4 hi;
    hi.x = pack2<BF16>(v[0], v[1]); hi.y = pack2<BF16>(v[2], v[3]);
    hi.z = pack2<BF16>(v[4], v[5]); hi.w = pack2<BF16>(v[6], v[7]);
    const size_t tile_bytes = (size_t)(NPROD == 3 ? 2 : 1) * N * TJ * 2;
    uint8_t *base = img + (size_t)t * tile_bytes;
    const size_t off = (size_t)g * 1024 + (size_t)kq * 128 + (size_t)cr * 16;
    *reinterpret_cast<uint4 *>(base + off) = hi;
    if (NPROD == 3) {
        uint4 lo;
        uint32_t *hp = &hi.x, *lp = &lo.x;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            float2 f = unpack2<BF16>(hp[w]);
            lp[w] = pack2<BF16>(v[2 * w] - f.x, v[2 * w + 1] - f.y);
        }
        *reinterpret_cast<uint4 *>(base + (size_t)N * TJ * 2 + off) = lo;
    }
}

int nprod_of(int precision) { return precision == LD_F16X3_TC ? 3 : 1; }

int chunk_N(int c) {
    int N = std::min(c, MAX_N);
    return ((N + 15) / 16) * 16;
}

int stages_for(int N, int d, int nprod) {
    for (int s = 4; s >= 2; --s)
        if (make_layout(N, d, nprod, s).total <= 200 * 1024) return s;
    return 2;
}

template <int KIND, int DC, int NPROD, bool BF16, bool DRAIN>
int launch_main(const TcParams &p, const Layout &L, int nblocks, cudaStream_t st) {
    auto fn = kz_tc_kernel<KIND, DC, NPROD, BF16, DRAIN>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) {
        set_error("kz_tc: cannot reserve %d bytes of shared memory: %s", L.total, cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    const double nn = (double)p.n * (double)p.n;
    const int slot = prof_begin_launch(st, nn, 2.0 * nn * p.N * NPROD);
    fn<<<nblocks, NTHREADS, L.total, st>>>(p, L);
    prof_end_launch(st, slot);
    return check_launch("kz_tc_kernel");
}

template <int KIND, int NPROD, bool BF16>
int launch_d(const TcParams &p, const Layout &L, int nblocks, cudaStream_t st) {
    const bool drain = NPROD == 3 && p.N <= DRAIN_MAX_N;
    if (drain) {
        switch (p.d) {
            case 1: return launch_main<KIND, 1, NPROD, BF16, NPROD == 3>(p, L, nblocks, st);
            case 2: return launch_main<KIND, 2, NPROD, BF16, NPROD == 3>(p, L, nblocks, st);
            case 3: return launch_main<KIND, 3, NPROD, BF16, NPROD == 3>(p, L, nblocks, st);
            case 4: return launch_main<KIND, 4, NPROD, BF16, NPROD == 3>(p, L, nblocks, st);
            default: return launch_main<KIND, 0, NPROD, BF16, NPROD == 3>(p, L, nblocks, st);
        }
    }
    switch (p.d) {
        case 1: return launch_main<KIND, 1, NPROD, BF16, false>(p, L, nblocks, st);
        case 2: return launch_main<KIND, 2, NPROD, BF16, false>(p, L, nblocks, st);
        case 3: return launch_main<KIND, 3, NPROD, BF16, false>(p, L, nblocks, st);
        case 4: return launch_main<KIND, 4, NPROD, BF16, false>(p, L, nblocks, st);
        default: return launch_main<KIND, 0, NPROD, BF16, false>(p, L, nblocks, st);
    }
}

}  // namespace

size_t kz_tc_workspace(int64_t n, int d, int c, int precision) {
    const int64_t ntiles = (n + TJ - 1) / TJ;
    const int N = chunk_N(c);
    const int nprod = nprod_of(precision);
    Arena a;
    a.measuring = true;
    a.take<float>((size_t)(ntiles * TJ + TM) * d);                  // padded points
    a.take<uint8_t>((size_t)ntiles * (nprod == 3 ? 2 : 1) * N * TJ * 2);  // operand image
    a.take<float>(MAX_N);                                            // scale
    a.take<float>(MAX_N);                                            // 1/scale
    a.take<float>((size_t)256 * MAX_N);                              // colmax partials
    a.take<int>(4);                                                  // error word
    return a.off;
}

int kz_tc(const float *Xs, int64_t n, int d, int kind, double variance, double noise, const float *V,
          float *W, int c, int precision, Arena &ws, cudaStream_t st) {
    if (n == 0 || c == 0) return LD_OK;
    if (d > 8) {
        set_error("kz_tc: d must be <= 8");
        return LD_ERR_INVALID;
    }
    const int64_t ntiles = (n + TJ - 1) / TJ;
    const int nprod = nprod_of(precision);
    const bool bf16 = precision == LD_BF16_TC;
    const int Nmax = chunk_N(c);
    // carve from the caller's arena (already sized by kz_any_workspace)
    const size_t mark = ws.off;
    float *Xp = ws.take<float>((size_t)(ntiles * TJ + TM) * d);
    uint8_t *img = ws.take<uint8_t>((size_t)ntiles * (nprod == 3 ? 2 : 1) * Nmax * TJ * 2);
    float *scale = ws.take<float>(MAX_N);
    float *colinv = ws.take<float>(MAX_N);
    float *part = ws.take<float>((size_t)256 * MAX_N);
    int *err = ws.take<int>(4);
    if (ws.overflow || !Xp) {
        set_error("kz_tc: workspace too small");
        ws.off = mark;
        return LD_ERR_WORKSPACE;
    }
    int code = [&]() -> int {
        LD_CHECK_CUDA(cudaMemsetAsync(Xp, 0, sizeof(float) * (size_t)(ntiles * TJ + TM) * d, st));
        LD_CHECK_CUDA(cudaMemcpyAsync(Xp, Xs, sizeof(float) * (size_t)n * d, cudaMemcpyDeviceToDevice, st));
        LD_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        for (int c0 = 0; c0 < c; c0 += MAX_N) {
            const int N = chunk_N(std::min(MAX_N, c - c0));
            const int nb = 256;
            colmax_kernel<<<nb, MAX_N, 0, st>>>(V, n, c, c0, N, part);
            colscale_kernel<<<1, MAX_N, 0, st>>>(part, nb, N, scale, colinv);
            const int64_t nthr = (int64_t)ntiles * N * 8;
            const unsigned gb = (unsigned)((nthr + 255) / 256);
            if (bf16) image_kernel<true, 1><<<gb, 256, 0, st>>>(V, n, c, c0, N, (int)ntiles, scale, img);
            else if (nprod == 3) image_kernel<false, 3><<<gb, 256, 0, st>>>(V, n, c, c0, N, (int)ntiles, scale, img);
            else image_kernel<false, 1><<<gb, 256, 0, st>>>(V, n, c, c0, N, (int)ntiles, scale, img);
            LD_TRY(check_launch("kz_tc prep", 3));
            TcParams p;
            p.Xp = Xp;
            p.img = img;
            p.V = V;
            p.colinv = colinv;
            p.W = W;
            p.n = n;
            p.d = d;
            p.c = c;
            p.c0 = c0;
            p.N = N;
            const int tcols = (nprod == 3 && N <= DRAIN_MAX_N) ? 2 * N : N;  // ping-pong buffers
            p.ncols_tmem = tcols <= 32 ? 32 : (tcols <= 64 ? 64 : (tcols <= 128 ? 128 : (tcols <= 256 ? 256 : 512)));
            p.ntiles = (int)ntiles;
            p.variance = (float)variance;
            p.noise = (float)noise;
            p.err = err;
            Layout L = make_layout(N, d, nprod, stages_for(N, d, nprod));
            // keep (CTAs per SM) x (TMEM columns) <= 512: reserve enough shared memory
            const int max_ctas = std::max(1, 512 / p.ncols_tmem);
            const int min_smem = (228 * 1024) / (max_ctas + 1) + 1024;
            if (L.total < min_smem) L.total = min_smem;
            const int nblocks = (int)((n + TM - 1) / TM);
            if (kind == LD_RBF) {
                if (bf16) LD_TRY(launch_d<LD_RBF, 1, true>(p, L, nblocks, st));
                else if (nprod == 3) LD_TRY(launch_d<LD_RBF, 3, false>(p, L, nblocks, st));
                else LD_TRY(launch_d<LD_RBF, 1, false>(p, L, nblocks, st));
            } else {
                if (bf16) LD_TRY(launch_d<LD_MATERN52, 1, true>(p, L, nblocks, st));
                else if (nprod == 3) LD_TRY(launch_d<LD_MATERN52, 3, false>(p, L, nblocks, st));
                else LD_TRY(launch_d<LD_MATERN52, 1, false>(p, L, nblocks, st));
            }
        }
        int herr = 0;
        LD_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        LD_CHECK_CUDA(cudaStreamSynchronize(st));
        if (herr) {
            set_error("kz_tc: a device-side wait timed out (error word %d)", herr);
            return LD_ERR_DEVICE_TIMEOUT;
        }
        return LD_OK;
    }();
    ws.off = mark;
    return code;
}

}  // namespace ld
