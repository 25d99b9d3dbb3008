// Tensor-core kernel product W = (K(X, X) + noise I) V for sm_103a (tcgen05).
//
// The O(n^2) step of Algorithm 1 (Section 2, complexity paragraph) evaluated
// matrix-free: each CTA owns 128 rows i and sweeps all points j in tiles of 64.
//   * 8 "eval" warps compute k(x_i, x_j) on the CUDA cores with packed f32x2
//     arithmetic on pairs of j (differences, squared distance, polynomial) and
//     one MUFU sqrt + ex2 per pair, round to fp16 (or bf16), optionally split
//     hi/lo, and store the 128 x 64 tile into shared memory in the canonical
//     no-swizzle K-major UMMA layout (two A buffers);
//   * 1 producer warp streams point tiles X_j (transposed, padded with far
//     points whose kernel value is exactly 0) and the pre-converted operand
//     image of V_j into a deeper ring of shared-memory stages with
//     cp.async.bulk (mbarrier tx counts);
//   * 1 MMA warp issues tcgen05.mma (M=128, N=c, K=16) accumulating D = K V in
//     tensor memory (fp32), and releases each stage with tcgen05.commit;
//   * at the end the eval warps read D with tcgen05.ld, undo the column
//     scaling, add noise * V and store W.
// Every mbarrier wait is bounded (clock64 budget); on timeout the CTA records
// an error word, drains what it issued (again bounded), frees TMEM and exits.
//
// Precisions: LD_F16_TC (K, V in fp16), LD_BF16_TC (bf16), LD_F16X3_TC
// (K = Kh + Kl, V = Vh + Vl in fp16; D += Kh Vh + Kh Vl + Kl Vh).  V columns are
// scaled by powers of two so max |V_col| lies in [KSCALE / 2, KSCALE) before
// rounding; K is computed with unit
// variance times KSCALE (tc_common.cuh) and variance / KSCALE is applied in the
// epilogue.
//
// The same pipeline serves a stored dense M = K + noise I (FROMM): the eval warps
// then read 4 x 8 values each of every 128 x 64 tile of M from HBM (streaming
// loads, three tiles in flight per thread, 8 rows x 128 bytes per warp load),
// scale them by a power of two that brings max |M_ii| into [KSCALE / 2, KSCALE)
// and round/split them exactly as computed values; the producer streams only the operand image
// of V.  One pass reads M once, so the product is bound by HBM instead of the
// FP32 pipes of the SIMT GEMM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace ld {

using namespace tc;

namespace {

constexpr int TM = 128;        // rows per CTA (MMA M)
constexpr int TJ = 64;         // j per tile (4 MMA K-steps of 16)
constexpr int NEVAL = 8;       // eval warps
constexpr int NTHREADS = (NEVAL + 2) * 32;
constexpr int A_BYTES = TM * TJ * 2;  // one 128 x 64 half tile
constexpr int MAX_N = 256;
constexpr int KCH = 8;          // j-tiles accumulated in TMEM before a drain
constexpr int DRAIN_MAX_N = 128;

struct TcParams {
    const float *Xp;        // point tiles: per 64-point tile, d x 64 floats (transposed)
    const uint8_t *img;     // operand image: per tile, nprod x (N x 64) halves
    const float *V;         // original V (n x c, row-major)
    const float *colinv;    // 1 / column scale (N)
    float *W;
    int64_t n;
    int d, c, c0, N, ncols_tmem;
    int ntiles;             // ceil(n / 64)
    float variance, noise;
    int *err;
    const float *M;         // stored dense M (FROMM), row-major n x n
    const float *mscale;    // FROMM: [0] power-of-two scale of M, [1] its inverse
    int vec4;               // FROMM: n % 4 == 0 and M 16-byte aligned (float4 loads)
};

// Dynamic shared memory (from a 1024-aligned base):
//   [0, 1024)            mbarriers, TMEM address, error word
//   sa A stages          128 x 64 halves (hi, and lo for hi/lo mode)
//   sl load stages       V operand image tile + transposed point tile
//   drained sums         128 x (N + 1) floats (hi/lo mode with N <= 128)
struct Layout {
    int sa, sl, a_bytes, b_bytes, x_bytes, l_bytes, a_off, l_off, acc_off, total;
};

__host__ __device__ inline Layout make_layout(int N, int d, int nprod, int sl) {
    Layout L;
    L.sa = 2;
    L.sl = sl;
    L.a_bytes = (nprod == 3 ? 2 : 1) * A_BYTES;
    L.b_bytes = (nprod == 3 ? 2 : 1) * N * TJ * 2;
    L.x_bytes = TJ * d * 4;
    L.l_bytes = ((L.b_bytes + L.x_bytes + 1023) / 1024) * 1024;
    L.a_off = 1024;
    L.l_off = L.a_off + L.sa * L.a_bytes;
    L.acc_off = L.l_off + L.sl * L.l_bytes;
    const int acc = (nprod == 3 && N <= DRAIN_MAX_N) ? TM * (N + 1) * 4 : 0;
    L.total = L.acc_off + acc + 1024;  // + alignment slack of the dynamic base
    return L;
}

template <int KIND, int DC, int NPROD, bool BF16, bool DRAIN, bool FROMM>
__global__ void __launch_bounds__(NTHREADS, FROMM ? 1 : 2) kz_tc_kernel(TcParams p, Layout L) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned base by pointer arithmetic on the shared array itself, so the
    // compiler keeps shared-window loads and stores (an integer round trip would
    // turn every access into a generic one)
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);  // [sl] loads landed
    uint64_t *empty = full + 8;                           // [sl] MMA done with load stage
    uint64_t *afull = empty + 8;                          // [sa] A tile written
    uint64_t *aempty = afull + 4;                         // [sa] MMA done with A tile
    uint64_t *done = aempty + 4;                          // all MMAs done
    uint64_t *cfull = done + 1;                           // [2] chunk accumulated in TMEM buffer
    uint64_t *cempty = cfull + 2;                         // [2] TMEM buffer drained
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(cempty + 2);
    int *s_err = reinterpret_cast<int *>(tmem_slot + 1);
    uint8_t *abase = smem + L.a_off;
    uint8_t *lbase = smem + L.l_off;
    float *sacc = reinterpret_cast<float *>(smem + L.acc_off);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int dd = DC > 0 ? DC : p.d;
    const int64_t row0 = (int64_t)blockIdx.x * TM;
    const int SA = L.sa, SL = L.sl;
    const int T = p.ntiles;
    const int ldacc = p.N + 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SL; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < SA; ++s) {
            mbar_init(&afull[s], NEVAL * 32);
            mbar_init(&aempty[s], 1);
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
        // ---------------- producer: point tile and operand image of V per j-tile
        if (lane == 0) {
            const uint32_t xb = FROMM ? 0u : (uint32_t)(TJ * dd * 4);
            const uint32_t bb = (uint32_t)L.b_bytes;
            int t = 0;
            for (; t < T; ++t) {
                const int s = t % SL;
                if (t >= SL && !mbar_wait(&empty[s], ((t / SL) - 1) & 1)) {
                    atomicOr(s_err, ERR_TIMEOUT);
                    break;
                }
                uint8_t *st = lbase + (size_t)s * L.l_bytes;
                mbar_expect_tx(&full[s], xb + bb);
                bulk_g2s(st, p.img + (size_t)t * bb, bb, &full[s]);
                if (!FROMM) bulk_g2s(st + L.b_bytes, p.Xp + (size_t)t * TJ * dd, xb, &full[s]);
            }
            // every issued copy must land before the CTA may exit
            for (int u = std::max(0, t - SL); u < t; ++u) {
                if (!mbar_wait(&full[u % SL], (u / SL) & 1)) atomicOr(s_err, ERR_TIMEOUT);
            }
        }
    } else if (warp == NEVAL) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = make_idesc(TM, p.N, BF16 ? 1u : 0u);
            const uint32_t lbo = 128, sbo = 1024;
            const uint32_t bhalf = (uint32_t)(p.N * TJ * 2);
            bool ok = true;
            for (int t = 0; t < T && ok; ++t) {
                const int sl = t % SL, sa = t % SA;
                const int k = t / KCH;
                const bool first = DRAIN ? (t % KCH == 0) : (t == 0);
                const uint32_t dt = tmem + (DRAIN ? (uint32_t)((k & 1) * p.N) : 0u);
                if (DRAIN && first && k >= 2 && !mbar_wait(&cempty[k & 1], ((k - 2) >> 1) & 1)) {
                    ok = false;
                    break;
                }
                if (!mbar_wait(&afull[sa], (t / SA) & 1) || !mbar_wait(&full[sl], (t / SL) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(abase + (size_t)sa * L.a_bytes);
                const uint32_t b0 = smem_u32(lbase + (size_t)sl * L.l_bytes);
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
                mma_commit(&empty[sl]);
                mma_commit(&aempty[sa]);
                if (DRAIN && (t % KCH == KCH - 1 || t == T - 1)) mma_commit(&cfull[k & 1]);
            }
            if (!ok) atomicOr(s_err, ERR_TIMEOUT);
            mma_commit(done);  // arrives once all issued MMAs completed
        }
    } else {
        // ---------------- eval warps: K tile into shared memory
        // thread (lane, warp): rows lane + 32 k (k = 0..3), j in [8 warp, 8 warp + 8)
        const int rg = lane;
        const int kq = warp;                // core-matrix column (8 j values) of this warp
        const int quad = warp & 3;          // TMEM lane quadrant of this warp
        const int halfc = warp >> 2;        // column half handled in drains/epilogue
        const int ncol_half = p.N / 2;
        // own coordinates, negated and duplicated into pairs
        float2 xr[4][8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (FROMM) break;
            const int r = rg + 32 * k;
            const float *tile = p.Xp + (size_t)(2 * blockIdx.x + (r >> 6)) * TJ * dd;
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const float v = a < dd ? -tile[a * TJ + (r & 63)] : 0.f;
                xr[k][a] = make_float2(v, v);
            }
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
        if (FROMM) {
            // stored M: unit k of this thread is row mr(k) = 16 warp + 8 (k >> 1) + lane % 8 and
            // the 8 columns 8 mq(k) .. 8 mq(k) + 7 of each tile, mq(k) = 4 (k & 1) + lane / 8, so
            // one warp-wide load covers 8 rows x 128 contiguous bytes (8 cache lines) and the
            // 8 lanes of each 16-byte store phase write 8 distinct rows (no bank conflicts)
            const float ms = __ldg(p.mscale);
            auto mr = [&](int k) { return 16 * warp + 8 * (k >> 1) + (lane & 7); };
            auto mq = [&](int k) { return 4 * (k & 1) + (lane >> 3); };
            const float *mrow[4];
            bool rok[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t i = row0 + mr(k);
                rok[k] = i < p.n;
                mrow[k] = p.M + (rok[k] ? i : 0) * p.n + mq(k) * 8;
            }
            // this thread's 4 x 8 values of tile t (zero past row or column n), streaming loads
            auto fetch = [&](int t, float4 (&b)[8]) {
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int64_t j = (int64_t)t * TJ + mq(k) * 8;
                    const float *src = mrow[k] + (int64_t)t * TJ;
                    if (p.vec4) {
                        // n % 4 == 0 and j % 8 == 0: each float4 lies wholly inside or past column n
                        b[2 * k] = (rok[k] && j < p.n) ? __ldcs(reinterpret_cast<const float4 *>(src)) : z;
                        b[2 * k + 1] =
                            (rok[k] && j + 4 < p.n) ? __ldcs(reinterpret_cast<const float4 *>(src + 4)) : z;
                    } else {
                        float e[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) e[q] = (rok[k] && j + q < p.n) ? __ldcs(src + q) : 0.f;
                        b[2 * k] = make_float4(e[0], e[1], e[2], e[3]);
                        b[2 * k + 1] = make_float4(e[4], e[5], e[6], e[7]);
                    }
                }
            };
            constexpr int PD = 3;  // tiles in flight per thread
            float4 buf[PD][8];
#pragma unroll
            for (int u = 0; u < PD; ++u)
                if (u < T) fetch(u, buf[u]);
            for (int t0 = 0; t0 < T && ok; t0 += PD) {
#pragma unroll
                for (int ph = 0; ph < PD; ++ph) {
                    const int t = t0 + ph;
                    if (t >= T) break;
                    const int sa = t % SA;
                    if (DRAIN && t % KCH == KCH / 2 && t >= KCH + KCH / 2) {
                        if (!drain(drained)) {
                            ok = false;
                            break;
                        }
                        ++drained;
                    }
                    if (t >= SA && !mbar_wait(&aempty[sa], ((t / SA) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    uint8_t *ast = abase + (size_t)sa * L.a_bytes;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float4 v0 = buf[ph][2 * k], v1 = buf[ph][2 * k + 1];
                        const float2 f[4] = {make_float2(v0.x * ms, v0.y * ms), make_float2(v0.z * ms, v0.w * ms),
                                             make_float2(v1.x * ms, v1.y * ms), make_float2(v1.z * ms, v1.w * ms)};
                        uint32_t w[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) w[q] = pack2<BF16>(f[q].x, f[q].y);
                        const int r = mr(k);
                        const size_t off = (size_t)(r >> 3) * 1024 + (size_t)mq(k) * 128 + (size_t)(r & 7) * 16;
                        *reinterpret_cast<uint4 *>(ast + off) = make_uint4(w[0], w[1], w[2], w[3]);
                        if (NPROD == 3) {
                            const float2 m1 = make_float2(-1.f, -1.f);
                            uint32_t l[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float2 rq = __ffma2_rn(unpack2<BF16>(w[q]), m1, f[q]);  // m - hi
                                l[q] = pack2<BF16>(rq.x, rq.y);
                            }
                            *reinterpret_cast<uint4 *>(ast + A_BYTES + off) = make_uint4(l[0], l[1], l[2], l[3]);
                        }
                    }
                    fence_async_smem();
                    mbar_arrive(&afull[sa]);
                    if (t + PD < T) fetch(t + PD, buf[ph]);
                }
            }
        }
        for (int t = 0; t < T && !FROMM; ++t) {
            const int sl = t % SL, sa = t % SA;
            if (DRAIN && t % KCH == KCH / 2 && t >= KCH + KCH / 2) {
                // chunk t / KCH - 1 finished half a chunk ago
                if (!drain(drained)) {
                    ok = false;
                    break;
                }
                ++drained;
            }
            if (!mbar_wait(&full[sl], (t / SL) & 1) || (t >= SA && !mbar_wait(&aempty[sa], ((t / SA) - 1) & 1))) {
                ok = false;
                break;
            }
            uint8_t *ast = abase + (size_t)sa * L.a_bytes;
            const float *xs = reinterpret_cast<const float *>(lbase + (size_t)sl * L.l_bytes + L.b_bytes);
            // the 8 points j of this warp, per coordinate (two 16-byte broadcast loads each)
            float2 xj[8][4];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                if (a < dd) {
                    const float4 lo4 = *reinterpret_cast<const float4 *>(xs + a * TJ + kq * 8);
                    const float4 hi4 = *reinterpret_cast<const float4 *>(xs + a * TJ + kq * 8 + 4);
                    xj[a][0] = make_float2(lo4.x, lo4.y);
                    xj[a][1] = make_float2(lo4.z, lo4.w);
                    xj[a][2] = make_float2(hi4.x, hi4.y);
                    xj[a][3] = make_float2(hi4.z, hi4.w);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t w[4];
                float2 f[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float2 u = make_float2(0.f, 0.f);
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        if (a < dd) {
                            const float2 dv = __fadd2_rn(xj[a][q], xr[k][a]);
                            u = __ffma2_rn(dv, dv, u);
                        }
                    }
                    f[q] = kval2<KIND>(u);
                    w[q] = pack2<BF16>(f[q].x, f[q].y);
                }
                const int r = rg + 32 * k;
                const size_t off = (size_t)(r >> 3) * 1024 + (size_t)kq * 128 + (size_t)(r & 7) * 16;
                *reinterpret_cast<uint4 *>(ast + off) = make_uint4(w[0], w[1], w[2], w[3]);
                if (NPROD == 3) {
                    const float2 m1 = make_float2(-1.f, -1.f);
                    uint32_t l[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 rq = __ffma2_rn(unpack2<BF16>(w[q]), m1, f[q]);  // k - hi
                        l[q] = pack2<BF16>(rq.x, rq.y);
                    }
                    *reinterpret_cast<uint4 *>(ast + A_BYTES + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
            }
            fence_async_smem();
            mbar_arrive(&afull[sa]);
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
            const float post = FROMM ? __ldg(p.mscale + 1) : 1.f;  // undo the scale of M
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
                            if (FROMM) {
                                p.W[i * p.c + col] = v[q] * post * p.colinv[c8 + q];
                            } else {
                                const float vin = p.V[i * p.c + col];
                                p.W[i * p.c + col] = v[q] * p.variance * p.colinv[c8 + q] + p.noise * vin;
                            }
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

// Point tiles for the kernel: per 64-point tile, coordinate-major (d x 64) so a
// pair of neighbouring points is one 8-byte load; coordinates scaled once more
// by `factor`; points past n are placed at PAD_COORD so every kernel value with them
// is exactly 0 (2^-x underflows) and no bounds test is needed.
__global__ void point_tiles_kernel(const float *Xs, int64_t n, int d, float factor, int64_t ntiles_alloc,
                                   float *Xp) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)TJ * d;
    if (idx >= per * ntiles_alloc) return;
    const int64_t t = idx / per;
    const int rem = (int)(idx % per);
    const int a = rem / TJ, jj = rem % TJ;
    const int64_t i = t * TJ + jj;
    Xp[idx] = i < n ? Xs[i * d + a] * factor : PAD_COORD;
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
    // power of two (exact rescaling)
    int e = 0;
    if (m > 0.f) {
        frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
    }
    // max |V_col| s in [KSCALE / 2, KSCALE): the lo part of the split stays out of
    // fp16 subnormals (as for the kernel values, tc_common.cuh)
    const float s = ldexpf(1.0f, KSCALE_LOG2 - e);
    scale[col] = s;
    colinv[col] = 1.0f / s;
}

// max_i |M_ii| over many blocks: the bit patterns of non-negative floats order like the
// floats, so an integer atomic max of them is the float max (NaN entries are skipped by
// fmaxf, as in a serial scan).  mx must be zero before the launch.
__global__ void diag_max_kernel(const float *M, int64_t n, unsigned *mx) {
    __shared__ float red[256];
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(M[i * n + i]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(mx, __float_as_uint(red[0]));
}

// Scale of a stored M: the power of two s with max_i |M_ii| s in [KSCALE / 2, KSCALE)
// (s = KSCALE when the diagonal is zero or not finite); for a positive semidefinite M
// every entry satisfies |M_ij| <= max_i M_ii, so every scaled entry lies in
// [-KSCALE, KSCALE], inside fp16's range with full precision down to ~1e-9 max M_ii
// (as for the computed kernel values).
__global__ void diag_scale_kernel(const unsigned *mx, float *mscale) {
    const float m = __uint_as_float(*mx);
    int e = 0;
    if (m > 0.f && isfinite(m)) frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
    mscale[0] = ldexpf(1.0f, KSCALE_LOG2 - e);
    mscale[1] = ldexpf(1.0f, e - KSCALE_LOG2);
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

// Load stages: as many as fit with two CTAs per SM (<= 113 KB each, 16 eval
// warps per SM); one CTA per SM only if even two stages do not fit.
int stages_for(int N, int d, int nprod) {
    for (int s = 6; s >= 2; --s)
        if (make_layout(N, d, nprod, s).total <= 113 * 1024) return s;
    for (int s = 4; s >= 2; --s)
        if (make_layout(N, d, nprod, s).total <= 220 * 1024) return s;
    return 2;
}

template <int KIND, int DC, int NPROD, bool BF16, bool DRAIN, bool FROMM = false>
int launch_main(const TcParams &p, const Layout &L, int nblocks, cudaStream_t st) {
    auto fn = kz_tc_kernel<KIND, DC, NPROD, BF16, DRAIN, FROMM>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) {
        set_error("kz_tc: cannot reserve %d bytes of shared memory: %s", L.total, cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    const double nn = (double)p.n * (double)p.n;
    const int slot = prof_begin_launch(st, FROMM ? PROF_DENSE : PROF_KZ_TC, nn, 2.0 * nn * p.N * NPROD);
    fn<<<nblocks, NTHREADS, L.total, st>>>(p, L);
    prof_end_launch(st, slot);
    return check_launch(FROMM ? "kz_tc_kernel (stored M)" : "kz_tc_kernel");
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

// Column scales and the operand image of columns c0 .. c0 + N - 1 of V.
int prep_chunk(const float *V, int64_t n, int c, int c0, int N, int64_t ntiles, int nprod, bool bf16, float *part,
               float *scale, float *colinv, uint8_t *img, cudaStream_t st) {
    const int nb = 256;
    colmax_kernel<<<nb, MAX_N, 0, st>>>(V, n, c, c0, N, part);
    colscale_kernel<<<1, MAX_N, 0, st>>>(part, nb, N, scale, colinv);
    const int64_t nthr = (int64_t)ntiles * N * 8;
    const unsigned gb = (unsigned)((nthr + 255) / 256);
    if (bf16) image_kernel<true, 1><<<gb, 256, 0, st>>>(V, n, c, c0, N, (int)ntiles, scale, img);
    else if (nprod == 3) image_kernel<false, 3><<<gb, 256, 0, st>>>(V, n, c, c0, N, (int)ntiles, scale, img);
    else image_kernel<false, 1><<<gb, 256, 0, st>>>(V, n, c, c0, N, (int)ntiles, scale, img);
    return check_launch("kz_tc prep", 3);
}

// TMEM columns: the next power of two >= cols (at least 32)
int tmem_cols(int cols) {
    return cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512)));
}

}  // namespace

size_t kz_tc_workspace(int64_t n, int d, int c, int precision) {
    if (kz_sym_eligible(n, d, c, precision)) return kz_sym_workspace(n, d, c, precision);
    if (kz_wide_eligible(n, d, c, precision)) return kz_wide_workspace(n, d, c, precision);
    const int64_t ntiles = (n + TJ - 1) / TJ;
    const int N = chunk_N(c);
    const int nprod = nprod_of(precision);
    Arena a;
    a.measuring = true;
    a.take<float>((size_t)(ntiles + 2) * TJ * d);                    // point tiles
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
    if (kz_sym_eligible(n, d, c, precision))
        return kz_sym(Xs, n, d, kind, variance, noise, V, W, c, precision, ws, st);
    if (kz_wide_eligible(n, d, c, precision))
        return kz_wide(Xs, n, d, kind, variance, noise, V, W, c, precision, ws, st);
    const int64_t ntiles = (n + TJ - 1) / TJ;
    const int nprod = nprod_of(precision);
    const bool bf16 = precision == LD_BF16_TC;
    const int Nmax = chunk_N(c);
    // carve from the caller's arena (already sized by kz_any_workspace)
    const size_t mark = ws.off;
    float *Xp = ws.take<float>((size_t)(ntiles + 2) * TJ * d);
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
        {
            // exponentials are evaluated as 2^-x: fold log2(e) into the coordinates
            const float factor = kind == LD_RBF ? 1.2011224087864498f /* sqrt(log2 e) */
                                                : 1.4426950408889634f /* log2 e */;
            const int64_t cnt = (ntiles + 2) * TJ * d;
            point_tiles_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(Xs, n, d, factor, ntiles + 2, Xp);
            LD_TRY(check_launch("point_tiles"));
        }
        LD_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        for (int c0 = 0; c0 < c; c0 += MAX_N) {
            const int N = chunk_N(std::min(MAX_N, c - c0));
            LD_TRY(prep_chunk(V, n, c, c0, N, ntiles, nprod, bf16, part, scale, colinv, img, st));
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
            p.ncols_tmem = tmem_cols(tcols);
            p.ntiles = (int)ntiles;
            p.variance = (float)variance * KSCALE_INV;  // kernel values carry KSCALE
            p.noise = (float)noise;
            p.err = err;
            p.M = nullptr;
            p.mscale = nullptr;
            p.vec4 = 0;
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

// ------------------------------------------------------- stored dense M
size_t dense_tc_workspace(int64_t n, int c, int precision) {
    const int64_t ntiles = (n + TJ - 1) / TJ;
    const int N = chunk_N(c);
    const int nprod = nprod_of(precision);
    Arena a;
    a.measuring = true;
    a.take<uint8_t>((size_t)ntiles * (nprod == 3 ? 2 : 1) * N * TJ * 2);  // operand image
    a.take<float>(MAX_N);                                                // scale
    a.take<float>(MAX_N);                                                // 1/scale
    a.take<float>((size_t)256 * MAX_N);                                  // colmax partials
    a.take<float>(4);                                                    // scale of M
    a.take<int>(4);                                                      // error word
    return a.off;
}

int dense_tc(const float *M, int64_t n, const float *V, float *W, int c, int precision, Arena &ws,
             cudaStream_t st) {
    if (n == 0 || c == 0) return LD_OK;
    if (precision != LD_F16_TC && precision != LD_BF16_TC && precision != LD_F16X3_TC) {
        set_error("dense_tc: not a tensor-core precision");
        return LD_ERR_INVALID;
    }
    const int64_t ntiles = (n + TJ - 1) / TJ;
    const int nprod = nprod_of(precision);
    const bool bf16 = precision == LD_BF16_TC;
    const int Nmax = chunk_N(c);
    const size_t mark = ws.off;
    uint8_t *img = ws.take<uint8_t>((size_t)ntiles * (nprod == 3 ? 2 : 1) * Nmax * TJ * 2);
    float *scale = ws.take<float>(MAX_N);
    float *colinv = ws.take<float>(MAX_N);
    float *part = ws.take<float>((size_t)256 * MAX_N);
    float *mscale = ws.take<float>(4);
    int *err = ws.take<int>(4);
    if (ws.overflow || !img) {
        set_error("dense_tc: workspace too small");
        ws.off = mark;
        return LD_ERR_WORKSPACE;
    }
    int code = [&]() -> int {
        unsigned *mx = reinterpret_cast<unsigned *>(mscale + 2);
        LD_CHECK_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned), st));
        diag_max_kernel<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, st>>>(M, n, mx);
        diag_scale_kernel<<<1, 1, 0, st>>>(mx, mscale);
        LD_TRY(check_launch("diag_scale", 2));
        LD_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        const bool vec4 = n % 4 == 0 && reinterpret_cast<uintptr_t>(M) % 16 == 0;
        for (int c0 = 0; c0 < c; c0 += MAX_N) {
            const int N = chunk_N(std::min(MAX_N, c - c0));
            LD_TRY(prep_chunk(V, n, c, c0, N, ntiles, nprod, bf16, part, scale, colinv, img, st));
            if (dense_tma_eligible(M, n, N, precision)) {  // M streamed by tensor copies
                LD_TRY(dense_tma(M, n, img, colinv, mscale, W, c, c0, N, precision, err, st));
                continue;
            }
            TcParams p;
            p.Xp = nullptr;
            p.img = img;
            p.V = V;
            p.colinv = colinv;
            p.W = W;
            p.n = n;
            p.d = 1;
            p.c = c;
            p.c0 = c0;
            p.N = N;
            const bool drain = nprod == 3 && N <= DRAIN_MAX_N;
            p.ncols_tmem = tmem_cols(drain ? 2 * N : N);
            p.ntiles = (int)ntiles;
            p.variance = 1.f;
            p.noise = 0.f;
            p.err = err;
            p.M = M;
            p.mscale = mscale;
            p.vec4 = vec4 ? 1 : 0;
            // no point tiles in the load stages; one CTA per SM (its registers hold three
            // tiles of M per thread in flight)
            Layout L = make_layout(N, 0, nprod, stages_for(N, 0, nprod));
            const int max_ctas = std::max(1, 512 / p.ncols_tmem);  // TMEM columns per SM
            L.total = std::max(L.total, (228 * 1024) / (max_ctas + 1) + 1024);
            const int nblocks = (int)((n + TM - 1) / TM);
            if (bf16) LD_TRY((launch_main<LD_RBF, 1, 1, true, false, true>(p, L, nblocks, st)));
            else if (nprod == 1) LD_TRY((launch_main<LD_RBF, 1, 1, false, false, true>(p, L, nblocks, st)));
            else if (drain) LD_TRY((launch_main<LD_RBF, 1, 3, false, true, true>(p, L, nblocks, st)));
            else LD_TRY((launch_main<LD_RBF, 1, 3, false, false, true>(p, L, nblocks, st)));
        }
        int herr = 0;
        LD_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        LD_CHECK_CUDA(cudaStreamSynchronize(st));
        if (herr) {
            set_error("dense_tc: a device-side wait timed out (error word %d)", herr);
            return LD_ERR_DEVICE_TIMEOUT;
        }
        return LD_OK;
    }();
    ws.off = mark;
    return code;
}

namespace {
// A wait that nothing completes: one thread waits on an mbarrier no one arrives at,
// with the same bounded wait the kernel product uses but a caller-chosen budget.
__global__ void wait_timeout_selftest_kernel(long long budget, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the same bounded wait the kernel products use, on a phase nothing completes
        *err = mbar_wait_budget(&bar, 0, budget) ? 0 : ERR_TIMEOUT;
    }
}
}  // namespace

}  // namespace ld

extern "C" int ld_selftest_wait_timeout(int64_t budget_cycles, void *stream) {
    ld::clear_error();
    if (budget_cycles < 0 || budget_cycles > 4000000000ll) {
        ld::set_error("ld_selftest_wait_timeout: budget must be in [0, 4e9] cycles");
        return LD_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int *d_err = nullptr;
    LD_CHECK_CUDA(cudaMalloc(&d_err, sizeof(int)));
    int herr = -1;
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        ld::wait_timeout_selftest_kernel<<<1, 32, 0, st>>>(budget_cycles, d_err);
        e = cudaGetLastError();
        ld::count_launches(1);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_err);
    if (e != cudaSuccess) {
        ld::set_error("ld_selftest_wait_timeout: %s", cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    if (herr) {
        ld::set_error("device-side wait gave up after %lld cycles (as intended by the self-test)",
                      (long long)budget_cycles);
        return LD_ERR_DEVICE_TIMEOUT;
    }
    return LD_OK;
}
