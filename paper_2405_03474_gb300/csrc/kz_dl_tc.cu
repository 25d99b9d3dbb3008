// Tensor-core pass of the gradient: W = K V and W_dl = (dK/dl) V in one sweep over the
// point pairs (Section 3's CG-based gradient of log det; the adjoint needs
// y^T (dM/dtheta) y for the shifted solutions y, dM/dl = dK/dl, dM/dv = K / v).
//
// Each CTA owns 128 rows i and sweeps all points j in tiles of 64 (as the general
// tensor-core product):
//   * 16 eval warps evaluate, per pair, the kernel value and its lengthscale
//     derivative from one squared distance, one MUFU sqrt and one MUFU ex2
//     (the exponential is shared), and write four 128 x 64 fp16 tiles into shared
//     memory: K and G = dK/dl, each split hi/lo (or rounded once in the single-
//     precision modes), in the canonical no-swizzle K-major layout;
//   * the MMA thread accumulates D1 += K [V_hi | V_lo] (+ K_lo V_hi) and
//     D2 += G [V_hi | V_lo] (+ G_lo V_hi) in two tensor-memory accumulators;
//   * every 8 tiles the eval warps drain both accumulators (ping-pong buffers) into
//     fp32 round-to-nearest sums held in registers, and write W and W_dl at the end.
// Up to 64 columns per launch (the host loops over column chunks).  Values carry
// KSCALE like the other tensor-core products; the epilogue applies
// variance / KSCALE (K) and the derivative's constant / KSCALE (G):
//   Matern-5/2, u = sqrt(5) r / l:  dk/dl = (v / l) (u^2 / 3) (1 + u) e^-u
//   RBF, u2 = r^2 / (2 l^2):        dk/dl = (2 v / l) u2 e^-u2.
// Every mbarrier wait is bounded; on a timeout the CTA sets the error word, skips
// the rest of its work and releases tensor memory.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace ld {

using namespace tc;

namespace {

constexpr int DM = 128;                  // rows per CTA (MMA M)
constexpr int DJ = 64;                   // j per tile (4 MMA K-steps of 16)
constexpr int DEVAL = 16;                // eval warps
constexpr int DTHREADS = (DEVAL + 2) * 32;
constexpr int DTILE = DM * DJ * 2;       // one 128 x 64 tile of halves (16 KB)
constexpr int DN = 64;                   // columns per launch (padded)
constexpr int DKCH = 8;                  // j-tiles accumulated in TMEM before a drain
constexpr int DCPT = DN / 4;             // columns per eval thread in drains (16)

struct DlParams {
    const float *Xp;     // per 64-point tile: d x 64 floats, far-padded, log2 e folded in
    const uint8_t *img;  // per tile: nprod x (DN x 64) halves (hi, then lo), canonical K-major
    const float *colinv; // 1 / column scale (DN)
    float *W, *Wdl;      // n x c (written, columns c0 .. c0 + DN - 1 below c)
    int64_t n;
    int d, c, c0, ntiles;
    float sk, sg;        // epilogue scales of D1 and D2
    int *err;
};

struct DlLayout {
    int sl, a_bytes, b_bytes, x_bytes, l_bytes, a_off, l_off, total;
};

DlLayout make_dl_layout(int d, int nprod, int sl) {
    DlLayout L;
    L.sl = sl;
    L.a_bytes = (nprod == 3 ? 4 : 2) * DTILE;  // K (hi, lo), G (hi, lo)
    L.b_bytes = (nprod == 3 ? 2 : 1) * DN * DJ * 2;
    L.x_bytes = DJ * d * 4;
    L.l_bytes = ((L.b_bytes + L.x_bytes + 1023) / 1024) * 1024;
    L.a_off = 1024;
    L.l_off = L.a_off + 2 * L.a_bytes;
    L.total = L.l_off + sl * L.l_bytes + 1024;  // + alignment slack of the dynamic base
    return L;
}

int dl_stages(int d, int nprod) {
    for (int s = 4; s >= 2; --s)
        if (make_dl_layout(d, nprod, s).total <= 225 * 1024) return s;
    return 0;
}

// KSCALE times the unit-variance kernel value k and the derivative factor g of two
// pairs from their squared scaled distances (coordinates carry log2 e, or
// sqrt(log2 e) for RBF, as for kval2), sharing the square root and the exponential:
//   Matern: u' = u log2 e, e = 2^-u', k = (1 + u + u^2/3) e,
//           g = (u^2 / 3) (1 + u) e = (ln2^2 / 3) u'^2 (1 + ln2 u') e
//   RBF:    e = 2^-u2', k = e, g = u2' e   (u2 = ln2 u2'; ln2 goes to the epilogue)
// g is formed as u2' (t e) so that the padding points (e = 0 exactly, u2' ~ 1e24)
// give 0, not inf x 0.
template <int KIND>
__device__ __forceinline__ void kdk2(float2 u2, float2 &k, float2 &g) {
    if (KIND == LD_RBF) {
        const float2 e = make_float2(mufu_ex2_neg(u2.x), mufu_ex2_neg(u2.y));
        k = __fmul2_rn(e, make_float2(KSCALE, KSCALE));
        g = __fmul2_rn(u2, k);
        return;
    }
    const float2 u = make_float2(mufu_sqrt(u2.x), mufu_sqrt(u2.y));
    const float2 e = make_float2(mufu_ex2_neg(u.x), mufu_ex2_neg(u.y));
    const float2 poly = __ffma2_rn(__ffma2_rn(u, make_float2(LN2SQ_3 * KSCALE, LN2SQ_3 * KSCALE),
                                              make_float2(LN2 * KSCALE, LN2 * KSCALE)),
                                   u, make_float2(KSCALE, KSCALE));
    k = __fmul2_rn(poly, e);
    const float2 t = __ffma2_rn(u, make_float2(LN2 * LN2SQ_3 * KSCALE, LN2 * LN2SQ_3 * KSCALE),
                                make_float2(LN2SQ_3 * KSCALE, LN2SQ_3 * KSCALE));
    g = __fmul2_rn(u2, __fmul2_rn(t, e));
}

// Round two values to fp16/bf16 (hi) and, for the split, the exact remainder (lo).
template <bool BF16, int NPROD>
__device__ __forceinline__ void round_split(float2 f, uint32_t &hi, uint32_t &lo) {
    hi = pack2<BF16>(f.x, f.y);
    if (NPROD == 3) {
        const float2 r = __ffma2_rn(unpack2<BF16>(hi), make_float2(-1.f, -1.f), f);
        lo = pack2<BF16>(r.x, r.y);
    }
}

// TMEM loads of 16 columns (32 lanes) as four x4 loads: issue, then wait before use.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
#pragma unroll
    for (int g = 0; g < 4; ++g)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[4 * g]), "=r"(r[4 * g + 1]), "=r"(r[4 * g + 2]), "=r"(r[4 * g + 3])
                     : "r"(taddr + 4u * g));
}
__device__ __forceinline__ void tmem_ld_wait2(uint32_t (&a)[16], uint32_t (&b)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) asm volatile("" : "+r"(a[q]), "+r"(b[q]));
}

template <int KIND, int DC, int NPROD, bool BF16>
__global__ void __launch_bounds__(DTHREADS, 1) kz_dl_tc_kernel(DlParams p, DlLayout L) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);  // [sl] loads landed
    uint64_t *empty = full + 8;                           // [sl] MMA done with the load stage
    uint64_t *afull = empty + 8;                          // [2] K / G tiles written
    uint64_t *aempty = afull + 2;                         // [2] MMA done with the tiles
    uint64_t *cfull = aempty + 2;                         // [2] chunk accumulated in TMEM
    uint64_t *cempty = cfull + 2;                         // [2] chunk drained
    uint64_t *done = cempty + 2;                          // every MMA finished
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    int *s_err = reinterpret_cast<int *>(tmem_slot + 1);
    uint8_t *abase = smem + L.a_off;
    uint8_t *lbase = smem + L.l_off;

    // tensor memory: D1 ping-pong [0, 2 NW), D2 ping-pong [2 NW, 4 NW); with the hi/lo
    // split an accumulator is [K_hi V_hi | K_hi V_lo + K_lo V_hi] (2 DN columns)
    constexpr uint32_t NW = NPROD == 3 ? 2 * DN : DN;
    constexpr uint32_t NCOLS = 4 * NW <= 256 ? 256 : 512;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int dd = DC > 0 ? DC : p.d;
    const int64_t row0 = (int64_t)blockIdx.x * DM;
    const int SL = L.sl;
    const int T = p.ntiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SL; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&afull[s], DEVAL * 32);
            mbar_init(&aempty[s], 1);
            mbar_init(&cfull[s], 1);
            mbar_init(&cempty[s], DEVAL * 32);
        }
        mbar_init(done, 1);
        *s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == DEVAL) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == DEVAL + 1) {
        // ---------------- producer: operand image of V and point tile per j-tile
        if (lane == 0) {
            const uint32_t xb = (uint32_t)(DJ * dd * 4);
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
                bulk_g2s(st + L.b_bytes, p.Xp + (size_t)t * DJ * dd, xb, &full[s]);
            }
            // every issued copy lands before the CTA may exit
            for (int u = std::max(0, t - SL); u < t; ++u)
                if (!mbar_wait(&full[u % SL], (u / SL) & 1)) atomicOr(s_err, ERR_TIMEOUT);
        }
    } else if (warp == DEVAL) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc_w = make_idesc(DM, (int)NW, BF16 ? 1u : 0u);  // B = [V_hi | V_lo]
            const uint32_t idesc = make_idesc(DM, DN, BF16 ? 1u : 0u);         // B = V_hi
            bool ok = true;
            for (int t = 0; t < T && ok; ++t) {
                const int sl = t % SL, sa = t & 1;
                const int k = t / DKCH;
                const bool first = t % DKCH == 0;
                const uint32_t d1 = tmem + (uint32_t)((k & 1) * NW);
                const uint32_t d2 = d1 + 2 * NW;
                if (first && k >= 2 && !mbar_wait(&cempty[k & 1], ((k - 2) >> 1) & 1)) {
                    ok = false;
                    break;
                }
                if (!mbar_wait(&afull[sa], (t >> 1) & 1) || !mbar_wait(&full[sl], (t / SL) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(abase + (size_t)sa * L.a_bytes);
                const uint32_t b0 = smem_u32(lbase + (size_t)sl * L.l_bytes);
                // K hi at a0, K lo at +DTILE, G hi at +2 DTILE (hi/lo) or +DTILE, G lo after it
                const uint64_t dk_hi = make_desc(a0, 128, 1024);
                const uint64_t dk_lo = dk_hi + (uint64_t)(DTILE >> 4);
                const uint64_t dg_hi = dk_hi + (uint64_t)(((NPROD == 3 ? 2 : 1) * DTILE) >> 4);
                const uint64_t dg_lo = dg_hi + (uint64_t)(DTILE >> 4);
                const uint64_t db = make_desc(b0, 128, 1024);  // NW rows: V_hi then V_lo
#pragma unroll
                for (int ks = 0; ks < DJ / 16; ++ks) {
                    const uint64_t step = (uint64_t)(ks * (256 >> 4));
                    const uint32_t acc = (first && ks == 0) ? 0u : 1u;
                    mma_f16(d1, dk_hi + step, db + step, idesc_w, acc);
                    mma_f16(d2, dg_hi + step, db + step, idesc_w, acc);
                    if (NPROD == 3) {
                        mma_f16(d1 + DN, dk_lo + step, db + step, idesc, 1u);
                        mma_f16(d2 + DN, dg_lo + step, db + step, idesc, 1u);
                    }
                }
                mma_commit(&empty[sl]);
                mma_commit(&aempty[sa]);
                if (t % DKCH == DKCH - 1 || t == T - 1) mma_commit(&cfull[k & 1]);
            }
            if (!ok) atomicOr(s_err, ERR_TIMEOUT);
            mma_commit(done);
            // every issued MMA completes before tensor memory is released
            if (!mbar_wait(done, 0)) atomicOr(s_err, ERR_TIMEOUT);
        }
    } else {
        // ---------------- eval warps: rows lane + 32 (2 rh + kk), kk = 0, 1, j in [8 kq, 8 kq + 8)
        const int kq = warp & 7;
        const int rh = warp >> 3;
        const int quad = warp & 3;    // TMEM lane quadrant (drains, epilogue)
        const int part = warp >> 2;   // column quarter (drains, epilogue)
        const uint32_t tlane = (uint32_t)(quad * 32) << 16;
        float2 xr[2][8];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int r = lane + 32 * (2 * rh + kk);
            const float *tile = p.Xp + (size_t)(2 * blockIdx.x + (r >> 6)) * DJ * dd;
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const float v = a < dd ? -tile[a * DJ + (r & 63)] : 0.f;
                xr[kk][a] = make_float2(v, v);
            }
        }
        float acc1[DCPT], acc2[DCPT];
#pragma unroll
        for (int q = 0; q < DCPT; ++q) acc1[q] = acc2[q] = 0.f;
        // waits never leave the loops: after the first timeout every later wait is skipped
        bool err_seen = false;
        auto wait_ok = [&](uint64_t *bar, uint32_t parity) {
            if (err_seen) return;
            if (!mbar_wait(bar, parity)) {
                atomicOr(s_err, ERR_TIMEOUT);
                err_seen = true;
            }
        };
        // chunk k of both accumulators -> fp32 sums (round to nearest)
        auto drain = [&](int k) {
            wait_ok(&cfull[k & 1], (k >> 1) & 1);
            tc_fence_after();
            const uint32_t ta = tmem + tlane + (uint32_t)((k & 1) * NW + part * DCPT);
            uint32_t h[DCPT], l[DCPT];
#pragma unroll
            for (int q = 0; q < DCPT; ++q) l[q] = 0u;
            tmem_ld16_issue(ta, h);
            if (NPROD == 3) tmem_ld16_issue(ta + DN, l);
            tmem_ld_wait2(h, l);
#pragma unroll
            for (int q = 0; q < DCPT; ++q) acc1[q] += __uint_as_float(h[q]) + __uint_as_float(l[q]);
            tmem_ld16_issue(ta + 2 * NW, h);
            if (NPROD == 3) tmem_ld16_issue(ta + 2 * NW + DN, l);
            tmem_ld_wait2(h, l);
#pragma unroll
            for (int q = 0; q < DCPT; ++q) acc2[q] += __uint_as_float(h[q]) + __uint_as_float(l[q]);
            tc_fence_before();
            mbar_arrive(&cempty[k & 1]);
        };
        const int C = (T + DKCH - 1) / DKCH;
        int drained = 0;
        for (int t = 0; t < T; ++t) {
            const int sl = t % SL, sa = t & 1;
            err_seen = err_seen || *reinterpret_cast<volatile int *>(s_err) != 0;
            // chunk t / DKCH - 1 finished half a chunk ago
            if (t % DKCH == DKCH / 2 && t >= DKCH + DKCH / 2) drain(drained++);
            wait_ok(&full[sl], (t / SL) & 1);
            if (t >= 2) wait_ok(&aempty[sa], ((t >> 1) - 1) & 1);
            uint8_t *ast = abase + (size_t)sa * L.a_bytes;
            uint8_t *gst = ast + (size_t)(NPROD == 3 ? 2 : 1) * DTILE;
            const float *xs = reinterpret_cast<const float *>(lbase + (size_t)sl * L.l_bytes + L.b_bytes);
            // the 8 points j of this warp, per coordinate (two 16-byte broadcast loads each)
            float2 xj[8][4];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                if (a < dd) {
                    const float4 lo4 = *reinterpret_cast<const float4 *>(xs + a * DJ + kq * 8);
                    const float4 hi4 = *reinterpret_cast<const float4 *>(xs + a * DJ + kq * 8 + 4);
                    xj[a][0] = make_float2(lo4.x, lo4.y);
                    xj[a][1] = make_float2(lo4.z, lo4.w);
                    xj[a][2] = make_float2(hi4.x, hi4.y);
                    xj[a][3] = make_float2(hi4.z, hi4.w);
                }
            }
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                uint32_t kh[4], kl[4], gh[4], gl[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float2 u = make_float2(0.f, 0.f);
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        if (a < dd) {
                            const float2 dv = __fadd2_rn(xj[a][q], xr[kk][a]);
                            u = __ffma2_rn(dv, dv, u);
                        }
                    }
                    float2 kv, gv;
                    kdk2<KIND>(u, kv, gv);
                    round_split<BF16, NPROD>(kv, kh[q], kl[q]);
                    round_split<BF16, NPROD>(gv, gh[q], gl[q]);
                }
                const int r = lane + 32 * (2 * rh + kk);
                const size_t off = (size_t)(r >> 3) * 1024 + (size_t)kq * 128 + (size_t)(r & 7) * 16;
                *reinterpret_cast<uint4 *>(ast + off) = make_uint4(kh[0], kh[1], kh[2], kh[3]);
                *reinterpret_cast<uint4 *>(gst + off) = make_uint4(gh[0], gh[1], gh[2], gh[3]);
                if (NPROD == 3) {
                    *reinterpret_cast<uint4 *>(ast + DTILE + off) = make_uint4(kl[0], kl[1], kl[2], kl[3]);
                    *reinterpret_cast<uint4 *>(gst + DTILE + off) = make_uint4(gl[0], gl[1], gl[2], gl[3]);
                }
            }
            fence_async_smem();
            mbar_arrive(&afull[sa]);
        }
        // ---------------- epilogue: remaining chunks, then W and W_dl
        wait_ok(done, 0);
        tc_fence_after();
        for (; drained < C; ++drained) drain(drained);
        const int64_t i = row0 + quad * 32 + lane;
        if (i < p.n && !err_seen && !*reinterpret_cast<volatile int *>(s_err)) {
#pragma unroll
            for (int q = 0; q < DCPT; ++q) {
                const int cc = part * DCPT + q;
                const int col = p.c0 + cc;
                if (col < p.c) {
                    const float ci = p.colinv[cc];
                    p.W[i * p.c + col] = acc1[q] * p.sk * ci;
                    p.Wdl[i * p.c + col] = acc2[q] * p.sg * ci;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == DEVAL) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
    }
    if (threadIdx.x == 0 && *s_err) atomicOr(p.err, *s_err);
}

// 64-point tiles, coordinate-major, log2 e folded in, points past n at PAD_COORD
__global__ void dl_point_tiles_kernel(const float *Xs, int64_t n, int d, float factor, int64_t ntiles, float *Xp) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)DJ * d;
    if (idx >= per * ntiles) return;
    const int64_t t = idx / per;
    const int rem = (int)(idx % per);
    const int a = rem / DJ, jj = rem % DJ;
    const int64_t i = t * DJ + jj;
    Xp[idx] = i < n ? Xs[i * d + a] * factor : PAD_COORD;
}

__global__ void dl_colmax_kernel(const float *V, int64_t n, int c, int c0, float *part) {
    const int col = threadIdx.x;
    const int nb = gridDim.x;
    const int64_t per = (n + nb - 1) / nb;
    const int64_t r0 = blockIdx.x * per, r1 = min(n, r0 + per);
    float m = 0.f;
    if (c0 + col < c)
        for (int64_t i = r0; i < r1; ++i) m = fmaxf(m, fabsf(V[i * c + c0 + col]));
    part[(size_t)blockIdx.x * DN + col] = m;
}

__global__ void dl_colscale_kernel(const float *part, int nb, float *scale, float *colinv) {
    const int col = threadIdx.x;
    float m = 0.f;
    for (int b = 0; b < nb; ++b) m = fmaxf(m, part[(size_t)b * DN + col]);
    int e = 0;
    if (m > 0.f) frexpf(m, &e);
    // max |V_col| s in [KSCALE / 2, KSCALE): the lo part stays out of fp16 subnormals
    const float s = ldexpf(1.0f, KSCALE_LOG2 - e);
    scale[col] = s;
    colinv[col] = 1.0f / s;
}

// Operand image of columns c0 .. c0 + DN - 1 of V per 64-point tile: hi (then lo) rows,
// DN x 64 K values each, canonical K-major (byte offset (col/8)*1024 + (jj/8)*128 +
// (col%8)*16 + (jj%8)*2).
template <bool BF16, int NPROD>
__global__ void dl_image_kernel(const float *V, int64_t n, int c, int c0, int ntiles, const float *scale,
                                uint8_t *img) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per_tile = (int64_t)DN * 8;
    if (idx >= per_tile * ntiles) return;
    const int64_t t = idx / per_tile;
    const int rem = (int)(idx % per_tile);
    const int cr = rem & 7;
    const int kq = (rem >> 3) & 7;
    const int g = rem >> 6;
    const int col = g * 8 + cr;
    const float s = scale[col];
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t j = t * DJ + kq * 8 + q;
        v[q] = (j < n && c0 + col < c) ? V[j * c + c0 + col] * s : 0.f;
    }
    uint4 hi;
    hi.x = pack2<BF16>(v[0], v[1]); hi.y = pack2<BF16>(v[2], v[3]);
    hi.z = pack2<BF16>(v[4], v[5]); hi.w = pack2<BF16>(v[6], v[7]);
    uint8_t *base = img + (size_t)t * (NPROD == 3 ? 2 : 1) * DN * DJ * 2;
    const size_t off = (size_t)g * 1024 + (size_t)kq * 128 + (size_t)cr * 16;
    *reinterpret_cast<uint4 *>(base + off) = hi;
    if (NPROD == 3) {
        uint4 lo;
        uint32_t *hp = &hi.x, *lp = &lo.x;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const float2 f = unpack2<BF16>(hp[w]);
            lp[w] = pack2<BF16>(v[2 * w] - f.x, v[2 * w + 1] - f.y);
        }
        *reinterpret_cast<uint4 *>(base + (size_t)DN * DJ * 2 + off) = lo;
    }
}

template <int KIND, int DC, int NPROD, bool BF16>
int launch_dl(const DlParams &p, const DlLayout &L, int nblocks, cudaStream_t st) {
    auto fn = kz_dl_tc_kernel<KIND, DC, NPROD, BF16>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) {
        set_error("kz_dl_tc: cannot reserve %d bytes of shared memory: %s", L.total, cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    // pairs: n^2 per launch (both products from each evaluated pair); flops: both products
    const double nn = (double)p.n * (double)p.n;
    const int slot = prof_begin_launch(st, PROF_KZ_DL, nn, 2.0 * 2.0 * nn * DN * NPROD);
    fn<<<nblocks, DTHREADS, L.total, st>>>(p, L);
    prof_end_launch(st, slot);
    return check_launch("kz_dl_tc_kernel");
}

template <int KIND, int NPROD, bool BF16>
int launch_dl_d(const DlParams &p, const DlLayout &L, int nblocks, cudaStream_t st) {
    switch (p.d) {
        case 1: return launch_dl<KIND, 1, NPROD, BF16>(p, L, nblocks, st);
        case 2: return launch_dl<KIND, 2, NPROD, BF16>(p, L, nblocks, st);
        case 3: return launch_dl<KIND, 3, NPROD, BF16>(p, L, nblocks, st);
        case 4: return launch_dl<KIND, 4, NPROD, BF16>(p, L, nblocks, st);
        default: return launch_dl<KIND, 0, NPROD, BF16>(p, L, nblocks, st);
    }
}

}  // namespace

size_t kz_dl_tc_workspace(int64_t n, int d, int precision) {
    const int64_t ntiles = (n + DJ - 1) / DJ;
    const int nprod = precision == LD_F16X3_TC ? 3 : 1;
    Arena a;
    a.measuring = true;
    a.take<float>((size_t)(ntiles + 2) * DJ * d);                      // point tiles
    a.take<uint8_t>((size_t)ntiles * (nprod == 3 ? 2 : 1) * DN * DJ * 2);  // operand image
    a.take<float>(DN);                                                 // scale
    a.take<float>(DN);                                                 // 1 / scale
    a.take<float>((size_t)256 * DN);                                   // colmax partials
    a.take<int>(4);                                                    // error word
    return a.off;
}

int kz_dl_tc(const float *Xs, int64_t n, int d, int kind, double lengthscale, double variance, const float *V,
             float *W, float *Wdl, int c, int precision, Arena &ws, cudaStream_t st) {
    NvtxRange range("ld: derivative product");
    if (n == 0 || c == 0) return LD_OK;
    if (d > 8 || !is_tc_precision(precision)) {
        set_error("kz_dl_tc: tensor-core precision and d <= 8 required");
        return LD_ERR_INVALID;
    }
    const int64_t ntiles = (n + DJ - 1) / DJ;
    const int nprod = precision == LD_F16X3_TC ? 3 : 1;
    const bool bf16 = precision == LD_BF16_TC;
    const size_t mark = ws.off;
    float *Xp = ws.take<float>((size_t)(ntiles + 2) * DJ * d);
    uint8_t *img = ws.take<uint8_t>((size_t)ntiles * (nprod == 3 ? 2 : 1) * DN * DJ * 2);
    float *scale = ws.take<float>(DN);
    float *colinv = ws.take<float>(DN);
    float *part = ws.take<float>((size_t)256 * DN);
    int *err = ws.take<int>(4);
    if (ws.overflow || !Xp) {
        set_error("kz_dl_tc: workspace too small");
        ws.off = mark;
        return LD_ERR_WORKSPACE;
    }
    int code = [&]() -> int {
        const float factor = kind == LD_RBF ? 1.2011224087864498f /* sqrt(log2 e) */
                                            : 1.4426950408889634f /* log2 e */;
        const int64_t cnt = (ntiles + 2) * DJ * d;
        dl_point_tiles_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(Xs, n, d, factor, ntiles + 2, Xp);
        LD_TRY(check_launch("kz_dl_tc point tiles"));
        LD_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        const int sl = dl_stages(d, nprod);
        const DlLayout L = make_dl_layout(d, nprod, sl);
        for (int c0 = 0; c0 < c; c0 += DN) {
            dl_colmax_kernel<<<256, DN, 0, st>>>(V, n, c, c0, part);
            dl_colscale_kernel<<<1, DN, 0, st>>>(part, 256, scale, colinv);
            const int64_t nthr = ntiles * DN * 8;
            const unsigned gb = (unsigned)((nthr + 255) / 256);
            if (bf16) dl_image_kernel<true, 1><<<gb, 256, 0, st>>>(V, n, c, c0, (int)ntiles, scale, img);
            else if (nprod == 3) dl_image_kernel<false, 3><<<gb, 256, 0, st>>>(V, n, c, c0, (int)ntiles, scale, img);
            else dl_image_kernel<false, 1><<<gb, 256, 0, st>>>(V, n, c, c0, (int)ntiles, scale, img);
            LD_TRY(check_launch("kz_dl_tc prep", 3));
            DlParams p;
            p.Xp = Xp;
            p.img = img;
            p.colinv = colinv;
            p.W = W;
            p.Wdl = Wdl;
            p.n = n;
            p.d = d;
            p.c = c;
            p.c0 = c0;
            p.ntiles = (int)ntiles;
            // kernel values carry KSCALE; dk/dl = (v / l) g (Matern), (2 v ln2 / l) g (RBF)
            p.sk = (float)(variance * KSCALE_INV);
            p.sg = (float)((kind == LD_RBF ? 2.0 * 0.69314718055994531 : 1.0) * variance / lengthscale * KSCALE_INV);
            p.err = err;
            const int nblocks = (int)((n + DM - 1) / DM);
            if (kind == LD_RBF) {
                if (bf16) LD_TRY(launch_dl_d<LD_RBF, 1, true>(p, L, nblocks, st));
                else if (nprod == 3) LD_TRY(launch_dl_d<LD_RBF, 3, false>(p, L, nblocks, st));
                else LD_TRY(launch_dl_d<LD_RBF, 1, false>(p, L, nblocks, st));
            } else {
                if (bf16) LD_TRY(launch_dl_d<LD_MATERN52, 1, true>(p, L, nblocks, st));
                else if (nprod == 3) LD_TRY(launch_dl_d<LD_MATERN52, 3, false>(p, L, nblocks, st));
                else LD_TRY(launch_dl_d<LD_MATERN52, 1, false>(p, L, nblocks, st));
            }
        }
        int herr = 0;
        LD_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        LD_CHECK_CUDA(cudaStreamSynchronize(st));
        if (herr) {
            set_error("kz_dl_tc: a device-side wait timed out (error word %d)", herr);
            return LD_ERR_DEVICE_TIMEOUT;
        }
        return LD_OK;
    }();
    ws.off = mark;
    return code;
}

}  // namespace ld
