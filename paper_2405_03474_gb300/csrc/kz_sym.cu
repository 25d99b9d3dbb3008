// Symmetric tensor-core kernel product W = (K + noise I) V for up to 48 columns
// (the CG passes: one column per probe; the residual pass: probes x shifts),
// evaluating each kernel value once.
//
// K is symmetric, so the 128 x 128 block K_IJ serves two products: W_I += K_IJ V_J
// and W_J += K_IJ^T V_I.  The CTA owning row block I visits the blocks
// J = (I + b) mod NB, b = 0 .. NB/2 (for even NB the block at distance NB/2 goes
// to the smaller I only), so every unordered pair of blocks is evaluated once and
// the work per CTA is balanced.  Per block:
//   * 16 eval warps evaluate the 128 x 128 tile into shared memory (packed f32x2
//     differences and polynomial, one MUFU sqrt + ex2 per pair, fp16 hi/lo);
//   * the MMA thread issues D_I += K_IJ V_J (K-major A: rows i, K = j) and
//     D'_J = K_IJ^T V_I (the same shared tile read as an MN-major A: rows j, K = i);
//   * two blocks later the eval warps read D'_J from tensor memory (the load is
//     issued before the next tile's evaluation and completed after it) and add it
//     into W_J, each thread one 16-byte vector reduction (red.global.add.v4.f32)
//     of 4 columns of one row.
// The product accumulates into a zeroed buffer in tile order; every contribution
// (including the owner's own rows, at the end) is added, so the order of additions
// across CTAs is the only run-to-run difference (fp32 rounding).  D_I is accumulated in tensor
// memory in chunks of 4 blocks and drained to fp32 round-to-nearest partial
// sums, held in registers (each eval thread owns a quarter of one row's columns),
// as in the non-symmetric kernel.  The kernel is compiled for SN = 16 and SN = 48
// columns (padded).  Every mbarrier wait is bounded.
//
// The tiles hold the points in Morton order (point_order.cu), so most tiles are compact
// and most pairs of tiles are far apart.  With the hi/lo split, a block whose tiles'
// boxes are so far apart that every kernel value is <= 2^-10 (of the variance) is rounded
// to fp16 once and its K_lo products are skipped: one rounding of such values errs by at
// most 2^-21, no more than the split does near 1.  The tile-order product is scattered
// back to the caller's order by one pass that also adds the noise term.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "tc_common.cuh"

namespace ld {

using namespace tc;

namespace {

constexpr int BR = 128;                     // block rows and block columns
constexpr int SNEVAL = 16;                  // eval warps
constexpr int SNTHREADS = (SNEVAL + 2) * 32;
constexpr int HALF_TILE = BR * BR * 2;      // one 128 x 128 tile of halves (32 KB)
constexpr int SKCH = 4;                     // blocks per TMEM chunk before a drain (hi/lo)
constexpr int CORE_SBO = (BR / 8) * 128;    // 2048: byte step between 8-row groups
constexpr int SN_MAX = 48;

struct SymParams {
    const float *tbox;   // per tile: d minima then d maxima of its coordinates (kernel units)
    float thr2;          // squared distance (kernel units) beyond which k <= 2^-10: one fp16 rounding
    int far_on;          // 1: blocks between tiles at least sqrt(thr2) apart skip the hi/lo split
    const float *Xp;     // per 128-point tile: d x 128 floats, far-padded, log2 e folded in
    const uint8_t *img;  // per 128-point tile: nprod x (SN x 128) halves, canonical K-major
    const float *colinv; // 1 / column scale (SN)
    float *W;            // n x c in tile order (row r is point perm[r]); zeroed, every contribution added
    int64_t n;
    int d, c, NB, ncols_tmem, vec_ok;
    float variance;
    int *err;
};

struct SymLayout {
    int sl, a_bytes, b_bytes, x_bytes, l_bytes;
    int a_off, l_off, vi_off, total;
};

inline int round1k(int b) { return ((b + 1023) / 1024) * 1024; }

SymLayout make_sym_layout(int sn, int d, int nprod, int sl) {
    SymLayout L;
    L.sl = sl;
    L.a_bytes = (nprod == 3 ? 2 : 1) * HALF_TILE;
    L.b_bytes = (nprod == 3 ? 2 : 1) * sn * BR * 2;
    L.x_bytes = BR * d * 4;
    L.l_bytes = round1k(L.b_bytes + L.x_bytes);
    L.a_off = 1024;
    L.l_off = L.a_off + 2 * L.a_bytes;
    L.vi_off = L.l_off + sl * L.l_bytes;
    L.total = L.vi_off + round1k(L.b_bytes) + 1024;
    return L;
}

int sym_stages(int sn, int d, int nprod) {
    for (int s = 4; s >= 2; --s)
        if (make_sym_layout(sn, d, nprod, s).total <= 225 * 1024) return s;
    return 0;
}

// Asynchronous TMEM loads of G x 4 columns (32 lanes): issue, then wait before use.  The
// wait names the destination registers so no use is scheduled ahead of it.
template <int G>
__device__ __forceinline__ void tmem_ld_issue(uint32_t taddr, uint32_t (&r)[4 * G]) {
#pragma unroll
    for (int g = 0; g < G; ++g)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[4 * g]), "=r"(r[4 * g + 1]), "=r"(r[4 * g + 2]), "=r"(r[4 * g + 3])
                     : "r"(taddr + 4u * g));
}
template <int G>
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[4 * G], uint32_t (&t)[4 * G]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 4 * G; ++q) asm volatile("" : "+r"(r[q]), "+r"(t[q]));
}

template <int KIND, int DC, int NPROD, bool BF16, int SN>
__global__ void __launch_bounds__(SNTHREADS, 1) kz_sym_kernel(SymParams p, SymLayout L) {
    constexpr bool DRAIN = NPROD == 3;
    constexpr int CPT = SN / 4;   // columns per eval thread (a quarter of a row)
    constexpr int G4 = CPT / 4;   // groups of 4 columns per thread
    // the D' load is issued before the next tile's evaluation and completed after it
    // when its registers fit beside the evaluation's (16 columns)
    constexpr bool ASYNC_T = SN == 16;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);  // [sl]
    uint64_t *empty = full + 8;                           // [sl]
    uint64_t *afull = empty + 8;                          // [2]
    uint64_t *aempty = afull + 2;                         // [2]
    uint64_t *vfull = aempty + 2;                         // own V image landed
    uint64_t *done = vfull + 1;
    uint64_t *cfull = done + 1;                           // [2] D chunk in TMEM
    uint64_t *cempty = cfull + 2;                         // [2] D chunk drained
    uint64_t *tfull = cempty + 2;                         // [2] D' of a block in TMEM
    uint64_t *tempty = tfull + 2;                         // [2] D' drained
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    int *s_err = reinterpret_cast<int *>(tmem_slot + 1);
    // per load stage: 1 if the block in it is far (single fp16, no K_lo products); written
    // by the producer before the stage's copies are issued, read after its full barrier
    volatile int *s_far = reinterpret_cast<volatile int *>(s_err + 1);
    uint8_t *abase = smem + L.a_off;
    uint8_t *lbase = smem + L.l_off;
    uint8_t *vimg = smem + L.vi_off;
    // variance / column scale per column, read at each drain (not held in registers)
    float *s_cscale = reinterpret_cast<float *>(smem + 512);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int dd = DC > 0 ? DC : p.d;
    const int I = blockIdx.x;
    const int NB = p.NB, H = NB / 2;
    const int T = (NB & 1) ? H + 1 : (I < H ? H + 1 : H);  // blocks J = (I + b) % NB
    const int SL = L.sl;
    // With the hi/lo split an accumulator is 2 SN columns wide: [K_hi V_hi | K_hi V_lo + K_lo V_hi]
    // (one N = 2 SN MMA reads the K_hi tile once for both V halves); the halves are summed when
    // drained.  D ping-pong (drained) or single D, then the two D' buffers.
    constexpr uint32_t NW = NPROD == 3 ? 2 * SN : SN;
    const uint32_t doff = DRAIN ? 2 * NW : NW;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SL; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&afull[s], SNEVAL * 32);
            mbar_init(&aempty[s], 1);
            mbar_init(&cfull[s], 1);
            mbar_init(&cempty[s], SNEVAL * 32);
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], SNEVAL * 32);
        }
        mbar_init(vfull, 1);
        mbar_init(done, 1);
        *s_err = 0;
        for (int q = 0; q < SN; ++q) s_cscale[q] = p.variance * p.colinv[q];
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == SNEVAL) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(p.ncols_tmem)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == SNEVAL + 1) {
        // ---------------- producer: lane 0 issues the copies; the warp classifies the next
        // 32 blocks at a time (one box test per lane, one ballot), so no per-block load
        // waits in front of a copy
        const uint32_t xb = (uint32_t)(BR * dd * 4);
        const uint32_t bb = (uint32_t)L.b_bytes;
        float blo[8], bhi[8];  // this CTA's tile box
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            blo[a] = a < dd ? p.tbox[(size_t)I * 2 * dd + a] : 0.f;
            bhi[a] = a < dd ? p.tbox[(size_t)I * 2 * dd + dd + a] : 0.f;
        }
        if (lane == 0) {
            mbar_expect_tx(vfull, bb);
            bulk_g2s(vimg, p.img + (size_t)I * bb, bb, vfull);
        }
        int b = 0;
        int J = I;
        bool stop = false;
        for (int b0 = 0; b0 < T && !stop; b0 += 32) {
            // far: the boxes of tiles I and Jl are at least sqrt(thr2) apart
            bool f = false;
            const int bl = b0 + lane;
            if (p.far_on && bl < T) {
                const int Jl = (I + bl) % NB;
                float gap2 = 0.f;
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    if (a < dd) {
                        const float lj = p.tbox[(size_t)Jl * 2 * dd + a], hj = p.tbox[(size_t)Jl * 2 * dd + dd + a];
                        const float g = fmaxf(0.f, fmaxf(lj - bhi[a], blo[a] - hj));
                        gap2 = fmaf(g, g, gap2);
                    }
                }
                f = gap2 >= p.thr2;
            }
            const uint32_t fm = __ballot_sync(0xffffffffu, f);
            if (lane == 0) {
                const int bend = min(T, b0 + 32);
                for (; b < bend; ++b, J = (J + 1 == NB) ? 0 : J + 1) {
                    const int s = b % SL;
                    if (b >= SL && !mbar_wait(&empty[s], ((b / SL) - 1) & 1)) {
                        atomicOr(s_err, ERR_TIMEOUT);
                        stop = true;
                        break;
                    }
                    uint8_t *st = lbase + (size_t)s * L.l_bytes;
                    s_far[s] = (int)((fm >> (b - b0)) & 1u);
                    mbar_expect_tx(&full[s], xb + bb);
                    bulk_g2s(st, p.img + (size_t)J * bb, bb, &full[s]);
                    bulk_g2s(st + L.b_bytes, p.Xp + (size_t)J * BR * dd, xb, &full[s]);
                }
            }
            stop = __shfl_sync(0xffffffffu, stop ? 1 : 0, 0) != 0;
        }
        if (lane == 0) {
            for (int u = b - SL > 0 ? b - SL : 0; u < b; ++u)
                if (!mbar_wait(&full[u % SL], (u / SL) & 1)) atomicOr(s_err, ERR_TIMEOUT);
            if (!mbar_wait(vfull, 0)) atomicOr(s_err, ERR_TIMEOUT);
        }
    } else if (warp == SNEVAL) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = make_idesc(BR, SN, BF16 ? 1u : 0u, 0u);
            const uint32_t idesc_t = make_idesc(BR, SN, BF16 ? 1u : 0u, 1u);  // A read MN-major
            const uint32_t idesc_w = make_idesc(BR, (int)NW, BF16 ? 1u : 0u, 0u);  // B = [V_hi | V_lo]
            const uint32_t idesc_wt = make_idesc(BR, (int)NW, BF16 ? 1u : 0u, 1u);
            bool ok = mbar_wait(vfull, 0);
            const uint64_t dvi = make_desc(smem_u32(vimg), 128, CORE_SBO);
            for (int b = 0; b < T && ok; ++b) {
                const int s = b % SL, sa = b & 1;
                const int k = b / SKCH;
                const bool first = DRAIN ? (b % SKCH == 0) : (b == 0);
                const uint32_t dt = tmem + (DRAIN ? (uint32_t)((k & 1) * NW) : 0u);
                if (DRAIN && first && k >= 2 && !mbar_wait(&cempty[k & 1], ((k - 2) >> 1) & 1)) {
                    ok = false;
                    break;
                }
                if (b >= 3 && !mbar_wait(&tempty[b & 1], ((b - 3) >> 1) & 1)) {
                    ok = false;
                    break;
                }
                if (!mbar_wait(&afull[sa], (b >> 1) & 1) || !mbar_wait(&full[s], (b / SL) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const bool lo = NPROD == 3 && !s_far[s];  // K_lo products (near blocks only)
                // Descriptors advance by a constant per K-step (the start address field is
                // address >> 4 and no step carries out of it), so they are formed once.
                const uint32_t a0 = smem_u32(abase + (size_t)sa * L.a_bytes);
                const uint32_t b0 = smem_u32(lbase + (size_t)s * L.l_bytes);
                // D_I += K_IJ V_J: A K-major (lbo = 128 along j, sbo = 2048 along i)
                const uint64_t dah = make_desc(a0, 128, CORE_SBO);
                const uint64_t dal = dah + (uint64_t)(HALF_TILE >> 4);
                const uint64_t dbh = make_desc(b0, 128, CORE_SBO);  // N = NW spans hi, lo
#pragma unroll
                for (int ks = 0; ks < BR / 16; ++ks) {
                    const uint64_t step = (uint64_t)(ks * (256 >> 4));
                    mma_f16(dt, dah + step, dbh + step, idesc_w, (first && ks == 0) ? 0u : 1u);
                    if (lo) mma_f16(dt + SN, dal + step, dbh + step, idesc, 1u);
                }
                if (b >= 1) {
                    // D'_J = K_IJ^T V_I: the same tile MN-major (rows j; lbo = 2048 along i,
                    // sbo = 128 along j), B = own V image (K = i)
                    const uint32_t tdt = tmem + doff + (uint32_t)((b & 1) * NW);
                    const uint64_t dat = make_desc(a0, CORE_SBO, 128);
                    const uint64_t dalt = dat + (uint64_t)(HALF_TILE >> 4);
#pragma unroll
                    for (int ks = 0; ks < BR / 16; ++ks) {
                        const uint64_t astep = (uint64_t)(ks * ((2 * CORE_SBO) >> 4));
                        const uint64_t bstep = (uint64_t)(ks * (256 >> 4));
                        mma_f16(tdt, dat + astep, dvi + bstep, idesc_wt, ks == 0 ? 0u : 1u);
                        if (lo) mma_f16(tdt + SN, dalt + astep, dvi + bstep, idesc_t, 1u);
                    }
                    mma_commit(&tfull[b & 1]);
                }
                mma_commit(&empty[s]);
                mma_commit(&aempty[sa]);
                if (DRAIN && (b % SKCH == SKCH - 1 || b == T - 1)) mma_commit(&cfull[k & 1]);
            }
            if (!ok) atomicOr(s_err, ERR_TIMEOUT);
            mma_commit(done);
            // every issued MMA has finished before tensor memory is released below
            if (!mbar_wait(done, 0)) atomicOr(s_err, ERR_TIMEOUT);
        }
    } else {
        // ---------------- eval warps: rows lane + 32 k (k = 0..3), j in [8 warp, 8 warp + 8)
        const int rg = lane;
        const int kq = warp;
        const int quad = warp & 3;       // TMEM lane quadrant
        const int part = warp >> 2;      // a quarter of the columns in drains / epilogue
        const int c0 = part * CPT;
        const int row = quad * 32 + lane;
        const uint32_t tlane = (uint32_t)(quad * 32) << 16;
        float2 xr[4][8];
        {
            const float *tile = p.Xp + (size_t)I * BR * dd;
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const float v = a < dd ? -tile[a * BR + rg + 32 * k] : 0.f;
                    xr[k][a] = make_float2(v, v);
                }
        }
        // column scales: registers for 16 columns (4 per thread), shared memory for 48
        float cs_reg[SN == 16 ? CPT : 1];
        if (SN == 16)
#pragma unroll
            for (int q = 0; q < (SN == 16 ? CPT : 1); ++q) cs_reg[q] = s_cscale[c0 + q];
        auto cscale_of = [&](int q) -> float { return SN == 16 ? cs_reg[q] : s_cscale[c0 + q]; };
        float acc[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q] = 0.f;

        // Waits of the eval threads never leave the loop: after the first timeout (error
        // word set) every later wait is skipped and nothing more is added to W, so all
        // threads finish quickly.
        // (the shared error word is read once per block into err_seen)
        bool err_seen = false;
        auto wait_ok = [&](uint64_t *bar, uint32_t parity) {
            if (err_seen) return;
            if (!mbar_wait(bar, parity)) {
                atomicOr(s_err, ERR_TIMEOUT);
                err_seen = true;
            }
        };
        // D chunk k -> fp32 partial sums in registers
        auto drain_d = [&](int k) {
            wait_ok(&cfull[k & 1], (k >> 1) & 1);
            tc_fence_after();
            uint32_t h[CPT], l[CPT];
            const uint32_t ta = tmem + tlane + (uint32_t)((k & 1) * NW + c0);
            tmem_ld_issue<G4>(ta, h);
            tmem_ld_issue<G4>(ta + SN, l);
            tmem_ld_wait<G4>(h, l);
#pragma unroll
            for (int q = 0; q < CPT; ++q) acc[q] += __uint_as_float(h[q]) + __uint_as_float(l[q]);
            tc_fence_before();
            mbar_arrive(&cempty[k & 1]);
        };
        // Add CPT values of one W row (columns c0 ..): 16-byte vector reductions when rows
        // are 16-byte aligned, else per element.
        auto add_row = [&](int64_t grow, const float (&val)[CPT]) {
            float *dst = p.W + grow * p.c + c0;
            if (p.vec_ok) {
#pragma unroll
                for (int g = 0; g < G4; ++g)
                    if (c0 + 4 * g < p.c)
                        atomicAdd(reinterpret_cast<float4 *>(dst + 4 * g),
                                  make_float4(val[4 * g], val[4 * g + 1], val[4 * g + 2], val[4 * g + 3]));
            } else {
#pragma unroll
                for (int q = 0; q < CPT; ++q)
                    if (c0 + q < p.c) atomicAdd(dst + q, val[q]);
            }
        };
        // D' of block bb -> W rows of block J = (I + bb) % NB
        uint32_t tr[CPT], tl[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) tr[q] = tl[q] = 0u;
        auto drain_t_issue = [&](int bb) {
            wait_ok(&tfull[bb & 1], ((bb - 1) >> 1) & 1);
            tc_fence_after();
            const uint32_t ta = tmem + tlane + doff + (uint32_t)((bb & 1) * NW + c0);
            tmem_ld_issue<G4>(ta, tr);
            if (NPROD == 3) tmem_ld_issue<G4>(ta + SN, tl);
        };
        auto drain_t_finish = [&](int bb) {
            tmem_ld_wait<G4>(tr, tl);
            tc_fence_before();
            mbar_arrive(&tempty[bb & 1]);
            int J = I + bb;
            if (J >= NB) J -= NB;
            const int64_t gj = (int64_t)J * BR + row;  // W row in tile order
            if (gj < p.n && !err_seen) {
                float val[CPT];
#pragma unroll
                for (int q = 0; q < CPT; ++q)
                    val[q] = (NPROD == 3 ? __uint_as_float(tr[q]) + __uint_as_float(tl[q]) : __uint_as_float(tr[q])) *
                             cscale_of(q);
                add_row(gj, val);
            }
        };

        const int C = (T + SKCH - 1) / SKCH;
        int drained = 0;
        for (int b = 0; b < T; ++b) {
            const int s = b % SL, sa = b & 1;
            err_seen = err_seen || *reinterpret_cast<volatile int *>(s_err) != 0;
            if (DRAIN && b % SKCH == SKCH / 2 && b >= SKCH + SKCH / 2) drain_d(drained++);
            if (b >= 3) {
                drain_t_issue(b - 2);
                if (!ASYNC_T) drain_t_finish(b - 2);
            }
            wait_ok(&full[s], (b / SL) & 1);
            if (b >= 2) wait_ok(&aempty[sa], ((b >> 1) - 1) & 1);
            uint8_t *ast = abase + (size_t)sa * L.a_bytes;
            const float *xs = reinterpret_cast<const float *>(lbase + (size_t)s * L.l_bytes + L.b_bytes);
            float2 xj[8][4];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                if (a < dd) {
                    const float4 lo4 = *reinterpret_cast<const float4 *>(xs + a * BR + kq * 8);
                    const float4 hi4 = *reinterpret_cast<const float4 *>(xs + a * BR + kq * 8 + 4);
                    xj[a][0] = make_float2(lo4.x, lo4.y);
                    xj[a][1] = make_float2(lo4.z, lo4.w);
                    xj[a][2] = make_float2(hi4.x, hi4.y);
                    xj[a][3] = make_float2(hi4.z, hi4.w);
                }
            }
            // near block: hi/lo split; far block: one fp16 rounding.  The choice is uniform
            // over the block, so each form is compiled on its own (no predicated double work).
            auto eval_tile = [&](auto split_tag) {
                constexpr bool SPLIT = decltype(split_tag)::value;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t w[4], l[4];
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
                        const float2 f = kval2<KIND>(u);
                        if (SPLIT) split_f16(f, w[q], l[q]);
                        else w[q] = pack2<BF16>(f.x, f.y);
                    }
                    const int r = rg + 32 * k;
                    const size_t off = (size_t)(r >> 3) * CORE_SBO + (size_t)kq * 128 + (size_t)(r & 7) * 16;
                    *reinterpret_cast<uint4 *>(ast + off) = make_uint4(w[0], w[1], w[2], w[3]);
                    if (SPLIT) *reinterpret_cast<uint4 *>(ast + HALF_TILE + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
            };
            if (NPROD == 3 && !s_far[s]) eval_tile(std::true_type{});
            else eval_tile(std::false_type{});
            fence_async_smem();
            // D' buffer (b - 2) & 1 is released before this tile's MMA needs it
            if (ASYNC_T && b >= 3) drain_t_finish(b - 2);
            mbar_arrive(&afull[sa]);
        }
        // ---------------- tail: remaining transposed blocks, D chunks, own rows
        err_seen = err_seen || *reinterpret_cast<volatile int *>(s_err) != 0;
        wait_ok(done, 0);
        tc_fence_after();
        for (int bb = std::max(1, T - 2); bb < T; ++bb) {
            drain_t_issue(bb);
            drain_t_finish(bb);
        }
        if (DRAIN)
            for (; drained < C; ++drained) drain_d(drained);
        {
            float v[CPT];
            if (DRAIN) {
#pragma unroll
                for (int q = 0; q < CPT; ++q) v[q] = acc[q];
            } else {
                uint32_t h[CPT], l[CPT];
#pragma unroll
                for (int q = 0; q < CPT; ++q) l[q] = 0u;
                tmem_ld_issue<G4>(tmem + tlane + (uint32_t)c0, h);
                tmem_ld_wait<G4>(h, l);
#pragma unroll
                for (int q = 0; q < CPT; ++q) v[q] = __uint_as_float(h[q]);
            }
            const int64_t gi = (int64_t)I * BR + row;  // W row in tile order
            if (gi < p.n && !err_seen && !*reinterpret_cast<volatile int *>(s_err)) {
                float outv[CPT];
#pragma unroll
                for (int q = 0; q < CPT; ++q) outv[q] = c0 + q < p.c ? v[q] * cscale_of(q) : 0.f;
                add_row(gi, outv);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == SNEVAL) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.ncols_tmem)
                     : "memory");
    }
    if (threadIdx.x == 0 && *s_err) atomicOr(p.err, *s_err);
}

// 128-point tiles of the points in the order perm, coordinate-major, log2 e folded in,
// far padding
__global__ void sym_point_tiles_kernel(const float *Xs, const int *perm, int64_t n, int d, float factor,
                                       int64_t ntiles, float *Xp) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)BR * d;
    if (idx >= per * ntiles) return;
    const int64_t t = idx / per;
    const int rem = (int)(idx % per);
    const int a = rem / BR, jj = rem % BR;
    const int64_t i = t * BR + jj;
    const int64_t g = i < n ? (int64_t)perm[i] : -1;  // guarded: a position maps to a point < n
    Xp[idx] = (g >= 0 && g < n) ? Xs[g * d + a] * factor : PAD_COORD;
}

// Box of each tile's real points (kernel units): tbox[t] = d minima, then d maxima.
__global__ void sym_tile_box_kernel(const float *Xp, int64_t n, int d, int64_t ntiles, float *tbox) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= ntiles * d) return;
    const int64_t t = idx / d;
    const int a = (int)(idx % d);
    const int cnt = (int)min((int64_t)BR, n - t * BR);
    const float *x = Xp + t * BR * d + (int64_t)a * BR;
    float lo = x[0], hi = x[0];
    for (int jj = 1; jj < cnt; ++jj) {
        lo = fminf(lo, x[jj]);
        hi = fmaxf(hi, x[jj]);
    }
    tbox[t * 2 * d + a] = lo;
    tbox[t * 2 * d + d + a] = hi;
}

// V operand image per 128-point tile: SN columns x 128 K values, canonical K-major
// (byte offset (col/8)*2048 + (jj/8)*128 + (col%8)*16 + (jj%8)*2), hi then lo.
template <bool BF16, int NPROD>
__global__ void sym_image_kernel(const float *V, const int *perm, int64_t n, int c, int sn, int ntiles,
                                 const float *scale, uint8_t *img) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per_tile = (int64_t)sn * (BR / 8);
    if (idx >= per_tile * ntiles) return;
    const int64_t t = idx / per_tile;
    const int rem = (int)(idx % per_tile);
    const int cr = rem & 7;
    const int kq = (rem >> 3) % (BR / 8);
    const int g = rem / (8 * (BR / 8));
    const int col = g * 8 + cr;
    const float s = scale[col];
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t j = t * BR + kq * 8 + q;
        const int64_t g = j < n ? (int64_t)perm[j] : -1;
        v[q] = (g >= 0 && g < n && col < c) ? V[g * c + col] * s : 0.f;
    }
    uint4 hi;
    hi.x = pack2<BF16>(v[0], v[1]); hi.y = pack2<BF16>(v[2], v[3]);
    hi.z = pack2<BF16>(v[4], v[5]); hi.w = pack2<BF16>(v[6], v[7]);
    const size_t tile_bytes = (size_t)(NPROD == 3 ? 2 : 1) * sn * BR * 2;
    uint8_t *base = img + (size_t)t * tile_bytes;
    const size_t off = (size_t)g * CORE_SBO + (size_t)kq * 128 + (size_t)cr * 16;
    *reinterpret_cast<uint4 *>(base + off) = hi;
    if (NPROD == 3) {
        uint4 lo;
        uint32_t *hp = &hi.x, *lp = &lo.x;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const float2 f = unpack2<BF16>(hp[w]);
            lp[w] = pack2<BF16>(v[2 * w] - f.x, v[2 * w + 1] - f.y);
        }
        *reinterpret_cast<uint4 *>(base + (size_t)sn * BR * 2 + off) = lo;
    }
}

__global__ void sym_colmax_kernel(const float *V, int64_t n, int c, int sn, float *part) {
    const int col = threadIdx.x;
    const int nb = gridDim.x;
    const int64_t per = (n + nb - 1) / nb;
    const int64_t r0 = blockIdx.x * per, r1 = min(n, r0 + per);
    float m = 0.f;
    if (col < c)
        for (int64_t i = r0; i < r1; ++i) m = fmaxf(m, fabsf(V[i * c + col]));
    if (col < sn) part[(size_t)blockIdx.x * sn + col] = m;
}

__global__ void sym_colscale_kernel(const float *part, int nb, int sn, float *scale, float *colinv) {
    const int col = threadIdx.x;
    if (col >= sn) return;
    float m = 0.f;
    for (int b = 0; b < nb; ++b) m = fmaxf(m, part[(size_t)b * sn + col]);
    int e = 0;
    if (m > 0.f) frexpf(m, &e);
    // max |V_col| s in [KSCALE / 2, KSCALE): the lo part of the split stays out of
    // fp16 subnormals (as for the kernel values, tc_common.cuh)
    const float s = ldexpf(1.0f, KSCALE_LOG2 - e);
    scale[col] = s;
    colinv[col] = 1.0f / s;
}

// W[perm[r]] = Wt[r] + noise V[perm[r]]: the product back in the caller's point order,
// with the diagonal noise term (every row written once: perm is a permutation)
__global__ void sym_unpermute_kernel(const float *Wt, const int *perm, const float *V, int64_t n, int c, float noise,
                                     float *W) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * c) return;
    const int64_t r = idx / c;
    const int col = (int)(idx - r * c);
    const int64_t g = perm[r];
    if (g < 0 || g >= n) return;
    W[g * c + col] = Wt[idx] + noise * V[g * c + col];
}

template <int KIND, int DC, int NPROD, bool BF16, int SN>
int launch_sym(const SymParams &p, const SymLayout &L, cudaStream_t st) {
    auto fn = kz_sym_kernel<KIND, DC, NPROD, BF16, SN>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) {
        set_error("kz_sym: cannot reserve %d bytes of shared memory: %s", L.total, cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    // distinct kernel values evaluated: n (n + 1) / 2; tensor flops: D and D' per block
    const double nn = (double)p.n * (double)p.n;
    const int slot = prof_begin_launch(st, PROF_KZ_SYM, 0.5 * ((double)p.n * (double)(p.n + 1)), 2.0 * nn * SN * NPROD);
    fn<<<p.NB, SNTHREADS, L.total, st>>>(p, L);
    prof_end_launch(st, slot);
    return check_launch("kz_sym_kernel");
}

template <int KIND, int NPROD, bool BF16, int SN>
int launch_sym_d(const SymParams &p, const SymLayout &L, cudaStream_t st) {
    switch (p.d) {
        case 1: return launch_sym<KIND, 1, NPROD, BF16, SN>(p, L, st);
        case 2: return launch_sym<KIND, 2, NPROD, BF16, SN>(p, L, st);
        case 3: return launch_sym<KIND, 3, NPROD, BF16, SN>(p, L, st);
        case 4: return launch_sym<KIND, 4, NPROD, BF16, SN>(p, L, st);
        default: return launch_sym<KIND, 0, NPROD, BF16, SN>(p, L, st);
    }
}

template <int SN>
int launch_sym_all(int kind, int nprod, bool bf16, const SymParams &p, const SymLayout &L, cudaStream_t st) {
    if (kind == LD_RBF) {
        if (bf16) return launch_sym_d<LD_RBF, 1, true, SN>(p, L, st);
        if (nprod == 3) return launch_sym_d<LD_RBF, 3, false, SN>(p, L, st);
        return launch_sym_d<LD_RBF, 1, false, SN>(p, L, st);
    }
    if (bf16) return launch_sym_d<LD_MATERN52, 1, true, SN>(p, L, st);
    if (nprod == 3) return launch_sym_d<LD_MATERN52, 3, false, SN>(p, L, st);
    return launch_sym_d<LD_MATERN52, 1, false, SN>(p, L, st);
}

int sym_width(int c) { return c <= 16 ? 16 : SN_MAX; }

// Squared distance (kernel units) beyond which a unit-variance kernel value is <= 2^-10,
// so that one fp16 rounding (relative 2^-11) errs by at most 2^-21, as the hi/lo split of
// a value near 1 does.  Matern: coordinates carry sqrt(5)/l log2 e, k(u) = (1 + u + u^2/3)
// e^-u is decreasing; RBF: coordinates carry sqrt(log2 e)/(l sqrt 2), k = 2^-u2'.
float far_threshold2(int kind) {
    const double tau = 1.0 / 1024.0;
    if (kind == LD_RBF) return (float)std::log2(1.0 / tau);
    double lo = 0.0, hi = 100.0;
    for (int it = 0; it < 200; ++it) {
        const double u = 0.5 * (lo + hi);
        ((1.0 + u + u * u / 3.0) * std::exp(-u) > tau ? lo : hi) = u;
    }
    const double up = hi * 1.4426950408889634;  // in units carrying log2 e
    return (float)(up * up);
}

}  // namespace

bool kz_sym_eligible(int64_t n, int d, int c, int precision) {
    const int nprod = precision == LD_F16X3_TC ? 3 : 1;
    return c <= SN_MAX && n >= 2 * BR && d <= 8 && sym_stages(sym_width(c), d, nprod) > 0;
}

size_t kz_sym_workspace(int64_t n, int d, int c, int precision) {
    const int64_t NB = (n + BR - 1) / BR;
    const int nprod = precision == LD_F16X3_TC ? 3 : 1;
    const int sn = sym_width(c);
    Arena a;
    a.measuring = true;
    a.take<int>((size_t)n);                       // point order
    a.take<float>((size_t)n * c);                 // the product in tile order
    a.take<float>((size_t)NB * 2 * d);            // tile boxes
    a.take<float>((size_t)NB * BR * d);
    a.take<uint8_t>((size_t)NB * (nprod == 3 ? 2 : 1) * sn * BR * 2);
    a.take<float>(sn);
    a.take<float>(sn);
    a.take<float>((size_t)256 * sn);
    a.take<int>(4);
    a.take<char>(point_order_workspace(n, d));    // the sort's scratch (released after it)
    return a.off;
}

int kz_sym(const float *Xs, int64_t n, int d, int kind, double variance, double noise, const float *V, float *W,
           int c, int precision, Arena &ws, cudaStream_t st) {
    const int64_t NB = (n + BR - 1) / BR;
    const int nprod = precision == LD_F16X3_TC ? 3 : 1;
    const bool bf16 = precision == LD_BF16_TC;
    const int sn = sym_width(c);
    const size_t mark = ws.off;
    int *perm = ws.take<int>((size_t)n);
    float *Wt = ws.take<float>((size_t)n * c);
    float *tbox = ws.take<float>((size_t)NB * 2 * d);
    float *Xp = ws.take<float>((size_t)NB * BR * d);
    uint8_t *img = ws.take<uint8_t>((size_t)NB * (nprod == 3 ? 2 : 1) * sn * BR * 2);
    float *scale = ws.take<float>(sn);
    float *colinv = ws.take<float>(sn);
    float *part = ws.take<float>((size_t)256 * sn);
    int *err = ws.take<int>(4);
    if (ws.overflow || !Xp) {
        set_error("kz_sym: workspace too small");
        ws.off = mark;
        return LD_ERR_WORKSPACE;
    }
    int code = [&]() -> int {
        const float factor = kind == LD_RBF ? 1.2011224087864498f : 1.4426950408889634f;
        const int64_t cnt = NB * BR * d;
        LD_TRY(point_order(Xs, n, d, perm, ws, st));  // tiles of spatially close points
        sym_point_tiles_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(Xs, perm, n, d, factor, NB, Xp);
        sym_tile_box_kernel<<<(unsigned)((NB * d + 255) / 256), 256, 0, st>>>(Xp, n, d, NB, tbox);
        LD_TRY(check_launch("kz_sym tiles", 2));
        sym_colmax_kernel<<<256, 64, 0, st>>>(V, n, c, sn, part);
        sym_colscale_kernel<<<1, 64, 0, st>>>(part, 256, sn, scale, colinv);
        const int64_t nthr = NB * sn * (BR / 8);
        const unsigned gb = (unsigned)((nthr + 255) / 256);
        if (bf16) sym_image_kernel<true, 1><<<gb, 256, 0, st>>>(V, perm, n, c, sn, (int)NB, scale, img);
        else if (nprod == 3) sym_image_kernel<false, 3><<<gb, 256, 0, st>>>(V, perm, n, c, sn, (int)NB, scale, img);
        else sym_image_kernel<false, 1><<<gb, 256, 0, st>>>(V, perm, n, c, sn, (int)NB, scale, img);
        LD_TRY(check_launch("kz_sym prep", 3));
        LD_CHECK_CUDA(cudaMemsetAsync(Wt, 0, sizeof(float) * (size_t)n * c, st));
        LD_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        SymParams p;
        p.tbox = tbox;
        p.thr2 = far_threshold2(kind);
        p.far_on = nprod == 3 ? 1 : 0;
        p.Xp = Xp;
        p.img = img;
        p.colinv = colinv;
        p.W = Wt;
        p.n = n;
        p.d = d;
        p.c = c;
        p.NB = (int)NB;
        // D (x2 when drained, 2 SN wide with the hi/lo split) + two D'
        const int tcols = nprod == 3 ? 8 * sn : 3 * sn;
        p.ncols_tmem = tcols <= 32 ? 32 : (tcols <= 64 ? 64 : (tcols <= 128 ? 128 : (tcols <= 256 ? 256 : 512)));
        p.vec_ok = (reinterpret_cast<uintptr_t>(Wt) % 16 == 0) && ((c * 4) % 16 == 0);
        p.variance = (float)variance * KSCALE_INV;  // kernel values carry KSCALE
        p.err = err;
        const SymLayout L = make_sym_layout(sn, d, nprod, sym_stages(sn, d, nprod));
        if (sn == 16) LD_TRY(launch_sym_all<16>(kind, nprod, bf16, p, L, st));
        else LD_TRY(launch_sym_all<SN_MAX>(kind, nprod, bf16, p, L, st));
        const int64_t tot = n * c;
        sym_unpermute_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Wt, perm, V, n, c, (float)noise, W);
        LD_TRY(check_launch("kz_sym unpermute"));
        int herr = 0;
        LD_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        LD_CHECK_CUDA(cudaStreamSynchronize(st));
        if (herr) {
            set_error("kz_sym: a device-side wait timed out (error word %d)", herr);
            return LD_ERR_DEVICE_TIMEOUT;
        }
        return LD_OK;
    }();
    ws.off = mark;
    return code;
}

}  // namespace ld
