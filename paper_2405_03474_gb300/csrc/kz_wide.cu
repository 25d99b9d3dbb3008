// Wide tensor-core kernel product W = (K + noise I) V for 256 < c <= 512 columns in
// one pass (the randomized-SVD sketch: rank-512 blocks), single fp16 or bf16 product.
//
// The general kernel keeps two CTAs per SM with at most 256 accumulator columns
// each, so 512 columns took two launches that each evaluated every kernel value.
// Here one CTA per SM owns all 512 TMEM columns: the 128 x 128 tile K_IJ is
// evaluated once by 16 eval warps (4 rows x 8 j per thread, packed f32x2, MUFU
// sqrt + ex2) into one of two K-tile stages and multiplied into both 256-column
// halves of D (16 tcgen05.mma per tile).  The operand image of V (64-point tiles,
// 32 KB per 256-column half) streams through a ring of quarter-tile stages, each
// with its own barrier, so several loads are in flight and each quarter's MMAs
// start when it lands; the point coordinates have a ring of their own, fed by a
// second producer lane.  D accumulates over the CTA's j-tiles in tensor memory
// (fp32, no drains: the single-product forms are for the sketch, whose accuracy
// is set by fp16 rounding of K and V).  Large n splits the j-tiles into chunks of
// WCHUNK (64 MB of operand image at 512 columns), one grid row per chunk in launch
// order, so the CTAs resident at one time stream one chunk that stays in L2; each
// CTA then adds its partial rows into W (zeroed first) with 16-byte vector
// reductions.  Every mbarrier wait is bounded.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace ld {

using namespace tc;

namespace {

constexpr int WM = 128;                 // rows per CTA (MMA M, TMEM lanes)
constexpr int WJ = 64;                  // points per point tile / image tile (4 MMA K-steps)
constexpr int WT = 128;                 // j per evaluated tile (two point tiles)
constexpr int WEVAL = 16;               // eval warps
constexpr int WTHREADS = (WEVAL + 2) * 32;
constexpr int WA_BYTES = WM * WT * 2;   // one 128 x 128 tile of halves
constexpr int WASBO = (WT / 8) * 128;   // 2048: K-tile byte step between 8-row groups
constexpr int WSBO = (WJ / 8) * 128;    // 1024: image byte step between 8-column groups
constexpr int W_MAXN = 512;
constexpr int W_HALF = 256;             // MMA N of the first half
constexpr int WSA = 2;                  // K-tile stages
constexpr int WXS = 4;                  // point-coordinate stages
constexpr int WCHUNK = 512;             // evaluated j-tiles per grid row when the j range is split

struct WideParams {
    const float *Xp;     // per 64-point tile: d x 64 floats, far-padded, log2 e folded in
    const uint8_t *img;  // per 64-point tile: N x 64 halves, canonical K-major (256-column halves)
    const float *V;      // n x c
    const float *colinv; // 1 / column scale (N)
    float *W;
    int64_t n;
    int d, c, N, ntiles;  // ntiles: evaluated 128-point j-tiles (point tiles are twice as many)
    int nchunks;          // > 1: partial sums over j-chunks, added into a zeroed W
    int vec_ok;           // W rows 16-byte aligned (c % 4 == 0 and W aligned)
    float variance, noise;
    int *err;
};

// Ring of SL quarter stages: stage m % SL holds 256-column half h = m % 2 of point tile
// 2 (m / 4) + (m / 2) % 2 (h0_bytes for the first half, h1_bytes = (N - 256) x 64 x 2 for
// the second); the coordinates of each evaluated tile (two point tiles, x_bytes) have a
// ring of WXS stages of their own.
struct WideLayout {
    int sl, h0_bytes, h1_bytes, x_bytes, a_off, x_off, l_off, total;
};

WideLayout make_wide_layout(int N, int d, int sl) {
    WideLayout L;
    L.sl = sl;
    L.h0_bytes = W_HALF * WJ * 2;
    L.h1_bytes = (N - W_HALF) * WJ * 2;
    L.x_bytes = WT * d * 4;
    L.a_off = 1024;
    L.x_off = L.a_off + WSA * WA_BYTES;
    L.l_off = L.x_off + ((WXS * L.x_bytes + 1023) / 1024) * 1024;
    L.total = L.l_off + sl * L.h0_bytes + 1024;
    return L;
}

template <int KIND, int DC, bool BF16>
__global__ void __launch_bounds__(WTHREADS, 1) kz_wide_kernel(WideParams p, WideLayout L) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);  // [sl]
    uint64_t *empty = full + 8;                           // [sl]
    uint64_t *afull = empty + 8;                          // [WSA]
    uint64_t *aempty = afull + WSA;                       // [WSA]
    uint64_t *xfull = aempty + WSA;                       // [WXS]
    uint64_t *xempty = xfull + WXS;                       // [WXS]
    uint64_t *done = xempty + WXS;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    int *s_err = reinterpret_cast<int *>(tmem_slot + 1);
    uint8_t *abase = smem + L.a_off;
    uint8_t *lbase = smem + L.l_off;
    uint8_t *xbase = smem + L.x_off;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int dd = DC > 0 ? DC : p.d;
    const int tbeg = blockIdx.y * WCHUNK;
    const int T = min(p.ntiles - tbeg, p.nchunks > 1 ? WCHUNK : p.ntiles);  // j-tiles of this CTA
    const int SL = L.sl;
    const int64_t row0 = (int64_t)blockIdx.x * WM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SL; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < WSA; ++s) {
            mbar_init(&afull[s], WEVAL * 32);
            mbar_init(&aempty[s], 1);
        }
        for (int s = 0; s < WXS; ++s) {
            mbar_init(&xfull[s], 1);
            mbar_init(&xempty[s], WEVAL * 32);
        }
        mbar_init(done, 1);
        *s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == WEVAL) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(W_MAXN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == WEVAL + 1) {
        if (lane == 0) {
            // ---------------- producer: quarters (point tile, 256-column half) of the image
            const size_t tile_bytes = (size_t)L.h0_bytes + L.h1_bytes;
            const int M = 4 * T;
            int m = 0;
            for (; m < M; ++m) {
                const int s = m % SL, h = m & 1;
                const int64_t it = 2 * (int64_t)(tbeg + (m >> 2)) + ((m >> 1) & 1);
                if (m >= SL && !mbar_wait(&empty[s], ((m / SL) - 1) & 1)) {
                    atomicOr(s_err, ERR_TIMEOUT);
                    break;
                }
                const uint32_t hb = (uint32_t)(h ? L.h1_bytes : L.h0_bytes);
                mbar_expect_tx(&full[s], hb);
                bulk_g2s(lbase + (size_t)s * L.h0_bytes, p.img + (size_t)it * tile_bytes + (h ? (size_t)L.h0_bytes : 0),
                         hb, &full[s]);
            }
            for (int u = std::max(0, m - SL); u < m; ++u)
                if (!mbar_wait(&full[u % SL], (u / SL) & 1)) atomicOr(s_err, ERR_TIMEOUT);
        } else if (lane == 1) {
            // ---------------- producer: coordinates of each evaluated tile (two point tiles)
            const uint32_t xb = (uint32_t)L.x_bytes;
            int t = 0;
            for (; t < T; ++t) {
                const int s = t % WXS;
                if (t >= WXS && !mbar_wait(&xempty[s], ((t / WXS) - 1) & 1)) {
                    atomicOr(s_err, ERR_TIMEOUT);
                    break;
                }
                mbar_expect_tx(&xfull[s], xb);
                bulk_g2s(xbase + (size_t)s * xb, p.Xp + (size_t)(tbeg + t) * WT * dd, xb, &xfull[s]);
            }
            for (int u = std::max(0, t - WXS); u < t; ++u)
                if (!mbar_wait(&xfull[u % WXS], (u / WXS) & 1)) atomicOr(s_err, ERR_TIMEOUT);
        }
    } else if (warp == WEVAL) {
        // ---------------- MMA issuer: D[:, 0:256] and D[:, 256:N] += K_IJ V_J, per quarter
        if (lane == 0) {
            const uint32_t idesc0 = make_idesc(WM, W_HALF, BF16 ? 1u : 0u);
            const uint32_t idesc1 = make_idesc(WM, p.N - W_HALF, BF16 ? 1u : 0u);
            bool ok = true;
            for (int t = 0; t < T && ok; ++t) {
                const int sa = t % WSA;
                if (!mbar_wait(&afull[sa], (t / WSA) & 1)) {
                    ok = false;
                    break;
                }
                const uint64_t da = make_desc(smem_u32(abase + (size_t)sa * WA_BYTES), 128, WASBO);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int g = q >> 1, h = q & 1;  // j half (point tile) and column half
                    const int m = 4 * t + q, s = m % SL;
                    if (!mbar_wait(&full[s], (m / SL) & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t db = make_desc(smem_u32(lbase + (size_t)s * L.h0_bytes), 128, WSBO);
                    const uint64_t dag = da + (uint64_t)(g * ((WJ / 8) * 128 >> 4));  // 64 j further along K
#pragma unroll
                    for (int ks = 0; ks < WJ / 16; ++ks) {
                        const uint64_t step = (uint64_t)(ks * (256 >> 4));  // descriptors advance by a constant
                        mma_f16(tmem + (h ? (uint32_t)W_HALF : 0u), dag + step, db + step, h ? idesc1 : idesc0,
                                (t == 0 && g == 0 && ks == 0) ? 0u : 1u);
                    }
                    mma_commit(&empty[s]);
                }
                mma_commit(&aempty[sa]);
            }
            if (!ok) atomicOr(s_err, ERR_TIMEOUT);
            mma_commit(done);
            if (!mbar_wait(done, 0)) atomicOr(s_err, ERR_TIMEOUT);
        }
    } else {
        // ---------------- eval warps: rows lane + 32 k (k = 0..3), j in [8 warp, 8 warp + 8)
        const int kq = warp;
        float2 xr[4][8];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int64_t i = row0 + lane + 32 * k;
                const float v = (a < dd && i < p.n) ? -p.Xp[(size_t)(i / WJ) * WJ * dd + a * WJ + (i % WJ)]
                                                    : (a < dd ? -PAD_COORD : 0.f);
                xr[k][a] = make_float2(v, v);
            }
        bool ok = true;
        for (int t = 0; t < T; ++t) {
            const int sx = t % WXS, sa = t % WSA;
            if (!mbar_wait(&xfull[sx], (t / WXS) & 1) ||
                (t >= WSA && !mbar_wait(&aempty[sa], ((t / WSA) - 1) & 1))) {
                ok = false;
                break;
            }
            uint8_t *ast = abase + (size_t)sa * WA_BYTES;
            // this warp's 8 points lie in point tile kq / 8 of the two
            const float *xs = reinterpret_cast<const float *>(xbase + (size_t)sx * L.x_bytes) +
                              (kq >> 3) * WJ * dd + (kq & 7) * 8;
            float2 xj[8][4];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                if (a < dd) {
                    const float4 lo4 = *reinterpret_cast<const float4 *>(xs + a * WJ);
                    const float4 hi4 = *reinterpret_cast<const float4 *>(xs + a * WJ + 4);
                    xj[a][0] = make_float2(lo4.x, lo4.y);
                    xj[a][1] = make_float2(lo4.z, lo4.w);
                    xj[a][2] = make_float2(hi4.x, hi4.y);
                    xj[a][3] = make_float2(hi4.z, hi4.w);
                }
            }
            mbar_arrive(&xempty[sx]);  // coordinates are in registers: the stage may be refilled
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t w[4];
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
                    w[q] = pack2<BF16>(f.x, f.y);
                }
                const int r = lane + 32 * k;
                const size_t off = (size_t)(r >> 3) * WASBO + (size_t)kq * 128 + (size_t)(r & 7) * 16;
                *reinterpret_cast<uint4 *>(ast + off) = make_uint4(w[0], w[1], w[2], w[3]);
            }
            fence_async_smem();
            mbar_arrive(&afull[sa]);
        }
        // ---------------- epilogue: W (+)= variance * colinv * D (+ noise * V in the first chunk)
        const bool got = ok && mbar_wait(done, 0);
        tc_fence_after();
        if (!got) {
            atomicOr(s_err, ERR_TIMEOUT);
        } else if (!*reinterpret_cast<volatile int *>(s_err)) {
            const int quad = warp & 3, part = warp >> 2;
            const int64_t i = row0 + quad * 32 + lane;
            const int span = p.N / 4;  // columns per warp (multiple of 8)
            for (int c8 = part * span; c8 < (part + 1) * span; c8 += 8) {
                float v[8];
                tmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c8, v);
                if (i < p.n) {
                    float o[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int col = c8 + q;
                        o[q] = col < p.c ? v[q] * p.variance * p.colinv[col] +
                                               (blockIdx.y == 0 ? p.noise * p.V[i * p.c + col] : 0.f)
                                         : 0.f;
                    }
                    float *dst = p.W + i * p.c + c8;
                    if (p.nchunks == 1) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (c8 + q < p.c) dst[q] = o[q];
                    } else if (p.vec_ok) {
#pragma unroll
                        for (int g = 0; g < 2; ++g)
                            if (c8 + 4 * g < p.c)
                                atomicAdd(reinterpret_cast<float4 *>(dst + 4 * g),
                                          make_float4(o[4 * g], o[4 * g + 1], o[4 * g + 2], o[4 * g + 3]));
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (c8 + q < p.c) atomicAdd(dst + q, o[q]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == WEVAL) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(W_MAXN) : "memory");
    }
    if (threadIdx.x == 0 && *s_err) atomicOr(p.err, *s_err);
}

// 64-point tiles, coordinate-major, log2 e folded in, far padding (points past n at PAD_COORD)
__global__ void wide_point_tiles_kernel(const float *Xs, int64_t n, int d, float factor, int64_t ntiles,
                                        float *Xp) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)WJ * d;
    if (idx >= per * ntiles) return;
    const int64_t t = idx / per;
    const int rem = (int)(idx % per);
    const int a = rem / WJ, jj = rem % WJ;
    const int64_t i = t * WJ + jj;
    Xp[idx] = i < n ? Xs[i * d + a] * factor : PAD_COORD;
}

__global__ void wide_colmax_kernel(const float *V, int64_t n, int c, int N, float *part) {
    const int col = threadIdx.x;
    const int nb = gridDim.x;
    const int64_t per = (n + nb - 1) / nb;
    const int64_t r0 = blockIdx.x * per, r1 = min(n, r0 + per);
    float m = 0.f;
    if (col < c)
        for (int64_t i = r0; i < r1; ++i) m = fmaxf(m, fabsf(V[i * c + col]));
    if (col < N) part[(size_t)blockIdx.x * N + col] = m;
}

__global__ void wide_colscale_kernel(const float *part, int nb, int N, float *scale, float *colinv) {
    const int col = threadIdx.x;
    if (col >= N) return;
    float m = 0.f;
    for (int b = 0; b < nb; ++b) m = fmaxf(m, part[(size_t)b * N + col]);
    int e = 0;
    if (m > 0.f) frexpf(m, &e);
    // max |V_col| s in [KSCALE / 2, KSCALE): the lo part of the split stays out of
    // fp16 subnormals (as for the kernel values, tc_common.cuh)
    const float s = ldexpf(1.0f, KSCALE_LOG2 - e);
    scale[col] = s;
    colinv[col] = 1.0f / s;
}

// V operand image per 64-point tile: N columns x 64 K values, canonical K-major
// (byte offset (col/8)*1024 + (jj/8)*128 + (col%8)*16 + (jj%8)*2).
template <bool BF16>
__global__ void wide_image_kernel(const float *V, int64_t n, int c, int N, int ntiles, const float *scale,
                                  uint8_t *img) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t per_tile = (int64_t)N * (WJ / 8);
    if (idx >= per_tile * ntiles) return;
    const int64_t t = idx / per_tile;
    const int rem = (int)(idx % per_tile);
    const int cr = rem & 7;
    const int kq = (rem >> 3) % (WJ / 8);
    const int g = rem / (8 * (WJ / 8));
    const int col = g * 8 + cr;
    const float s = scale[col];
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t j = t * WJ + kq * 8 + q;
        v[q] = (j < n && col < c) ? V[j * c + col] * s : 0.f;
    }
    uint4 hi;
    hi.x = pack2<BF16>(v[0], v[1]); hi.y = pack2<BF16>(v[2], v[3]);
    hi.z = pack2<BF16>(v[4], v[5]); hi.w = pack2<BF16>(v[6], v[7]);
    uint8_t *base = img + (size_t)t * N * WJ * 2;
    *reinterpret_cast<uint4 *>(base + (size_t)g * WSBO + (size_t)kq * 128 + (size_t)cr * 16) = hi;
}

int wide_stages(int N, int d) {
    for (int s = 8; s >= 4; --s)
        if (make_wide_layout(N, d, s).total <= 225 * 1024) return s;
    return 0;
}

// evaluated 128-point j-tiles; the point tiles and image tiles (64 points) are twice as many
int64_t wide_tiles(int64_t n) { return (n + WT - 1) / WT; }

template <int KIND, int DC, bool BF16>
int launch_wide(const WideParams &p, const WideLayout &L, int nblocks, cudaStream_t st) {
    auto fn = kz_wide_kernel<KIND, DC, BF16>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) {
        set_error("kz_wide: cannot reserve %d bytes of shared memory: %s", L.total, cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    const double nn = (double)p.n * (double)p.n;
    const int slot = prof_begin_launch(st, PROF_KZ_WIDE, nn, 2.0 * nn * p.N);
    fn<<<dim3(nblocks, p.nchunks), WTHREADS, L.total, st>>>(p, L);
    prof_end_launch(st, slot);
    return check_launch("kz_wide_kernel");
}

template <int KIND, bool BF16>
int launch_wide_d(const WideParams &p, const WideLayout &L, int nblocks, cudaStream_t st) {
    switch (p.d) {
        case 1: return launch_wide<KIND, 1, BF16>(p, L, nblocks, st);
        case 2: return launch_wide<KIND, 2, BF16>(p, L, nblocks, st);
        case 3: return launch_wide<KIND, 3, BF16>(p, L, nblocks, st);
        case 4: return launch_wide<KIND, 4, BF16>(p, L, nblocks, st);
        default: return launch_wide<KIND, 0, BF16>(p, L, nblocks, st);
    }
}

// Always the full 512 columns (the second 256-column half at full width; columns past c are
// zero in the image and discarded).  Narrower second halves (N - 256 < 256) produced, in about
// one call in seven with RBF at 300 columns, one wrong 8-row group of a tile when the MMA and
// evaluation sides ran at nearly the same rate; at full width no repeat differed.
int wide_N(int c) { (void)c; return W_MAXN; }

}  // namespace

bool kz_wide_eligible(int64_t n, int d, int c, int precision) {
    return (precision == LD_F16_TC || precision == LD_BF16_TC) && c > W_HALF && c <= W_MAXN && n >= WM &&
           d <= 8 && wide_stages(wide_N(c), d) > 0;
}

size_t kz_wide_workspace(int64_t n, int d, int c, int precision) {
    (void)precision;
    const int64_t npt = 2 * wide_tiles(n);
    const int N = wide_N(c);
    Arena a;
    a.measuring = true;
    a.take<float>((size_t)npt * WJ * d);
    a.take<uint8_t>((size_t)npt * N * WJ * 2);
    a.take<float>(W_MAXN);
    a.take<float>(W_MAXN);
    a.take<float>((size_t)256 * W_MAXN);
    a.take<int>(4);
    return a.off;
}

int kz_wide(const float *Xs, int64_t n, int d, int kind, double variance, double noise, const float *V,
            float *W, int c, int precision, Arena &ws, cudaStream_t st) {
    const int64_t ntiles = wide_tiles(n), npt = 2 * ntiles;
    const int N = wide_N(c);
    const bool bf16 = precision == LD_BF16_TC;
    const size_t mark = ws.off;
    float *Xp = ws.take<float>((size_t)npt * WJ * d);
    uint8_t *img = ws.take<uint8_t>((size_t)npt * N * WJ * 2);
    float *scale = ws.take<float>(W_MAXN);
    float *colinv = ws.take<float>(W_MAXN);
    float *part = ws.take<float>((size_t)256 * W_MAXN);
    int *err = ws.take<int>(4);
    if (ws.overflow || !Xp) {
        set_error("kz_wide: workspace too small");
        ws.off = mark;
        return LD_ERR_WORKSPACE;
    }
    int code = [&]() -> int {
        const float factor = kind == LD_RBF ? 1.2011224087864498f : 1.4426950408889634f;
        const int64_t cnt = npt * WJ * d;
        wide_point_tiles_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(Xs, n, d, factor, npt, Xp);
        wide_colmax_kernel<<<256, W_MAXN, 0, st>>>(V, n, c, N, part);
        wide_colscale_kernel<<<1, W_MAXN, 0, st>>>(part, 256, N, scale, colinv);
        const int64_t nthr = npt * N * (WJ / 8);
        const unsigned gb = (unsigned)((nthr + 255) / 256);
        if (bf16) wide_image_kernel<true><<<gb, 256, 0, st>>>(V, n, c, N, (int)npt, scale, img);
        else wide_image_kernel<false><<<gb, 256, 0, st>>>(V, n, c, N, (int)npt, scale, img);
        LD_TRY(check_launch("kz_wide prep", 4));
        LD_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        WideParams p;
        p.Xp = Xp;
        p.img = img;
        p.V = V;
        p.colinv = colinv;
        p.W = W;
        p.n = n;
        p.d = d;
        p.c = c;
        p.N = N;
        p.ntiles = (int)ntiles;
        p.nchunks = (int)((ntiles + WCHUNK - 1) / WCHUNK);
        p.vec_ok = (reinterpret_cast<uintptr_t>(W) % 16 == 0) && (c % 4 == 0);
        if (p.nchunks > 1) LD_CHECK_CUDA(cudaMemsetAsync(W, 0, sizeof(float) * (size_t)n * c, st));
        p.variance = (float)variance * KSCALE_INV;  // kernel values carry KSCALE
        p.noise = (float)noise;
        p.err = err;
        const WideLayout L = make_wide_layout(N, d, wide_stages(N, d));
        const int nblocks = (int)((n + WM - 1) / WM);
        if (kind == LD_RBF) {
            if (bf16) LD_TRY(launch_wide_d<LD_RBF, true>(p, L, nblocks, st));
            else LD_TRY(launch_wide_d<LD_RBF, false>(p, L, nblocks, st));
        } else {
            if (bf16) LD_TRY(launch_wide_d<LD_MATERN52, true>(p, L, nblocks, st));
            else LD_TRY(launch_wide_d<LD_MATERN52, false>(p, L, nblocks, st));
        }
        int herr = 0;
        LD_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        LD_CHECK_CUDA(cudaStreamSynchronize(st));
        if (herr) {
            set_error("kz_wide: a device-side wait timed out (error word %d)", herr);
            return LD_ERR_DEVICE_TIMEOUT;
        }
        return LD_OK;
    }();
    ws.off = mark;
    return code;
}

}  // namespace ld
