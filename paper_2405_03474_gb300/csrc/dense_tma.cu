// Stored dense product W = M V on the tensor cores with M fed by the tensor memory
// accelerator (the stored-M mode of the estimator: M = K + noise I kept row-major in
// fp32, every CG pass one product; Section 4 of the paper applies M only through such
// products).
//
// Per CTA: 128 rows of M, all of j in 64-column tiles.  A producer thread copies each
// 128 x 64 fp32 tile of M into shared memory with two 2-D tensor copies (32-float boxes,
// 128-byte swizzle) and the operand image of V beside it with a bulk copy; M never
// passes through the load/store unit on its way in.  Eight eval warps read the tile
// back (16-byte loads; the 8 lanes of each load phase are 8 rows whose swizzled 16-byte
// chunks differ, so no bank conflicts), scale it by the power of two that brings
// max |M_ii| into [KSCALE / 2, KSCALE), round it (fp16 / bf16) or split it hi/lo (fp16
// x3) exactly as the pipeline of kz_tc.cu does, and store the canonical K-major fp16
// tile.  One thread issues the tcgen05 MMAs; with the hi/lo split one N = 2c MMA
// multiplies K_hi by [V_hi | V_lo] and a second adds K_lo V_hi into the upper half.
// The fp16 x3 accumulator is drained every 8 tiles into fp32 partial sums held in the
// eval threads' registers.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace ld {

using namespace tc;

namespace {

constexpr int DM = 128;                 // rows per CTA (MMA M)
constexpr int DJ = 64;                  // j per tile (4 MMA K-steps of 16)
constexpr int DBOX = 32;                // floats per tensor-copy box row (128 bytes: one swizzle span)
constexpr int DEVAL = 8;                // eval warps
constexpr int DTHREADS = (DEVAL + 2) * 32;
constexpr int DA_HALF = DM * DJ * 2;    // one 128 x 64 fp16 tile (16 KB)
constexpr int DM_TILE = DM * DJ * 4;    // one 128 x 64 fp32 tile of M (32 KB)
constexpr int DKCH = 8;                 // tiles accumulated in TMEM before a drain (hi/lo)
constexpr int DN_MAX = 128;             // columns per launch

struct DenseParams {
    const uint8_t *img;   // operand image of V: per tile, nprod x (N x 64) halves, canonical K-major
    const float *colinv;  // 1 / column scale (N)
    const float *mscale;  // [0] power-of-two scale of M, [1] its inverse
    float *W;             // n x c, columns c0 .. c0 + N - 1 written (added to, when split)
    int64_t n;
    int c, c0, N, ntiles, ncols_tmem;
    int split;            // CTAs per 128-row block, each over a contiguous range of the j tiles
    int *err;
};

// M stages (released by the eval warps once read), V image stages (released by the
// MMAs), two fp16 operand tiles
struct DenseLayout {
    int sm, sv, b_bytes, vstage_bytes, a_bytes, m_off, v_off, a_off, total;
};

inline int round1k(int b) { return ((b + 1023) / 1024) * 1024; }

DenseLayout make_dense_layout(int N, int nprod, int sm) {
    DenseLayout L;
    L.sm = sm;
    L.sv = 2;
    L.b_bytes = (nprod == 3 ? 2 : 1) * N * DJ * 2;
    L.vstage_bytes = round1k(L.b_bytes);
    L.a_bytes = (nprod == 3 ? 2 : 1) * DA_HALF;
    L.m_off = 1024;  // 1024-aligned for the 128-byte swizzle
    L.v_off = L.m_off + sm * DM_TILE;
    L.a_off = L.v_off + L.sv * L.vstage_bytes;
    L.total = L.a_off + 2 * L.a_bytes + 1024;  // + alignment slack of the dynamic base
    return L;
}

int dense_stages(int N, int nprod) {
    for (int s = 6; s >= 2; --s)
        if (make_dense_layout(N, nprod, s).total <= 226 * 1024) return s;
    return 0;
}

// 2-D tensor copy of one box (DBOX x DM floats at column x, row y) into shared memory
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

template <int G>
__device__ __forceinline__ void tmem_ld_x4(uint32_t taddr, uint32_t (&r)[4 * G]) {
#pragma unroll
    for (int g = 0; g < G; ++g)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[4 * g]), "=r"(r[4 * g + 1]), "=r"(r[4 * g + 2]), "=r"(r[4 * g + 3])
                     : "r"(taddr + 4u * g));
}

// Completes the TMEM loads in flight; naming the destination registers keeps every use
// of them after the wait.
__device__ __forceinline__ void tmem_wait_regs(uint32_t (&a)[8], uint32_t (&b)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) asm volatile("" : "+r"(a[q]), "+r"(b[q]));
}

// NH: columns per eval thread in drains and the epilogue (a half of N, at most 64)
template <int NPROD, bool BF16, int NH>
__global__ void __launch_bounds__(DTHREADS, 1)
    dense_tma_kernel(const __grid_constant__ CUtensorMap mmap, DenseParams p, DenseLayout L) {
    constexpr bool DRAIN = NPROD == 3;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *mfull = reinterpret_cast<uint64_t *>(smem);  // [sm] M tile landed
    uint64_t *mempty = mfull + 8;                          // [sm] eval warps done reading it
    uint64_t *vfull = mempty + 8;                          // [2] V image landed
    uint64_t *vempty = vfull + 2;                          // [2] MMAs done with it
    uint64_t *afull = vempty + 2;                          // [2] fp16 tile written
    uint64_t *aempty = afull + 2;                         // [2] MMAs done with the fp16 tile
    uint64_t *done = aempty + 2;                          // every MMA done
    uint64_t *cfull = done + 1;                           // [2] chunk accumulated in TMEM
    uint64_t *cempty = cfull + 2;                         // [2] chunk drained
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(cempty + 2);
    int *s_err = reinterpret_cast<int *>(tmem_slot + 1);
    uint8_t *mbase = smem + L.m_off;
    uint8_t *vbase = smem + L.v_off;
    uint8_t *abase = smem + L.a_off;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // this CTA: rows row0 .. row0 + 127, tiles t0 .. t0 + T - 1 (local index tl = t - t0)
    const int row0 = (blockIdx.x / p.split) * DM;
    const int part = blockIdx.x % p.split;
    const int t0 = (int)((int64_t)p.ntiles * part / p.split);
    const int T = (int)((int64_t)p.ntiles * (part + 1) / p.split) - t0;
    const int SM_ = L.sm, SV = L.sv;
    const int N = p.N;
    // accumulator columns: [K_hi V_hi | K_hi V_lo + K_lo V_hi] with the split, else N
    const uint32_t NW = NPROD == 3 ? 2u * (uint32_t)N : (uint32_t)N;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SM_; ++s) {
            mbar_init(&mfull[s], 1);
            mbar_init(&mempty[s], DEVAL * 32);
        }
        for (int s = 0; s < SV; ++s) {
            mbar_init(&vfull[s], 1);
            mbar_init(&vempty[s], 1);
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
                     "r"(p.ncols_tmem)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == DEVAL + 1) {
        // ---------------- producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mmap)) : "memory");
            const uint32_t bb = (uint32_t)L.b_bytes;
            int tm = 0, tv = 0;  // M tiles and V images whose copies were issued
            for (int tl = 0; tl < T; ++tl) {
                const int t = t0 + tl;
                const int sm = tl % SM_, sv = tl % SV;
                if (tl >= SM_ && !mbar_wait(&mempty[sm], ((tl / SM_) - 1) & 1)) {
                    atomicOr(s_err, ERR_TIMEOUT);
                    break;
                }
                uint8_t *mst = mbase + (size_t)sm * DM_TILE;
                mbar_expect_tx(&mfull[sm], (uint32_t)DM_TILE);
                // x = 64 t (+ 32): 128-byte aligned column offsets; rows or columns past n read as 0
                tma_load_2d(mst, &mmap, t * DJ, row0, &mfull[sm]);
                tma_load_2d(mst + DM_TILE / 2, &mmap, t * DJ + DBOX, row0, &mfull[sm]);
                tm = tl + 1;
                if (tl >= SV && !mbar_wait(&vempty[sv], ((tl / SV) - 1) & 1)) {
                    atomicOr(s_err, ERR_TIMEOUT);
                    break;
                }
                mbar_expect_tx(&vfull[sv], bb);
                bulk_g2s(vbase + (size_t)sv * L.vstage_bytes, p.img + (size_t)t * bb, bb, &vfull[sv]);
                tv = tl + 1;
            }
            // every issued copy lands before the CTA may exit
            for (int u = std::max(0, tm - SM_); u < tm; ++u)
                if (!mbar_wait(&mfull[u % SM_], (u / SM_) & 1)) atomicOr(s_err, ERR_TIMEOUT);
            for (int u = std::max(0, tv - SV); u < tv; ++u)
                if (!mbar_wait(&vfull[u % SV], (u / SV) & 1)) atomicOr(s_err, ERR_TIMEOUT);
        }
    } else if (warp == DEVAL) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc_w = make_idesc(DM, (int)NW, BF16 ? 1u : 0u);  // B = [V_hi ; V_lo] (or V)
            const uint32_t idesc = make_idesc(DM, N, BF16 ? 1u : 0u);
            bool ok = true;
            for (int t = 0; t < T && ok; ++t) {
                const int sv = t % SV, sa = t & 1;
                const int k = t / DKCH;
                const bool first = DRAIN ? (t % DKCH == 0) : (t == 0);
                const uint32_t dt = tmem + (DRAIN ? (uint32_t)((k & 1) * NW) : 0u);
                if (DRAIN && first && k >= 2 && !mbar_wait(&cempty[k & 1], ((k - 2) >> 1) & 1)) {
                    ok = false;
                    break;
                }
                if (!mbar_wait(&afull[sa], (t >> 1) & 1) || !mbar_wait(&vfull[sv], (t / SV) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(abase + (size_t)sa * L.a_bytes);
                const uint32_t b0 = smem_u32(vbase + (size_t)sv * L.vstage_bytes);
                // A: K-major no swizzle (lbo = 128 along j, sbo = 1024 along rows); B likewise,
                // rows of B = columns of V, the lo half's rows following the hi half's
                const uint64_t dah = make_desc(a0, 128, 1024);
                const uint64_t dal = dah + (uint64_t)(DA_HALF >> 4);
                const uint64_t dbh = make_desc(b0, 128, 1024);
#pragma unroll
                for (int ks = 0; ks < DJ / 16; ++ks) {
                    const uint64_t step = (uint64_t)(ks * (256 >> 4));
                    mma_f16(dt, dah + step, dbh + step, idesc_w, (first && ks == 0) ? 0u : 1u);
                    if (NPROD == 3) mma_f16(dt + (uint32_t)N, dal + step, dbh + step, idesc, 1u);
                }
                mma_commit(&vempty[sv]);
                mma_commit(&aempty[sa]);
                if (DRAIN && (t % DKCH == DKCH - 1 || t == T - 1)) mma_commit(&cfull[k & 1]);
            }
            if (!ok) atomicOr(s_err, ERR_TIMEOUT);
            mma_commit(done);
            // every issued MMA has finished before tensor memory is released below
            if (!mbar_wait(done, 0)) atomicOr(s_err, ERR_TIMEOUT);
        }
    } else {
        // ---------------- eval warps
        // unit k (0..3) of a thread: row mr(k) = 16 warp + 8 (k >> 1) + lane % 8, the 8 columns
        // 8 mq(k) .. 8 mq(k) + 7 of the tile, mq(k) = 4 (k & 1) + lane / 8
        auto mr = [&](int k) { return 16 * warp + 8 * (k >> 1) + (lane & 7); };
        auto mq = [&](int k) { return 4 * (k & 1) + (lane >> 3); };
        const float ms = __ldg(p.mscale);
        const int quad = warp & 3;   // TMEM lane quadrant
        const int half = warp >> 2;  // column half in drains and the epilogue
        const int nh = N / 2;        // columns of that half (N is a multiple of 16)
        const uint32_t tlane = (uint32_t)(quad * 32) << 16;
        float acc[NH];
#pragma unroll
        for (int q = 0; q < NH; ++q) acc[q] = 0.f;
        bool err_seen = false;
        auto wait_ok = [&](uint64_t *bar, uint32_t parity) {
            if (err_seen) return;
            if (!mbar_wait(bar, parity)) {
                atomicOr(s_err, ERR_TIMEOUT);
                err_seen = true;
            }
        };
        // chunk k of the accumulator -> fp32 partial sums (the two halves summed)
        auto drain = [&](int k) {
            wait_ok(&cfull[k & 1], (k >> 1) & 1);
            tc_fence_after();
            const uint32_t ta = tmem + tlane + (uint32_t)((k & 1) * NW + half * nh);
#pragma unroll
            for (int c8 = 0; c8 < NH; c8 += 8) {
                if (c8 < nh) {
                    uint32_t h[8], l[8];
                    tmem_ld_x4<2>(ta + (uint32_t)c8, h);
                    tmem_ld_x4<2>(ta + (uint32_t)(N + c8), l);
                    tmem_wait_regs(h, l);
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[c8 + q] += __uint_as_float(h[q]) + __uint_as_float(l[q]);
                }
            }
            tc_fence_before();
            mbar_arrive(&cempty[k & 1]);
        };
        const int C = (T + DKCH - 1) / DKCH;
        int drained = 0;
        for (int t = 0; t < T; ++t) {
            const int sm = t % SM_, sa = t & 1;
            err_seen = err_seen || *reinterpret_cast<volatile int *>(s_err) != 0;
            if (DRAIN && t % DKCH == DKCH / 2 && t >= DKCH + DKCH / 2) drain(drained++);
            wait_ok(&mfull[sm], (t / SM_) & 1);
            if (t >= 2) wait_ok(&aempty[sa], ((t >> 1) - 1) & 1);
            const uint8_t *mt = mbase + (size_t)sm * DM_TILE;
            uint8_t *ast = abase + (size_t)sa * L.a_bytes;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r = mr(k), kq = mq(k);
                // columns 8 kq .. 8 kq + 7: box kq / 4, 16-byte chunks 2 (kq % 4) and + 1 of
                // row r, stored at chunk ^ (r % 8) by the 128-byte swizzle
                const uint8_t *rowp = mt + (size_t)(kq >> 2) * (DM_TILE / 2) + (size_t)r * 128;
                const int c0 = 2 * (kq & 3);
                const float4 v0 = *reinterpret_cast<const float4 *>(rowp + ((c0 ^ (r & 7)) << 4));
                const float4 v1 = *reinterpret_cast<const float4 *>(rowp + (((c0 + 1) ^ (r & 7)) << 4));
                const float2 f[4] = {make_float2(v0.x * ms, v0.y * ms), make_float2(v0.z * ms, v0.w * ms),
                                     make_float2(v1.x * ms, v1.y * ms), make_float2(v1.z * ms, v1.w * ms)};
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) w[q] = pack2<BF16>(f[q].x, f[q].y);
                const size_t off = (size_t)(r >> 3) * 1024 + (size_t)kq * 128 + (size_t)(r & 7) * 16;
                *reinterpret_cast<uint4 *>(ast + off) = make_uint4(w[0], w[1], w[2], w[3]);
                if (NPROD == 3) {
                    const float2 m1 = make_float2(-1.f, -1.f);
                    uint32_t l[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 rq = __ffma2_rn(unpack2<BF16>(w[q]), m1, f[q]);  // m - hi
                        l[q] = pack2<BF16>(rq.x, rq.y);
                    }
                    *reinterpret_cast<uint4 *>(ast + DA_HALF + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
            }
            mbar_arrive(&mempty[sm]);  // M stage read (values in registers, stored above)
            fence_async_smem();
            mbar_arrive(&afull[sa]);
        }
        // ---------------- epilogue
        err_seen = err_seen || *reinterpret_cast<volatile int *>(s_err) != 0;
        wait_ok(done, 0);
        tc_fence_after();
        if (DRAIN)
            for (; drained < C; ++drained) drain(drained);
        if (!DRAIN && !err_seen) {
            const uint32_t ta = tmem + tlane + (uint32_t)(half * nh);
#pragma unroll
            for (int c8 = 0; c8 < NH; c8 += 8) {
                if (c8 < nh) {
                    uint32_t h[8], unused[8] = {};
                    tmem_ld_x4<2>(ta + (uint32_t)c8, h);
                    tmem_wait_regs(h, unused);
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[c8 + q] = __uint_as_float(h[q]);
                }
            }
        }
        const int64_t i = (int64_t)row0 + quad * 32 + lane;
        if (i < p.n && !err_seen && !*reinterpret_cast<volatile int *>(s_err)) {
            const float post = __ldg(p.mscale + 1);  // undo the scale of M
#pragma unroll
            for (int q = 0; q < NH; ++q) {
                const int cc = half * nh + q;
                if (q < nh && p.c0 + cc < p.c) {
                    const float v = acc[q] * post * p.colinv[cc];
                    // split row blocks: two partial sums added into a zeroed W (two fp32 adds
                    // to 0 commute, so the result does not depend on their order)
                    if (p.split > 1) atomicAdd(&p.W[i * p.c + p.c0 + cc], v);
                    else p.W[i * p.c + p.c0 + cc] = v;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == DEVAL) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.ncols_tmem)
                     : "memory");
    }
    if (threadIdx.x == 0 && *s_err) atomicOr(p.err, *s_err);
}

template <int NPROD, bool BF16, int NH>
int launch_dense_tma(const CUtensorMap &map, const DenseParams &p, const DenseLayout &L, int nblocks,
                     cudaStream_t st) {
    auto fn = dense_tma_kernel<NPROD, BF16, NH>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) {
        set_error("dense_tma: cannot reserve %d bytes of shared memory: %s", L.total, cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    const double nn = (double)p.n * (double)p.n;
    const int slot = prof_begin_launch(st, PROF_DENSE, nn, 2.0 * nn * p.N * NPROD);
    fn<<<nblocks, DTHREADS, L.total, st>>>(map, p, L);
    prof_end_launch(st, slot);
    return check_launch("dense_tma_kernel");
}

template <int NPROD, bool BF16>
int launch_dense_tma_n(const CUtensorMap &map, const DenseParams &p, const DenseLayout &L, int nblocks,
                       cudaStream_t st) {
    if (p.N <= 32) return launch_dense_tma<NPROD, BF16, 16>(map, p, L, nblocks, st);
    if (p.N <= 64) return launch_dense_tma<NPROD, BF16, 32>(map, p, L, nblocks, st);
    return launch_dense_tma<NPROD, BF16, 64>(map, p, L, nblocks, st);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the library takes no
// link-time dependency on the driver; resolved once)
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

}  // namespace

bool dense_tma_eligible(const float *M, int64_t n, int N, int precision) {
    const int nprod = precision == LD_F16X3_TC ? 3 : 1;
    // row stride a multiple of 16 bytes (tensor map), 16-byte aligned base, at least one
    // full box of rows and columns, and 32-bit coordinates
    return n % 4 == 0 && reinterpret_cast<uintptr_t>(M) % 16 == 0 && n >= DM && n < ((int64_t)1 << 31) - DJ &&
           N <= DN_MAX && N % 16 == 0 && dense_stages(N, nprod) > 0;
}

int dense_tma(const float *M, int64_t n, const uint8_t *img, const float *colinv, const float *mscale, float *W,
              int c, int c0, int N, int precision, int *err, cudaStream_t st) {
    const int nprod = precision == LD_F16X3_TC ? 3 : 1;
    const bool bf16 = precision == LD_BF16_TC;
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};   // columns (contiguous), rows
    const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(float)};  // bytes between rows
    const cuuint32_t box[2] = {(cuuint32_t)DBOX, (cuuint32_t)DM};
    const cuuint32_t estr[2] = {1, 1};
    const PFN_cuTensorMapEncodeTiled_v12000 encode = encode_tiled();
    if (!encode) {
        set_error("dense_tma: cuTensorMapEncodeTiled not available from the driver");
        return LD_ERR_CUDA;
    }
    const CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(M), dims,
                                               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        set_error("dense_tma: tensor map of M rejected (CUresult %d)", (int)cr);
        return LD_ERR_CUDA;
    }
    DenseParams p;
    p.img = img;
    p.colinv = colinv;
    p.mscale = mscale;
    p.W = W;
    p.n = n;
    p.c = c;
    p.c0 = c0;
    p.N = N;
    p.ntiles = (int)((n + DJ - 1) / DJ);
    const int cols = nprod == 3 ? 4 * N : N;  // two ping-pong accumulators of 2 N with the split
    p.ncols_tmem = cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512)));
    p.err = err;
    const DenseLayout L = make_dense_layout(N, nprod, dense_stages(N, nprod));
    // One CTA per SM: split each row block's tiles over two CTAs when that fills the last
    // wave better (n = 65536: 512 row blocks are 3.4 waves on 152 SMs, 1024 halves 6.7)
    const int rblocks = (int)((n + DM - 1) / DM);
    int dev = 0, sms = 0;
    LD_CHECK_CUDA(cudaGetDevice(&dev));
    LD_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    auto fill = [&](int split) {
        const int64_t units = (int64_t)rblocks * split;
        const int64_t waves = (units + sms - 1) / sms;
        return (double)units / (double)(waves * sms);
    };
    p.split = (p.ntiles >= 2 * DKCH && fill(2) > fill(1) + 0.02) ? 2 : 1;
    if (p.split > 1) {
        const int cols_here = std::min(N, c - c0);
        LD_CHECK_CUDA(cudaMemset2DAsync(W + c0, (size_t)c * sizeof(float), 0, (size_t)cols_here * sizeof(float),
                                        (size_t)n, st));
    }
    const int nblocks = rblocks * p.split;
    if (bf16) return launch_dense_tma_n<1, true>(map, p, L, nblocks, st);
    if (nprod == 3) return launch_dense_tma_n<3, false>(map, p, L, nblocks, st);
    return launch_dense_tma_n<1, false>(map, p, L, nblocks, st);
}

}  // namespace ld
