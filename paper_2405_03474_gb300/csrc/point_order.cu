// A spatially coherent order of the points for the tiled kernel products: Morton
// (bit-interleaved) codes of the coordinates quantised over their bounding box, sorted
// by a stable least-significant-digit radix sort (four passes of 8 bits).  Consecutive
// runs of 128 points then occupy compact regions, so a 128 x 128 block of kernel
// values between two distant tiles is uniformly small (the symmetric product rounds
// such blocks once instead of splitting them hi/lo).  Equal codes keep their input
// order, so the permutation is deterministic.
#include <stdint.h>

#include <algorithm>

#include "common.cuh"

namespace ld {

namespace {

constexpr int PO_BLOCKS = 256;   // blocks of the histogram / scatter passes (one chunk each)
constexpr int PO_THREADS = 256;  // threads per block (8 warps)

// per-block partial min / max of every coordinate
__global__ void bbox_partial_kernel(const float *Xs, int64_t n, int d, float *part) {
    __shared__ float mn[PO_THREADS], mx[PO_THREADS];
    for (int a = 0; a < d; ++a) {
        float lo = 3.0e38f, hi = -3.0e38f;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const float v = Xs[i * d + a];
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
        mn[threadIdx.x] = lo;
        mx[threadIdx.x] = hi;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) {
                mn[threadIdx.x] = fminf(mn[threadIdx.x], mn[threadIdx.x + h]);
                mx[threadIdx.x] = fmaxf(mx[threadIdx.x], mx[threadIdx.x + h]);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            part[(size_t)blockIdx.x * 2 * d + a] = mn[0];
            part[(size_t)blockIdx.x * 2 * d + d + a] = mx[0];
        }
        __syncthreads();
    }
}

// Morton code: coordinate a quantised to b bits over [lo_a, hi_a], bit k of it at
// position k d + a (d b <= 32).  The bounding box is the reduction of the partials.
__global__ void morton_kernel(const float *Xs, int64_t n, int d, int b, const float *part, int nparts,
                              uint32_t *key, uint32_t *idx) {
    __shared__ float lo[8], scale[8];
    if (threadIdx.x < d) {
        float l = 3.0e38f, h = -3.0e38f;
        for (int p = 0; p < nparts; ++p) {
            l = fminf(l, part[(size_t)p * 2 * d + threadIdx.x]);
            h = fmaxf(h, part[(size_t)p * 2 * d + d + threadIdx.x]);
        }
        lo[threadIdx.x] = l;
        scale[threadIdx.x] = h > l ? (float)(1u << b) / (h - l) : 0.f;
    }
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t top = (1u << b) - 1u;
    uint32_t code = 0;
    for (int a = 0; a < d; ++a) {
        const float t = (Xs[i * d + a] - lo[a]) * scale[a];
        const uint32_t q = t <= 0.f ? 0u : (t >= (float)top ? top : (uint32_t)t);
        for (int k = 0; k < b; ++k) code |= ((q >> k) & 1u) << (k * d + a);
    }
    key[i] = code;
    idx[i] = (uint32_t)i;
}

// digit counts of each block's contiguous chunk: cnt[digit * PO_BLOCKS + block]
__global__ void radix_hist_kernel(const uint32_t *key, int64_t n, int64_t chunk, int shift, uint32_t *cnt) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
    __syncthreads();
    cnt[(size_t)threadIdx.x * PO_BLOCKS + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of the 256 x PO_BLOCKS counts in digit-major order (one block)
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t *cnt) {
    constexpr int TOTAL = 256 * PO_BLOCKS;
    constexpr int PER = TOTAL / 1024;
    __shared__ uint32_t part[1024];
    uint32_t sum = 0;
    for (int k = 0; k < PER; ++k) sum += cnt[threadIdx.x * PER + k];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive Hillis-Steele scan of the per-thread sums
        const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - sum;
    for (int k = 0; k < PER; ++k) {
        const uint32_t c = cnt[threadIdx.x * PER + k];
        cnt[threadIdx.x * PER + k] = run;
        run += c;
    }
}

// Stable scatter: each block walks its chunk in rounds of PO_THREADS elements; an
// element's destination is its digit's base (earlier blocks, earlier rounds) plus the
// number of equal digits before it in the round (earlier warps, then earlier lanes).
__global__ void radix_scatter_kernel(const uint32_t *key, const uint32_t *idx, int64_t n, int64_t chunk, int shift,
                                     const uint32_t *off, uint32_t *key_out, uint32_t *idx_out) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[PO_THREADS / 32][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    base[threadIdx.x] = off[(size_t)threadIdx.x * PO_BLOCKS + blockIdx.x];
    const int64_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    const uint32_t lt = (1u << lane) - 1u;
    for (int64_t r0 = b0; r0 < b1; r0 += PO_THREADS) {
        for (int w = 0; w < PO_THREADS / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = r0 + threadIdx.x;
        const bool valid = i < b1;
        const uint32_t k = valid ? key[i] : 0u;
        const uint32_t v = valid ? idx[i] : 0u;
        const uint32_t dg = valid ? ((k >> shift) & 255u) : 256u;  // 256: no digit
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][dg] = __popc(peers);
        __syncthreads();
        {   // per digit: exclusive prefix over the warps, then advance the digit's base
            uint32_t run = base[threadIdx.x];
            for (int w = 0; w < PO_THREADS / 32; ++w) {
                const uint32_t c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = run;
                run += c;
            }
            base[threadIdx.x] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t dst = wcnt[warp][dg] + rank;  // < n: the counts are those of the same chunks
            if ((int64_t)dst < n) {
                key_out[dst] = k;
                idx_out[dst] = v;
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t point_order_workspace(int64_t n, int d) {
    Arena a;
    a.measuring = true;
    a.take<float>((size_t)PO_BLOCKS * 2 * d);
    a.take<uint32_t>((size_t)n);  // keys (ping)
    a.take<uint32_t>((size_t)n);  // keys (pong)
    a.take<uint32_t>((size_t)n);  // indices (pong; ping is the output)
    a.take<uint32_t>((size_t)256 * PO_BLOCKS);
    return a.off;
}

int point_order(const float *Xs, int64_t n, int d, int *perm, Arena &ws, cudaStream_t st) {
    if (d < 1 || d > 8 || n < 1 || n > ((int64_t)1 << 31) - 1) {
        set_error("point_order: need 1 <= d <= 8 and 1 <= n < 2^31");
        return LD_ERR_INVALID;
    }
    const size_t mark = ws.off;
    float *part = ws.take<float>((size_t)PO_BLOCKS * 2 * d);
    uint32_t *k0 = ws.take<uint32_t>((size_t)n);
    uint32_t *k1 = ws.take<uint32_t>((size_t)n);
    uint32_t *i1 = ws.take<uint32_t>((size_t)n);
    uint32_t *cnt = ws.take<uint32_t>((size_t)256 * PO_BLOCKS);
    if (ws.overflow || !part) {
        set_error("point_order: workspace too small");
        ws.off = mark;
        return LD_ERR_WORKSPACE;
    }
    uint32_t *i0 = reinterpret_cast<uint32_t *>(perm);
    const int bits = std::min(32 / d, 16);
    const int64_t chunk = (n + PO_BLOCKS - 1) / PO_BLOCKS;
    bbox_partial_kernel<<<PO_BLOCKS, PO_THREADS, 0, st>>>(Xs, n, d, part);
    morton_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Xs, n, d, bits, part, PO_BLOCKS, k0, i0);
    int code = check_launch("point_order codes", 2);
    // four stable passes of 8 bits; an even number, so the result lands back in (k0, i0)
    for (int pass = 0; pass < 4 && code == LD_OK; ++pass) {
        const int shift = 8 * pass;
        const uint32_t *ki = (pass & 1) ? k1 : k0;
        const uint32_t *ii = (pass & 1) ? i1 : i0;
        uint32_t *ko = (pass & 1) ? k0 : k1;
        uint32_t *io = (pass & 1) ? i0 : i1;
        radix_hist_kernel<<<PO_BLOCKS, 256, 0, st>>>(ki, n, chunk, shift, cnt);
        radix_scan_kernel<<<1, 1024, 0, st>>>(cnt);
        radix_scatter_kernel<<<PO_BLOCKS, PO_THREADS, 0, st>>>(ki, ii, n, chunk, shift, cnt, ko, io);
        code = check_launch("point_order radix pass", 3);
    }
    ws.off = mark;
    return code;
}

}  // namespace ld
