// Tall-skinny dense kernels of the preconditioner and CG: row-major GEMMs
// (C = A B and C = A^T B with a deterministic fp64 split reduction), column
// dot products with fp64 accumulation, and small elementwise helpers.  These
// are HBM-bound next to the kernel product and sized for n up to 2^22 rows
// and at most a few hundred columns.
#include <algorithm>

#include "common.cuh"

namespace ld {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// C(m x q) = alpha A(m x k) B(k x q) + beta C; 64x64 tile, 4x4 per thread.
template <typename T>
__global__ void __launch_bounds__(NT) gemm_nn_kernel(int64_t m, int q, int k, T alpha,
                                                     const T *__restrict__ A, int64_t lda,
                                                     const T *__restrict__ B, int64_t ldb, T beta,
                                                     T *__restrict__ C, int64_t ldc) {
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int col0 = blockIdx.y * BN;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
        for (int l = 0; l < (BM * BK) / NT; ++l) {
            int e = tid + l * NT;
            int mm = e / BK, kk = e % BK;
            int64_t gr = row0 + mm;
            int gk = k0 + kk;
            As[kk][mm] = (gr < m && gk < k) ? A[gr * lda + gk] : T(0);
        }
#pragma unroll
        for (int l = 0; l < (BK * BN) / NT; ++l) {
            int e = tid + l * NT;
            int kk = e / BN, nn = e % BN;
            int gk = k0 + kk, gc = col0 + nn;
            Bs[kk][nn] = (gk < k && gc < q) ? B[(int64_t)gk * ldb + gc] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int64_t gr = row0 + ty * 4 + a;
        if (gr >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int gc = col0 + tx * 4 + b;
            if (gc >= q) continue;
            T v = alpha * acc[a][b];
            if (beta != T(0)) v += beta * C[gr * ldc + gc];
            C[gr * ldc + gc] = v;
        }
    }
}

// Skinny forms for q <= 64 (the preconditioner applies of the CG, 16 or 48 columns):
// 256 x 16 tiles (4 x 4 per thread, 64 row groups x 4 column groups), one column tile
// of 16 per grid row, so no thread computes padding columns.
constexpr int SBM = 256, SBN = 16;

// C(m x q) = alpha A(m x k) B(k x q) + beta C, skinny tile.
template <typename T>
__global__ void __launch_bounds__(NT) gemm_nn_skinny_kernel(int64_t m, int q, int k, T alpha,
                                                            const T *__restrict__ A, int64_t lda,
                                                            const T *__restrict__ B, int64_t ldb, T beta,
                                                            T *__restrict__ C, int64_t ldc) {
    __shared__ T As[BK][SBM + 1];
    __shared__ T Bs[BK][SBN];
    const int tid = threadIdx.x;
    const int tx = tid % 4, ty = tid / 4;
    const int64_t row0 = (int64_t)blockIdx.x * SBM;
    const int col0 = blockIdx.y * SBN;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
        for (int l = 0; l < (SBM * BK) / NT; ++l) {
            const int e = tid + l * NT;
            const int mm = e / BK, kk = e % BK;
            const int64_t gr = row0 + mm;
            const int gk = k0 + kk;
            As[kk][mm] = (gr < m && gk < k) ? A[gr * lda + gk] : T(0);
        }
        {
            const int kk = tid / SBN, nn = tid % SBN;
            const int gk = k0 + kk, gc = col0 + nn;
            Bs[kk][nn] = (gk < k && gc < q) ? B[(int64_t)gk * ldb + gc] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t gr = row0 + ty * 4 + a;
        if (gr >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int gc = col0 + tx * 4 + b;
            if (gc >= q) continue;
            T v = alpha * acc[a][b];
            if (beta != T(0)) v += beta * C[gr * ldc + gc];
            C[gr * ldc + gc] = v;
        }
    }
}

// partial[split](p x q) = A[rows of split]^T B[rows of split], skinny tile (p in 256s, q in 16s).
template <typename T>
__global__ void __launch_bounds__(NT) gemm_tn_skinny_kernel(int64_t m, int p, int q, int64_t rows_per,
                                                            const T *__restrict__ A, int64_t lda,
                                                            const T *__restrict__ B, int64_t ldb,
                                                            double *__restrict__ part) {
    __shared__ T As[BK][SBM];
    __shared__ T Bs[BK][SBN];
    const int tid = threadIdx.x;
    const int tx = tid % 4, ty = tid / 4;
    const int p0 = blockIdx.x * SBM, q0 = blockIdx.y * SBN;
    const int64_t r0 = (int64_t)blockIdx.z * rows_per;
    const int64_t r1 = min(m, r0 + rows_per);
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int64_t k0 = r0; k0 < r1; k0 += BK) {
#pragma unroll
        for (int l = 0; l < (SBM * BK) / NT; ++l) {
            const int e = tid + l * NT;
            const int kk = e / SBM, pp = e % SBM;
            const int64_t gr = k0 + kk;
            As[kk][pp] = (gr < r1 && p0 + pp < p) ? A[gr * lda + p0 + pp] : T(0);
        }
        {
            const int kk = tid / SBN, nn = tid % SBN;
            const int64_t gr = k0 + kk;
            Bs[kk][nn] = (gr < r1 && q0 + nn < q) ? B[gr * ldb + q0 + nn] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        __syncthreads();
    }
    double *out = part + (size_t)blockIdx.z * p * q;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int gp = p0 + ty * 4 + a;
        if (gp >= p) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int gq = q0 + tx * 4 + b;
            if (gq < q) out[(size_t)gp * q + gq] = (double)acc[a][b];
        }
    }
}

// partial[split](p x q) = A[rows of split]^T B[rows of split]
template <typename T>
__global__ void __launch_bounds__(NT) gemm_tn_kernel(int64_t m, int p, int q, int64_t rows_per,
                                                     const T *__restrict__ A, int64_t lda,
                                                     const T *__restrict__ B, int64_t ldb,
                                                     double *__restrict__ part) {
    __shared__ T As[BK][BM];
    __shared__ T Bs[BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int p0 = blockIdx.x * BM, q0 = blockIdx.y * BN;
    const int64_t r0 = (int64_t)blockIdx.z * rows_per;
    const int64_t r1 = min(m, r0 + rows_per);
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int64_t k0 = r0; k0 < r1; k0 += BK) {
#pragma unroll
        for (int l = 0; l < (BM * BK) / NT; ++l) {
            int e = tid + l * NT;
            int kk = e / BM, pp = e % BM;
            int64_t gr = k0 + kk;
            As[kk][pp] = (gr < r1 && p0 + pp < p) ? A[gr * lda + p0 + pp] : T(0);
        }
#pragma unroll
        for (int l = 0; l < (BN * BK) / NT; ++l) {
            int e = tid + l * NT;
            int kk = e / BN, nn = e % BN;
            int64_t gr = k0 + kk;
            Bs[kk][nn] = (gr < r1 && q0 + nn < q) ? B[gr * ldb + q0 + nn] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        __syncthreads();
    }
    double *out = part + (size_t)blockIdx.z * p * q;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int gp = p0 + ty * 4 + a;
        if (gp >= p) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int gq = q0 + tx * 4 + b;
            if (gq < q) out[(size_t)gp * q + gq] = (double)acc[a][b];
        }
    }
}

__global__ void reduce_splits_kernel(const double *__restrict__ part, int nsplit, int64_t count,
                                     double *__restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += part[(size_t)k * count + t];
    out[t] = s;
}

int tn_splits(int64_t m, int p, int q) {
    int tiles = ((p + BM - 1) / BM) * ((q + BN - 1) / BN);
    int64_t want = std::max<int64_t>(1, 2048 / tiles);
    int64_t maxs = std::max<int64_t>(1, (m + 255) / 256);
    return (int)std::min<int64_t>(std::min<int64_t>(want, maxs), 4096);
}

// column dots, c <= 256 packed: thread t owns column t % c
template <typename T>
__global__ void coldot_small_kernel(int64_t n, int c, int64_t rows_per, const T *__restrict__ A,
                                    const T *__restrict__ B, double *__restrict__ part) {
    __shared__ double sm[256];
    const int per = 256 / c;  // row lanes
    const int t = threadIdx.x;
    const int lane_row = t / c, col = t % c;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(n, r0 + rows_per);
    double s = 0.0;
    if (lane_row < per) {
        for (int64_t i = r0 + lane_row; i < r1; i += per) {
            size_t idx = (size_t)i * c + col;
            s += (double)A[idx] * (double)B[idx];
        }
    }
    sm[t] = s;
    __syncthreads();
    if (t < c) {
        double acc = 0.0;
        for (int k = 0; k < per; ++k) acc += sm[k * c + t];
        part[(size_t)blockIdx.x * c + t] = acc;
    }
}

// column dots, c > 256: thread owns one column of the block's column group
template <typename T>
__global__ void coldot_wide_kernel(int64_t n, int c, int64_t rows_per, const T *__restrict__ A,
                                   const T *__restrict__ B, double *__restrict__ part) {
    const int col = blockIdx.y * 256 + threadIdx.x;
    if (col >= c) return;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(n, r0 + rows_per);
    double s = 0.0;
    for (int64_t i = r0; i < r1; ++i) {
        size_t idx = (size_t)i * c + col;
        s += (double)A[idx] * (double)B[idx];
    }
    part[(size_t)blockIdx.x * c + col] = s;
}

int coldot_blocks(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(1216, (n + 511) / 512));
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin *in, Tout *out, int64_t count) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < count) out[t] = (Tout)in[t];
}

template <typename T>
__global__ void scale_rows_kernel(const T *in, const T *rs, T *out, int64_t n, int c) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n * c) out[t] = in[t] * rs[t / c];
}

template <typename T>
__global__ void axpy_kernel(int64_t count, T alpha, const T *x, T *y) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < count) y[t] += alpha * x[t];
}

// SplitMix64 (Steele, Lea & Flood 2014): the k-th output of the stream seeded
// with `seed` is mix64(seed + (k + 1) * 0x9E3779B97F4A7C15).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// N(0,1) by Box-Muller from SplitMix64 outputs 2k, 2k+1 (uniforms (m + 1/2) 2^-53)
template <typename T>
__global__ void gaussian_kernel(uint64_t seed, int64_t n, int s, int col0, T *Z) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * s) return;
    int64_t i = t / s;
    int j = (int)(t % s);
    uint64_t k = (uint64_t)(col0 + j) * (uint64_t)n + (uint64_t)i;
    const double u1 = ((double)(splitmix64_at(seed, 2 * k) >> 11) + 0.5) * 1.1102230246251565e-16;
    const double u2 = ((double)(splitmix64_at(seed, 2 * k + 1) >> 11) + 0.5) * 1.1102230246251565e-16;
    Z[t] = (T)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
}

__global__ void rademacher_kernel(uint64_t seed, int64_t n, int s, int col0, int8_t *Z) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * s) return;
    int64_t i = t / s;
    int j = (int)(t % s);
    uint64_t k = (uint64_t)(col0 + j) * (uint64_t)n + (uint64_t)i;
    Z[t] = (splitmix64_at(seed, k) >> 63) ? (int8_t)-1 : (int8_t)1;
}

inline unsigned blocks_for(int64_t count, int per = 256) {
    return (unsigned)((count + per - 1) / per);
}

}  // namespace

template <typename T>
int gemm_nn(int64_t m, int q, int k, T alpha, const T *A, int64_t lda, const T *B, int64_t ldb,
            T beta, T *C, int64_t ldc, cudaStream_t st) {
    if (m == 0 || q == 0) return LD_OK;
    if (q <= 64) {
        dim3 grid((unsigned)((m + SBM - 1) / SBM), (unsigned)((q + SBN - 1) / SBN));
        gemm_nn_skinny_kernel<T><<<grid, NT, 0, st>>>(m, q, k, alpha, A, lda, B, ldb, beta, C, ldc);
        return check_launch("gemm_nn");
    }
    dim3 grid((unsigned)((m + BM - 1) / BM), (unsigned)((q + BN - 1) / BN));
    gemm_nn_kernel<T><<<grid, NT, 0, st>>>(m, q, k, alpha, A, lda, B, ldb, beta, C, ldc);
    return check_launch("gemm_nn");
}

size_t gemm_tn_partials(int64_t m, int p, int q) {
    return (size_t)tn_splits(m, p, q) * p * q;
}

template <typename T>
int gemm_tn(int64_t m, int p, int q, const T *A, int64_t lda, const T *B, int64_t ldb, double *Cd,
            double *part, cudaStream_t st) {
    if (p == 0 || q == 0) return LD_OK;
    int ns = tn_splits(m, p, q);
    int64_t rows_per = (m + ns - 1) / ns;
    rows_per = ((rows_per + BK - 1) / BK) * BK;
    if (rows_per == 0) rows_per = BK;
    if (q <= 64) {
        dim3 grid((unsigned)((p + SBM - 1) / SBM), (unsigned)((q + SBN - 1) / SBN), (unsigned)ns);
        gemm_tn_skinny_kernel<T><<<grid, NT, 0, st>>>(m, p, q, rows_per, A, lda, B, ldb, part);
    } else {
        dim3 grid((unsigned)((p + BM - 1) / BM), (unsigned)((q + BN - 1) / BN), (unsigned)ns);
        gemm_tn_kernel<T><<<grid, NT, 0, st>>>(m, p, q, rows_per, A, lda, B, ldb, part);
    }
    LD_TRY(check_launch("gemm_tn"));
    int64_t count = (int64_t)p * q;
    reduce_splits_kernel<<<blocks_for(count), 256, 0, st>>>(part, ns, count, Cd);
    return check_launch("reduce_splits");
}

size_t coldot_partials(int64_t n, int c) { return (size_t)coldot_blocks(n) * c; }

template <typename T>
int coldot(int64_t n, int c, const T *A, const T *B, double *out, double *part, cudaStream_t st) {
    if (c == 0) return LD_OK;
    int nb = coldot_blocks(n);
    int64_t rows_per = (n + nb - 1) / nb;
    if (c <= 256) {
        coldot_small_kernel<T><<<nb, 256, 0, st>>>(n, c, rows_per, A, B, part);
    } else {
        dim3 grid(nb, (c + 255) / 256);
        coldot_wide_kernel<T><<<grid, 256, 0, st>>>(n, c, rows_per, A, B, part);
    }
    LD_TRY(check_launch("coldot"));
    reduce_splits_kernel<<<blocks_for(c), 256, 0, st>>>(part, nb, c, out);
    return check_launch("coldot_reduce");
}

template <typename Tin, typename Tout>
int convert(const Tin *in, Tout *out, int64_t count, cudaStream_t st) {
    if (count == 0) return LD_OK;
    convert_kernel<Tin, Tout><<<blocks_for(count), 256, 0, st>>>(in, out, count);
    return check_launch("convert");
}

template <typename T>
int int8_to(const int8_t *in, T *out, int64_t count, cudaStream_t st) {
    return convert<int8_t, T>(in, out, count, st);
}

template <typename T>
int scale_rows(const T *in, const T *rs, T *out, int64_t n, int c, cudaStream_t st) {
    if (n * c == 0) return LD_OK;
    scale_rows_kernel<T><<<blocks_for(n * c), 256, 0, st>>>(in, rs, out, n, c);
    return check_launch("scale_rows");
}

template <typename T>
int axpy(int64_t count, T alpha, const T *x, T *y, cudaStream_t st) {
    if (count == 0) return LD_OK;
    axpy_kernel<T><<<blocks_for(count), 256, 0, st>>>(count, alpha, x, y);
    return check_launch("axpy");
}

template <typename T>
int gaussian(uint64_t seed, int64_t n, int s, int col0, T *Z, cudaStream_t st) {
    if (n * s == 0) return LD_OK;
    gaussian_kernel<T><<<blocks_for(n * s), 256, 0, st>>>(seed, n, s, col0, Z);
    return check_launch("gaussian");
}
template int gaussian<float>(uint64_t, int64_t, int, int, float *, cudaStream_t);
template int gaussian<double>(uint64_t, int64_t, int, int, double *, cudaStream_t);

int rademacher(uint64_t seed, int64_t n, int s, int col0, int8_t *Z, cudaStream_t st) {
    if (n * s == 0) return LD_OK;
    rademacher_kernel<<<blocks_for(n * s), 256, 0, st>>>(seed, n, s, col0, Z);
    return check_launch("rademacher");
}

#define INST(T)                                                                                  \
    template int gemm_nn<T>(int64_t, int, int, T, const T *, int64_t, const T *, int64_t, T, T *, \
                            int64_t, cudaStream_t);                                              \
    template int gemm_tn<T>(int64_t, int, int, const T *, int64_t, const T *, int64_t, double *,  \
                            double *, cudaStream_t);                                             \
    template int coldot<T>(int64_t, int, const T *, const T *, double *, double *, cudaStream_t); \
    template int int8_to<T>(const int8_t *, T *, int64_t, cudaStream_t);                         \
    template int scale_rows<T>(const T *, const T *, T *, int64_t, int, cudaStream_t);           \
    template int axpy<T>(int64_t, T, const T *, T *, cudaStream_t);
INST(float)
INST(double)
#undef INST
template int convert<double, float>(const double *, float *, int64_t, cudaStream_t);
template int convert<float, double>(const float *, double *, int64_t, cudaStream_t);
template int convert<double, double>(const double *, double *, int64_t, cudaStream_t);
template int convert<float, float>(const float *, float *, int64_t, cudaStream_t);

}  // namespace ld

extern "C" int ld_rademacher(uint64_t seed, int64_t n, int32_t s, int32_t col0, int8_t *Z_dev,
                             void *stream) {
    ld::clear_error();
    if (n < 0 || s < 0 || col0 < 0 || (n * s > 0 && !Z_dev)) {
        ld::set_error("ld_rademacher: bad arguments");
        return LD_ERR_INVALID;
    }
    return ld::rademacher(seed, n, s, col0, Z_dev, (cudaStream_t)stream);
}

extern "C" int ld_gaussian(uint64_t seed, int64_t n, int32_t s, int32_t col0, double *Z_dev, void *stream) {
    ld::clear_error();
    if (n < 0 || s < 0 || col0 < 0 || (n * s > 0 && !Z_dev)) {
        ld::set_error("ld_gaussian: bad arguments");
        return LD_ERR_INVALID;
    }
    return ld::gaussian<double>(seed, n, s, col0, Z_dev, (cudaStream_t)stream);
}
