// Small dense fp64 linear algebra on r x r matrices (r <= 1024): Cholesky,
// lower-triangular inverse, small GEMMs and reductions.  These are the rank-r
// cores of the preconditioner (CholeskyQR Gram factors, the C = Q^T M Q core
// and the I + R_G R_G^T core whose Cholesky gives log det P).  GB300's fp64 rate
// is low, so the work is kept at O(r^3) on at most a few MB resident in L2.
#include <math.h>

#include "common.cuh"

namespace ld {

namespace {

constexpr int CHOL_THREADS = 1024;

// Right-looking Cholesky, one CTA of 32 x 32 threads.  A is r x r row-major; the
// lower triangle is read and overwritten by L, the strict upper triangle is
// zeroed.  Column k of L (below the diagonal) is kept in shared memory for the
// rank-1 update of the trailing lower triangle, whose rows go to the 32 thread
// rows and whose columns to the 32 lanes (coalesced, no index division).
__global__ void __launch_bounds__(CHOL_THREADS) chol_kernel(double *A, int r, double shift,
                                                            int *status) {
    extern __shared__ double s_col[];  // r: column k of L
    __shared__ double s_piv;
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    const int tx = tid & 31, ty = tid >> 5;
    if (tid == 0) s_bad = 0;
    for (int i = tid; i < r; i += CHOL_THREADS) A[(size_t)i * r + i] += shift;
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (tid == 0) {
            const double akk = A[(size_t)k * r + k];
            if (!(akk > 0.0)) {
                s_bad = k + 1;
                s_piv = 1.0;
            } else {
                s_piv = sqrt(akk);
                A[(size_t)k * r + k] = s_piv;
            }
        }
        __syncthreads();
        if (s_bad) break;
        const double piv = s_piv;
        for (int i = k + 1 + tid; i < r; i += CHOL_THREADS) {
            const double v = A[(size_t)i * r + k] / piv;
            A[(size_t)i * r + k] = v;
            s_col[i] = v;
        }
        __syncthreads();
        for (int i = k + 1 + ty; i < r; i += 32) {
            const double li = s_col[i];
            double *row = A + (size_t)i * r;
            for (int j = k + 1 + tx; j <= i; j += 32) row[j] -= li * s_col[j];
        }
        __syncthreads();
    }
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)r * r; e += CHOL_THREADS) {
        const int i = (int)(e / r), j = (int)(e % r);
        if (j > i) A[e] = 0.0;
    }
    if (tid == 0) *status = s_bad;
}

// Column j of L^-1 by forward substitution, one CTA per column.
__global__ void trinv_kernel(const double *L, double *Li, int r) {
    extern __shared__ double x[];  // r
    __shared__ double red[32];
    const int j = blockIdx.x;
    const int tid = threadIdx.x;
    for (int i = tid; i < r; i += blockDim.x) x[i] = 0.0;
    __syncthreads();
    for (int i = j; i < r; ++i) {
        // s = sum_{k=j}^{i-1} L[i,k] x[k]
        double s = 0.0;
        for (int k = j + tid; k < i; k += blockDim.x) s += L[(size_t)i * r + k] * x[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((tid & 31) == 0) red[tid >> 5] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            x[i] = ((i == j ? 1.0 : 0.0) - t) / L[(size_t)i * r + i];
        }
        __syncthreads();
    }
    for (int i = tid; i < r; i += blockDim.x) Li[(size_t)i * r + j] = x[i];
}

__global__ void dense_gemm_kernel(int m, int q, int k, double alpha, const double *A, int lda,
                                  bool ta, const double *B, int ldb, bool tb, double beta,
                                  double *C, int ldc) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * q) return;
    int i = (int)(t / q), j = (int)(t % q);
    double s = 0.0;
    for (int l = 0; l < k; ++l) {
        double a = ta ? A[(size_t)l * lda + i] : A[(size_t)i * lda + l];
        double b = tb ? B[(size_t)j * ldb + l] : B[(size_t)l * ldb + j];
        s += a * b;
    }
    double v = alpha * s;
    if (beta != 0.0) v += beta * C[(size_t)i * ldc + j];
    C[(size_t)i * ldc + j] = v;
}

__global__ void sumlogdiag_kernel(const double *L, int r, double *out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < r; i += blockDim.x) s += log(L[(size_t)i * r + i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

__global__ void trace_kernel(const double *A, int r, double *out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < r; i += blockDim.x) s += A[(size_t)i * r + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

__global__ void symmetrize_kernel(double *A, int r) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)r * r) return;
    int i = (int)(t / r), j = (int)(t % r);
    if (j <= i) return;
    double v = 0.5 * (A[(size_t)i * r + j] + A[(size_t)j * r + i]);
    A[(size_t)i * r + j] = v;
    A[(size_t)j * r + i] = v;
}

template <typename T>
__global__ void export_kernel(const double *src, T *dst, int r, double add, bool tr) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)r * r) return;
    int i = (int)(t / r), j = (int)(t % r);
    double v = tr ? src[(size_t)j * r + i] : src[(size_t)i * r + j];
    if (i == j) v += add;
    dst[t] = (T)v;
}

}  // namespace

int dense_chol(double *A, int r, double shift, int *status, cudaStream_t st) {
    if (r == 0) return LD_OK;
    chol_kernel<<<1, CHOL_THREADS, r * sizeof(double), st>>>(A, r, shift, status);
    return check_launch("dense_chol");
}

int dense_trinv_lower(const double *L, double *Linv, int r, cudaStream_t st) {
    if (r == 0) return LD_OK;
    trinv_kernel<<<r, 128, r * sizeof(double), st>>>(L, Linv, r);
    return check_launch("dense_trinv_lower");
}

int dense_gemm(int m, int q, int k, double alpha, const double *A, int lda, bool ta, const double *B,
               int ldb, bool tb, double beta, double *C, int ldc, cudaStream_t st) {
    int64_t cnt = (int64_t)m * q;
    if (cnt == 0) return LD_OK;
    dense_gemm_kernel<<<(unsigned)((cnt + 127) / 128), 128, 0, st>>>(m, q, k, alpha, A, lda, ta, B,
                                                                     ldb, tb, beta, C, ldc);
    return check_launch("dense_gemm");
}

int dense_sumlogdiag(const double *L, int r, double *out, cudaStream_t st) {
    sumlogdiag_kernel<<<1, 256, 0, st>>>(L, r, out);
    return check_launch("dense_sumlogdiag");
}

int dense_trace(const double *A, int r, double *out, cudaStream_t st) {
    trace_kernel<<<1, 256, 0, st>>>(A, r, out);
    return check_launch("dense_trace");
}

int dense_symmetrize(double *A, int r, cudaStream_t st) {
    int64_t cnt = (int64_t)r * r;
    if (cnt == 0) return LD_OK;
    symmetrize_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(A, r);
    return check_launch("dense_symmetrize");
}

template <typename T>
int dense_export(const double *src, T *dst, int r, double add_identity, bool transpose,
                 cudaStream_t st) {
    int64_t cnt = (int64_t)r * r;
    if (cnt == 0) return LD_OK;
    export_kernel<T><<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(src, dst, r, add_identity,
                                                                   transpose);
    return check_launch("dense_export");
}
template int dense_export<float>(const double *, float *, int, double, bool, cudaStream_t);
template int dense_export<double>(const double *, double *, int, double, bool, cudaStream_t);

}  // namespace ld
