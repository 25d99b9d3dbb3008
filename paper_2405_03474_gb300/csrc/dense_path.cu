// Stored dense M = K + noise I and its product W = M V: the variant of the
// O(n^2) step (Algorithm 1 step 2) that keeps M in HBM and reads it once per
// product, against evaluating K again in every pass (kz_simt.cu, kz_tc.cu).
// FP64 and FP32 products run on the CUDA cores (gemm_nn); the tensor-core
// precisions stream M through the tcgen05 pipeline of kz_tc.cu (dense_tc).
#include "common.cuh"
#include "kernel_fn.cuh"

namespace ld {

using namespace kfn;

namespace {

constexpr int TI = 32, TJD = 32, RPT = 4;  // 32 x 32 tile, 4 rows per thread (blockDim 32 x 8)

template <typename T, int KIND, int DC>
__global__ void materialize_kernel(const T *__restrict__ Xs, int64_t n, int d, int64_t ntj, T var, T noise,
                                   T *__restrict__ M) {
    constexpr int DMAX = DC > 0 ? DC : 32;
    const int dd = DC > 0 ? DC : d;
    const int64_t tile = blockIdx.x;
    const int64_t i0 = (tile / ntj) * TI, j0 = (tile % ntj) * TJD;
    const int64_t j = j0 + threadIdx.x;
    T xj[DMAX];
#pragma unroll
    for (int a = 0; a < DMAX; ++a) xj[a] = (a < dd && j < n) ? Xs[j * dd + a] : T(0);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int64_t i = i0 + threadIdx.y + 8 * r;
        if (i >= n || j >= n) continue;
        T u2 = T(0);
#pragma unroll
        for (int a = 0; a < DMAX; ++a) {
            if (a < dd) {
                const T df = Xs[i * dd + a] - xj[a];
                u2 += df * df;
            }
        }
        T k = kval<T, KIND>(u2, var);
        if (i == j) k += noise;
        M[i * n + j] = k;
    }
}

template <typename T, int KIND>
int launch_mat(const T *Xs, int64_t n, int d, T var, T noise, T *M, cudaStream_t st) {
    const int64_t nti = (n + TI - 1) / TI, ntj = (n + TJD - 1) / TJD;
    const dim3 block(32, 8);
    const unsigned grid = (unsigned)(nti * ntj);
    switch (d) {
        case 1: materialize_kernel<T, KIND, 1><<<grid, block, 0, st>>>(Xs, n, d, ntj, var, noise, M); break;
        case 2: materialize_kernel<T, KIND, 2><<<grid, block, 0, st>>>(Xs, n, d, ntj, var, noise, M); break;
        case 3: materialize_kernel<T, KIND, 3><<<grid, block, 0, st>>>(Xs, n, d, ntj, var, noise, M); break;
        case 4: materialize_kernel<T, KIND, 4><<<grid, block, 0, st>>>(Xs, n, d, ntj, var, noise, M); break;
        default: materialize_kernel<T, KIND, 0><<<grid, block, 0, st>>>(Xs, n, d, ntj, var, noise, M); break;
    }
    return check_launch("materialize");
}

}  // namespace

template <typename T>
int dense_materialize(const T *Xs, int64_t n, int d, const ld_kernel &k, T *M, cudaStream_t st) {
    if (k.kind == LD_RBF) return launch_mat<T, LD_RBF>(Xs, n, d, (T)k.variance, (T)k.noise, M, st);
    return launch_mat<T, LD_MATERN52>(Xs, n, d, (T)k.variance, (T)k.noise, M, st);
}

template <typename T>
int dense_product(const T *M, int64_t n, const T *V, T *W, int c, cudaStream_t st) {
    const double nn = (double)n * (double)n;
    const int slot = prof_begin_launch(st, PROF_DENSE, nn, 2.0 * nn * c);
    int code = gemm_nn<T>(n, c, (int)n, T(1), M, n, V, c, T(0), W, c, st);
    prof_end_launch(st, slot);
    return code;
}

template int dense_materialize<float>(const float *, int64_t, int, const ld_kernel &, float *, cudaStream_t);
template int dense_materialize<double>(const double *, int64_t, int, const ld_kernel &, double *, cudaStream_t);
template int dense_product<float>(const float *, int64_t, const float *, float *, int, cudaStream_t);
template int dense_product<double>(const double *, int64_t, const double *, double *, int, cudaStream_t);

}  // namespace ld

using namespace ld;

extern "C" {

size_t ld_dense_bytes(int64_t n, int32_t precision) {
    return (size_t)n * (size_t)n * (precision == LD_FP64 ? sizeof(double) : sizeof(float));
}

int ld_dense_materialize(const double *X_dev, int64_t n, int32_t d, ld_kernel kern, int32_t precision,
                         void *M_dev, void *stream) {
    clear_error();
    LD_REQUIRE(X_dev && M_dev && n > 0 && n <= (int64_t)1 << 31, "ld_dense_materialize: bad arguments");
    LD_REQUIRE(d >= 1 && d <= 32, "ld_dense_materialize: d must be in [1, 32]");
    LD_REQUIRE(kern.lengthscale > 0 && kern.variance > 0 && kern.noise >= 0 &&
                   (kern.kind == LD_RBF || kern.kind == LD_MATERN52),
               "ld_dense_materialize: bad kernel parameters");
    cudaStream_t st = (cudaStream_t)stream;
    Arena a;
    const size_t elt = precision == LD_FP64 ? sizeof(double) : sizeof(float);
    LD_TRY(arena_open(a, nullptr, 0, (size_t)n * d * elt + 256));
    int code;
    if (precision == LD_FP64) {
        double *Xs = a.take<double>((size_t)n * d);
        code = prep_points<double>(X_dev, n, d, point_scale(kern), Xs, st);
        if (code == LD_OK) code = dense_materialize<double>(Xs, n, d, kern, (double *)M_dev, st);
    } else {
        float *Xs = a.take<float>((size_t)n * d);
        code = prep_points<float>(X_dev, n, d, point_scale(kern), Xs, st);
        if (code == LD_OK) code = dense_materialize<float>(Xs, n, d, kern, (float *)M_dev, st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (code == LD_OK && e != cudaSuccess) {
        set_error("ld_dense_materialize: %s", cudaGetErrorString(e));
        code = LD_ERR_CUDA;
    }
    arena_close(a);
    return code;
}

int ld_dense_kz(const void *M_dev, int64_t n, const void *V_dev, void *W_dev, int32_t c, int32_t precision,
                void *stream) {
    clear_error();
    LD_REQUIRE(M_dev && V_dev && W_dev && n > 0 && c > 0 && V_dev != W_dev, "ld_dense_kz: bad arguments");
    LD_REQUIRE(n <= (int64_t)1 << 31, "ld_dense_kz: n too large");
    LD_REQUIRE(precision >= LD_FP64 && precision <= LD_F16X3_TC, "ld_dense_kz: bad precision");
    LD_REQUIRE(!is_tc_precision(precision) || c <= 4096, "ld_dense_kz: at most 4096 columns");
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == LD_FP64)
        return dense_product<double>((const double *)M_dev, n, (const double *)V_dev, (double *)W_dev, c, st);
    if (!is_tc_precision(precision))
        return dense_product<float>((const float *)M_dev, n, (const float *)V_dev, (float *)W_dev, c, st);
    // tensor cores: scratch for the operand image of V, allocated here and freed after the
    // product (the call synchronises the stream)
    Arena a;
    LD_TRY(arena_open(a, nullptr, 0, dense_tc_workspace(n, c, precision)));
    int code = dense_tc((const float *)M_dev, n, (const float *)V_dev, (float *)W_dev, c, precision, a, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (code == LD_OK && e != cudaSuccess) {
        set_error("ld_dense_kz: %s", cudaGetErrorString(e));
        code = LD_ERR_CUDA;
    }
    arena_close(a);
    return code;
}

}  // extern "C"
