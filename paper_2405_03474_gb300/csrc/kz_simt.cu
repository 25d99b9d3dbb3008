// Matrix-free kernel product W = (K(X, X) + noise I) V on the CUDA cores
// (FP64 and FP32 modes), and the fused K V / (dK/dl) V pass of the gradient.
//
// This is the O(n^2) work of Algorithm 1 step 2 (Section 2, complexity
// paragraph): every output row i sums k(x_i, x_j) V[j, :] over all n points j,
// without storing K.  One thread owns one row i and a chunk of CC columns;
// point and V tiles of TJ rows are staged in shared memory and read as
// broadcasts.
#include "common.cuh"
#include "kernel_fn.cuh"

namespace ld {

using namespace kfn;

namespace {

constexpr int TPB = 128;  // rows per block (one per thread)
constexpr int TJ = 64;    // j-tile staged in shared memory
constexpr int CC = 16;    // columns per thread

template <typename T>
__global__ void prep_points_kernel(const double *X, int64_t count, double scale, T *Xs) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < count) Xs[t] = (T)(X[t] * scale);
}

__global__ void finite_check_kernel(const double *X, int64_t count, int *flag) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < count && !isfinite(X[t])) atomicOr(flag, 1);
}

template <typename T, int KIND, int DC, bool DERIV>
__global__ void __launch_bounds__(TPB) kz_simt_kernel(const T *__restrict__ Xs, int64_t n, int d,
                                                      const T *__restrict__ V, T *__restrict__ W,
                                                      T *__restrict__ Wdl, int c, T var, T noise,
                                                      T inv_l) {
    constexpr int DMAX = DC > 0 ? DC : 32;
    __shared__ T sx[TJ * DMAX];
    __shared__ T sv[TJ * CC];
    const int dd = DC > 0 ? DC : d;
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const int c0 = blockIdx.y * CC;
    const int cw = min(CC, c - c0);
    T xi[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) xi[t] = (t < dd && i < n) ? Xs[i * dd + t] : T(0);
    T acc[CC], acc2[DERIV ? CC : 1];
#pragma unroll
    for (int q = 0; q < CC; ++q) acc[q] = T(0);
#pragma unroll
    for (int q = 0; q < (DERIV ? CC : 1); ++q) acc2[q] = T(0);

    for (int64_t j0 = 0; j0 < n; j0 += TJ) {
        __syncthreads();
        for (int t = threadIdx.x; t < TJ * dd; t += TPB) {
            int64_t jj = j0 + t / dd;
            sx[t] = jj < n ? Xs[j0 * dd + t] : T(0);
        }
        for (int t = threadIdx.x; t < TJ * CC; t += TPB) {
            int jj = t / CC, q = t % CC;
            sv[t] = (j0 + jj < n && q < cw) ? V[(j0 + jj) * c + c0 + q] : T(0);
        }
        __syncthreads();
        const int jn = (int)min((int64_t)TJ, n - j0);
        for (int jj = 0; jj < jn; ++jj) {
            T u2 = T(0);
#pragma unroll
            for (int t = 0; t < DMAX; ++t) {
                if (t < dd) {
                    T df = xi[t] - sx[jj * dd + t];
                    u2 += df * df;
                }
            }
            if (DERIV) {
                T k, dk;
                kval_dl<T, KIND>(u2, var, inv_l, k, dk);
#pragma unroll
                for (int q = 0; q < CC; ++q) {
                    acc[q] += k * sv[jj * CC + q];
                    acc2[q] += dk * sv[jj * CC + q];
                }
            } else {
                T k = kval<T, KIND>(u2, var);
#pragma unroll
                for (int q = 0; q < CC; ++q) acc[q] += k * sv[jj * CC + q];
            }
        }
    }
    if (i < n) {
        for (int q = 0; q < cw; ++q) {
            if (DERIV) {
                W[i * c + c0 + q] = acc[q];
                Wdl[i * c + c0 + q] = acc2[q];
            } else {
                W[i * c + c0 + q] = acc[q] + noise * V[i * c + c0 + q];
            }
        }
    }
}

template <typename T, int KIND, bool DERIV>
int launch_kz(const T *Xs, int64_t n, int d, const T *V, T *W, T *Wdl, int c, T var, T noise,
              T inv_l, cudaStream_t st) {
    dim3 grid((unsigned)((n + TPB - 1) / TPB), (unsigned)((c + CC - 1) / CC));
    const double nn = (double)n * (double)n;
    const int slot = prof_begin_launch(st, PROF_KZ_SIMT, nn, 2.0 * nn * c * (DERIV ? 2 : 1));
    switch (d) {
        case 1: kz_simt_kernel<T, KIND, 1, DERIV><<<grid, TPB, 0, st>>>(Xs, n, d, V, W, Wdl, c, var, noise, inv_l); break;
        case 2: kz_simt_kernel<T, KIND, 2, DERIV><<<grid, TPB, 0, st>>>(Xs, n, d, V, W, Wdl, c, var, noise, inv_l); break;
        case 3: kz_simt_kernel<T, KIND, 3, DERIV><<<grid, TPB, 0, st>>>(Xs, n, d, V, W, Wdl, c, var, noise, inv_l); break;
        case 4: kz_simt_kernel<T, KIND, 4, DERIV><<<grid, TPB, 0, st>>>(Xs, n, d, V, W, Wdl, c, var, noise, inv_l); break;
        default: kz_simt_kernel<T, KIND, 0, DERIV><<<grid, TPB, 0, st>>>(Xs, n, d, V, W, Wdl, c, var, noise, inv_l); break;
    }
    prof_end_launch(st, slot);
    return check_launch("kz_simt_kernel");
}

}  // namespace

int check_points_finite(const double *X, int64_t n, int d, int *flag_dev, cudaStream_t st) {
    const int64_t count = n * d;
    LD_CHECK_CUDA(cudaMemsetAsync(flag_dev, 0, sizeof(int), st));
    finite_check_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(X, count, flag_dev);
    LD_TRY(check_launch("finite_check"));
    int h = 0;
    LD_CHECK_CUDA(cudaMemcpyAsync(&h, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    LD_CHECK_CUDA(cudaStreamSynchronize(st));
    if (h) {
        set_error("non-finite point coordinate (NaN or Inf) in X");
        return LD_ERR_INVALID;
    }
    return LD_OK;
}

template <typename T>
int prep_points(const double *X, int64_t n, int d, double scale, T *Xs, cudaStream_t st) {
    int64_t count = n * d;
    if (count == 0) return LD_OK;
    prep_points_kernel<T><<<(unsigned)((count + 255) / 256), 256, 0, st>>>(X, count, scale, Xs);
    return check_launch("prep_points");
}

template <typename T>
int kz_simt(const T *Xs, int64_t n, int d, int kind, double variance, double noise, const T *V,
            T *W, int c, cudaStream_t st) {
    if (n == 0 || c == 0) return LD_OK;
    if (kind == LD_RBF)
        return launch_kz<T, LD_RBF, false>(Xs, n, d, V, W, nullptr, c, (T)variance, (T)noise, T(0), st);
    return launch_kz<T, LD_MATERN52, false>(Xs, n, d, V, W, nullptr, c, (T)variance, (T)noise, T(0), st);
}

template <typename T>
int kz_dl_simt(const T *Xs, int64_t n, int d, int kind, double lengthscale, double variance,
               const T *V, T *W, T *Wdl, int c, cudaStream_t st) {
    if (n == 0 || c == 0) return LD_OK;
    T inv_l = (T)(1.0 / lengthscale);
    if (kind == LD_RBF)
        return launch_kz<T, LD_RBF, true>(Xs, n, d, V, W, Wdl, c, (T)variance, T(0), inv_l, st);
    return launch_kz<T, LD_MATERN52, true>(Xs, n, d, V, W, Wdl, c, (T)variance, T(0), inv_l, st);
}

template int prep_points<float>(const double *, int64_t, int, double, float *, cudaStream_t);
template int prep_points<double>(const double *, int64_t, int, double, double *, cudaStream_t);
template int kz_simt<float>(const float *, int64_t, int, int, double, double, const float *, float *, int, cudaStream_t);
template int kz_simt<double>(const double *, int64_t, int, int, double, double, const double *, double *, int, cudaStream_t);
template int kz_dl_simt<float>(const float *, int64_t, int, int, double, double, const float *, float *, float *, int, cudaStream_t);
template int kz_dl_simt<double>(const double *, int64_t, int, int, double, double, const double *, double *, double *, int, cudaStream_t);

// ------------------------------------------------------------- dispatch
template <>
size_t kz_any_workspace<double>(int64_t, int, int, int) { return 0; }
template <>
size_t kz_any_workspace<float>(int64_t n, int d, int c, int precision) {
    if (precision == LD_FP32) return 0;
    return kz_tc_workspace(n, d, c, precision);
}

template <>
int kz_any<double>(const double *Xs, int64_t n, int d, const ld_kernel &k, const double *V, double *W,
                   int c, int precision, Arena &, cudaStream_t st) {
    NvtxRange range("ld: kernel product");
    (void)precision;
    return kz_simt<double>(Xs, n, d, k.kind, k.variance, k.noise, V, W, c, st);
}
template <>
int kz_any<float>(const float *Xs, int64_t n, int d, const ld_kernel &k, const float *V, float *W,
                  int c, int precision, Arena &ws, cudaStream_t st) {
    NvtxRange range("ld: kernel product");
    if (precision == LD_FP32 || precision == LD_FP64)
        return kz_simt<float>(Xs, n, d, k.kind, k.variance, k.noise, V, W, c, st);
    return kz_tc(Xs, n, d, k.kind, k.variance, k.noise, V, W, c, precision, ws, st);
}

}  // namespace ld
