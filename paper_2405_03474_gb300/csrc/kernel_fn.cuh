// Covariance functions of squared scaled distance (SIMT fp32/fp64), shared by the
// matrix-free product (kz_simt.cu) and the dense materialisation (dense_path.cu).
// Points are pre-scaled (point_scale): RBF k = v exp(-u2); Matern-5/2 k =
// v (1 + u + u^2/3) exp(-u), u = sqrt(u2) (Section 3 kernels, Rasmussen & Williams).
#pragma once

#include "common.cuh"

namespace ld {
namespace kfn {

template <typename T>
__device__ __forceinline__ T dev_exp(T x);
template <>
__device__ __forceinline__ double dev_exp<double>(double x) { return exp(x); }
template <>
__device__ __forceinline__ float dev_exp<float>(float x) { return expf(x); }
template <typename T>
__device__ __forceinline__ T dev_sqrt(T x);
template <>
__device__ __forceinline__ double dev_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dev_sqrt<float>(float x) { return sqrtf(x); }

// kernel value from squared scaled distance u2 (see point_scale)
template <typename T, int KIND>
__device__ __forceinline__ T kval(T u2, T var) {
    if (KIND == LD_RBF) return var * dev_exp<T>(-u2);
    T u = dev_sqrt<T>(u2);
    return var * (T(1) + u + u2 * T(1.0 / 3.0)) * dev_exp<T>(-u);
}

// kernel value and its lengthscale derivative
template <typename T, int KIND>
__device__ __forceinline__ void kval_dl(T u2, T var, T inv_l, T &k, T &dk) {
    if (KIND == LD_RBF) {
        k = var * dev_exp<T>(-u2);
        dk = k * T(2) * u2 * inv_l;  // r^2/l^3 = 2 u2 / l
    } else {
        T u = dev_sqrt<T>(u2);
        T e = var * dev_exp<T>(-u);
        k = (T(1) + u + u2 * T(1.0 / 3.0)) * e;
        dk = u2 * T(1.0 / 3.0) * inv_l * (T(1) + u) * e;  // v u^2/(3l) (1+u) e^-u
    }
}

}  // namespace kfn
}  // namespace ld
