// Public entry points of the kernel product (ld_kz, ld_kz_dl).
#include "common.cuh"

using namespace ld;

namespace {
int check_kz_args(const double *X, int64_t n, int d, const ld_kernel &k, const void *V, void *W,
                  int c, int precision) {
    LD_REQUIRE(X && V && W && n > 0 && c > 0, "ld_kz: bad pointers or sizes");
    LD_REQUIRE(V != W, "ld_kz: W must not alias V");
    LD_REQUIRE(d >= 1 && d <= 32, "ld_kz: d must be in [1, 32]");
    LD_REQUIRE(d <= 8 || precision == LD_FP64 || precision == LD_FP32,
               "ld_kz: tensor-core precisions support d <= 8");
    LD_REQUIRE(c <= 4096, "ld_kz: at most 4096 columns");
    LD_REQUIRE(k.lengthscale > 0 && k.variance > 0 && k.noise >= 0 &&
                   (k.kind == LD_RBF || k.kind == LD_MATERN52),
               "ld_kz: bad kernel parameters");
    LD_REQUIRE(precision >= LD_FP64 && precision <= LD_F16X3_TC, "ld_kz: bad precision");
    return LD_OK;
}
}  // namespace

extern "C" {

size_t ld_kz_workspace_size(int64_t n, int32_t d, int32_t c, int32_t precision) {
    Arena a;
    a.measuring = true;
    if (precision == LD_FP64) {
        a.take<double>((size_t)n * d);
    } else {
        a.take<float>((size_t)n * d);
        a.take<char>(kz_any_workspace<float>(n, d, c, precision));
    }
    return a.off;
}

int ld_kz(const double *X_dev, int64_t n, int32_t d, ld_kernel kern, const void *V_dev,
          void *W_dev, int32_t c, int32_t precision, void *ws, size_t ws_bytes, void *stream) {
    clear_error();
    LD_TRY(check_kz_args(X_dev, n, d, kern, V_dev, W_dev, c, precision));
    cudaStream_t st = (cudaStream_t)stream;
    Arena a;
    LD_TRY(arena_open(a, ws, ws_bytes, ld_kz_workspace_size(n, d, c, precision)));
    int code = [&]() -> int {
        if (precision == LD_FP64) {
            double *Xs = a.take<double>((size_t)n * d);
            LD_TRY(prep_points<double>(X_dev, n, d, point_scale(kern), Xs, st));
            return kz_any<double>(Xs, n, d, kern, (const double *)V_dev, (double *)W_dev, c, precision, a, st);
        }
        float *Xs = a.take<float>((size_t)n * d);
        LD_TRY(prep_points<float>(X_dev, n, d, point_scale(kern), Xs, st));
        return kz_any<float>(Xs, n, d, kern, (const float *)V_dev, (float *)W_dev, c, precision, a, st);
    }();
    if (a.owned) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess && code == LD_OK) {
            set_error("ld_kz: %s", cudaGetErrorString(e));
            code = LD_ERR_CUDA;
        }
    }
    arena_close(a);
    return code;
}

int ld_kz_dl(const double *X_dev, int64_t n, int32_t d, ld_kernel kern, const void *V_dev,
             void *W_dev, void *Wdl_dev, int32_t c, int32_t precision, void *stream) {
    clear_error();
    LD_TRY(check_kz_args(X_dev, n, d, kern, V_dev, W_dev, c, precision));
    LD_REQUIRE(Wdl_dev && Wdl_dev != V_dev && Wdl_dev != W_dev, "ld_kz_dl: bad Wdl");
    cudaStream_t st = (cudaStream_t)stream;
    Arena a;
    size_t elt = precision == LD_FP64 ? sizeof(double) : sizeof(float);
    const size_t tc_ws = is_tc_precision(precision) ? kz_dl_tc_workspace(n, d, precision) : 0;
    LD_TRY(arena_open(a, nullptr, 0, (size_t)n * d * elt + 256 + tc_ws));
    int code = [&]() -> int {
        if (precision == LD_FP64) {
            double *Xs = a.take<double>((size_t)n * d);
            LD_TRY(prep_points<double>(X_dev, n, d, point_scale(kern), Xs, st));
            return kz_dl_simt<double>(Xs, n, d, kern.kind, kern.lengthscale, kern.variance,
                                      (const double *)V_dev, (double *)W_dev, (double *)Wdl_dev, c, st);
        }
        float *Xs = a.take<float>((size_t)n * d);
        LD_TRY(prep_points<float>(X_dev, n, d, point_scale(kern), Xs, st));
        if (is_tc_precision(precision))
            return kz_dl_tc(Xs, n, d, kern.kind, kern.lengthscale, kern.variance, (const float *)V_dev,
                            (float *)W_dev, (float *)Wdl_dev, c, precision, a, st);
        return kz_dl_simt<float>(Xs, n, d, kern.kind, kern.lengthscale, kern.variance,
                                 (const float *)V_dev, (float *)W_dev, (float *)Wdl_dev, c, st);
    }();
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && code == LD_OK) {
        set_error("ld_kz_dl: %s", cudaGetErrorString(e));
        code = LD_ERR_CUDA;
    }
    arena_close(a);
    return code;
}

}  // extern "C"
