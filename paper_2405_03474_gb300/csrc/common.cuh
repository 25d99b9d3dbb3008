// Internal declarations shared by the translation units of liblogdet.so.
// Public API: include/logdet.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "logdet.h"

namespace ld {

// Scoped NVTX range around a phase (preconditioner build, sketch product, CG
// iteration, residual pass, adjoint, kernel product): visible in Nsight timelines,
// a no-op when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ------------------------------------------------------------ error state
void set_error(const char *fmt, ...);
const char *last_error();
void clear_error();

#define LD_CHECK_CUDA(...)                                                         \
    do {                                                                           \
        cudaError_t e_ = (__VA_ARGS__);                                            \
        if (e_ != cudaSuccess) {                                                   \
            ::ld::set_error("%s:%d %s: %s", __FILE__, __LINE__, #__VA_ARGS__,      \
                            cudaGetErrorString(e_));                               \
            return LD_ERR_CUDA;                                                    \
        }                                                                          \
    } while (0)

#define LD_TRY(...)                                                                \
    do {                                                                           \
        int st_ = (__VA_ARGS__);                                                   \
        if (st_ != LD_OK) return st_;                                              \
    } while (0)

#define LD_REQUIRE(cond, ...)                                                      \
    do {                                                                           \
        if (!(cond)) {                                                             \
            ::ld::set_error(__VA_ARGS__);                                          \
            return LD_ERR_INVALID;                                                 \
        }                                                                          \
    } while (0)

// Launch accounting: every kernel launch site reports through check_launch
// with the number of kernels it launched since the previous check.
void count_launches(int k);

inline int check_launch(const char *what, int launches = 1) {
    count_launches(launches);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    return LD_OK;
}

// Optional timing of the kernel-product launches (CUDA events on the launch
// stream), enabled between ld_profile_begin and ld_profile_end.
// kernel ids of the profile totals (ld_profile_kernel)
enum { PROF_KZ_TC = 0, PROF_KZ_SYM = 1, PROF_KZ_SIMT = 2, PROF_DENSE = 3, PROF_KZ_WIDE = 4, PROF_KZ_DL = 5,
       PROF_KERNELS = 6 };
int prof_begin_launch(cudaStream_t st, int kernel, double pairs, double mma_flops);  // -1 when off
void prof_end_launch(cudaStream_t st, int slot);

// ------------------------------------------------------------- workspace
// Bump allocator over caller scratch (or over one cudaMalloc when ws == NULL).
// Two modes: "measure" (base == nullptr, only counts bytes) and "carve".
struct Arena {
    char *base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    bool owned = false;
    bool measuring = false;
    bool overflow = false;

    template <typename T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        size_t at = off;
        off += bytes;
        if (measuring) return nullptr;
        if (off > cap) {
            overflow = true;
            return nullptr;
        }
        return reinterpret_cast<T *>(base + at);
    }
};

// Open an arena over caller scratch, or allocate `need` bytes when ws == NULL.
int arena_open(Arena &a, void *ws, size_t ws_bytes, size_t need);
void arena_close(Arena &a);

// ----------------------------------------------------------- coefficients
struct RkCoeffs {
    int m = 0;           // number of poles (= order)
    double b = 0.0;
    double c[5] = {0};
    double sigma[5] = {0};  // ascending
};
int rk_coeffs(int order, RkCoeffs &out);

// ----------------------------------------------------- kernel evaluation
// Points are pre-scaled so that the kernel is a function of the squared scaled
// distance u2 = |xs - ys|^2:
//   RBF:      xs = x / (l sqrt 2),  k = v exp(-u2)
//   Matern52: xs = x sqrt(5) / l,   k = v (1 + u + u^2/3) exp(-u), u = sqrt(u2)
double point_scale(const ld_kernel &k);

template <typename T>
int prep_points(const double *X, int64_t n, int d, double scale, T *Xs, cudaStream_t st);
// LD_ERR_INVALID if any of the n*d coordinates is NaN or Inf (flag_dev: one device
// int of scratch; synchronises the stream)
int check_points_finite(const double *X, int64_t n, int d, int *flag_dev, cudaStream_t st);

// W = (K + noise I) V (SIMT), V, W n-by-c row-major
template <typename T>
int kz_simt(const T *Xs, int64_t n, int d, int kind, double variance, double noise,
            const T *V, T *W, int c, cudaStream_t st);
// W = K V, Wdl = (dK/dl) V (SIMT, no noise)
template <typename T>
int kz_dl_simt(const T *Xs, int64_t n, int d, int kind, double lengthscale, double variance,
               const T *V, T *W, T *Wdl, int c, cudaStream_t st);

// A spatially coherent order of the n points (Morton codes over the bounding box, stable
// radix sort): perm[r] is the point at position r (point_order.cu); d <= 8, n < 2^31.
size_t point_order_workspace(int64_t n, int d);
int point_order(const float *Xs, int64_t n, int d, int *perm, Arena &ws, cudaStream_t st);

// W = K V, Wdl = (dK/dl) V on the tensor cores (no noise), any number of columns
// (kz_dl_tc.cu); Xs pre-scaled like every product
size_t kz_dl_tc_workspace(int64_t n, int d, int precision);
int kz_dl_tc(const float *Xs, int64_t n, int d, int kind, double lengthscale, double variance, const float *V,
             float *W, float *Wdl, int c, int precision, Arena &ws, cudaStream_t st);

// stored dense M = K + noise I (row-major n x n) and W = M V (dense_path.cu)
template <typename T>
int dense_materialize(const T *Xs, int64_t n, int d, const ld_kernel &k, T *M, cudaStream_t st);
template <typename T>
int dense_product(const T *M, int64_t n, const T *V, T *W, int c, cudaStream_t st);

// tensor-core product (float vectors)
inline bool is_tc_precision(int precision) {
    return precision == LD_BF16_TC || precision == LD_F16_TC || precision == LD_F16X3_TC;
}
size_t kz_tc_workspace(int64_t n, int d, int c, int precision);
// W = M V on the tensor cores for a stored dense M (row-major n x n float32, positive
// semidefinite: it is scaled by a power of two taken from its diagonal), kz_tc.cu
size_t dense_tc_workspace(int64_t n, int c, int precision);
// Stored-M product fed by tensor copies (dense_tma.cu): columns c0 .. c0 + N - 1 of
// W = M V from the operand image and column scales dense_tc prepared.
bool dense_tma_eligible(const float *M, int64_t n, int N, int precision);
int dense_tma(const float *M, int64_t n, const uint8_t *img, const float *colinv, const float *mscale, float *W,
              int c, int c0, int N, int precision, int *err, cudaStream_t st);
int dense_tc(const float *M, int64_t n, const float *V, float *W, int c, int precision, Arena &ws,
             cudaStream_t st);
// symmetric tensor-core product for c <= 16 (each kernel value evaluated once)
// the one-pass product for 256 < c <= 512 columns, single fp16 / bf16 product (kz_wide.cu)
bool kz_wide_eligible(int64_t n, int d, int c, int precision);
size_t kz_wide_workspace(int64_t n, int d, int c, int precision);
int kz_wide(const float *Xs, int64_t n, int d, int kind, double variance, double noise, const float *V,
            float *W, int c, int precision, Arena &ws, cudaStream_t st);
bool kz_sym_eligible(int64_t n, int d, int c, int precision);
size_t kz_sym_workspace(int64_t n, int d, int c, int precision);
int kz_sym(const float *Xs, int64_t n, int d, int kind, double variance, double noise, const float *V, float *W,
           int c, int precision, Arena &ws, cudaStream_t st);
int kz_tc(const float *Xs, int64_t n, int d, int kind, double variance, double noise,
          const float *V, float *W, int c, int precision, Arena &ws, cudaStream_t st);

// dispatch on precision: T = double for LD_FP64, float otherwise
template <typename T>
int kz_any(const T *Xs, int64_t n, int d, const ld_kernel &k, const T *V, T *W, int c,
           int precision, Arena &ws, cudaStream_t st);
template <typename T>
size_t kz_any_workspace(int64_t n, int d, int c, int precision);

// ------------------------------------------------------------------ BLAS
// C(m x q) = alpha A(m x k) B(k x q) + beta C, row-major with leading dims.
template <typename T>
int gemm_nn(int64_t m, int q, int k, T alpha, const T *A, int64_t lda, const T *B, int64_t ldb,
            T beta, T *C, int64_t ldc, cudaStream_t st);
// Cd(p x q) (double) = A(m x p)^T B(m x q), reduction over m split across CTAs
// with fp64 partials summed in a fixed order.  part: >= splitk_partials(...) doubles.
size_t gemm_tn_partials(int64_t m, int p, int q);
template <typename T>
int gemm_tn(int64_t m, int p, int q, const T *A, int64_t lda, const T *B, int64_t ldb,
            double *Cd, double *part, cudaStream_t st);
// out[j] = sum_i A[i*c+j] * B[i*c+j] in fp64, deterministic.
size_t coldot_partials(int64_t n, int c);
template <typename T>
int coldot(int64_t n, int c, const T *A, const T *B, double *out, double *part, cudaStream_t st);

// small helpers
template <typename Tin, typename Tout>
int convert(const Tin *in, Tout *out, int64_t count, cudaStream_t st);
template <typename T>
int int8_to(const int8_t *in, T *out, int64_t count, cudaStream_t st);
template <typename T>
int scale_rows(const T *in, const T *rowscale, T *out, int64_t n, int c, cudaStream_t st);
template <typename T>
int axpy(int64_t count, T alpha, const T *x, T *y, cudaStream_t st);  // y += alpha x
int rademacher(uint64_t seed, int64_t n, int s, int col0, int8_t *Z, cudaStream_t st);
template <typename T>
int gaussian(uint64_t seed, int64_t n, int s, int col0, T *Z, cudaStream_t st);
// Normal orthogonal probes: Z (n x s) = Q S, Q the orthonormal factor (positive
// R diagonal) of the Gaussian block of columns col0.., S_cc the norm of the
// Gaussian column ORF_NORM_COL0 + col0 + c.  G, H, tmp: n x s scratch; the r x r
// cores come from the arena's free tail (orth_probe_tail_bytes).
constexpr int ORF_NORM_COL0 = 1 << 30;
size_t orth_probe_tail_bytes(int64_t n, int s);
template <typename T>
int orthogonal_probes(uint64_t seed, int64_t n, int s, int col0, T *Z, T *G, T *H, T *tmp, Arena &a,
                      cudaStream_t st);

// ------------------------------------------------ small dense (fp64, r x r)
// In-place lower Cholesky of A (r x r row-major, lower part used) after adding
// `shift` to the diagonal; *status (device int) = 0 ok, k+1 if pivot k <= 0.
int dense_chol(double *A, int r, double shift, int *status, cudaStream_t st);
// Linv = L^-1 for lower-triangular L (r x r), zero above the diagonal.
int dense_trinv_lower(const double *L, double *Linv, int r, cudaStream_t st);
// C = alpha op(A) op(B) + beta C for small fp64 matrices (r x r or r x c).
int dense_gemm(int m, int q, int k, double alpha, const double *A, int lda, bool ta,
               const double *B, int ldb, bool tb, double beta, double *C, int ldc,
               cudaStream_t st);
// out = sum of log(diag(L)) over r entries (device scalar), plus trace helpers.
int dense_sumlogdiag(const double *L, int r, double *out, cudaStream_t st);
int dense_trace(const double *A, int r, double *out, cudaStream_t st);
// A(r x r) <- (A + A^T) / 2
int dense_symmetrize(double *A, int r, cudaStream_t st);
// dst (T, r x r) = src (+ add * I), optional transpose
template <typename T>
int dense_export(const double *src, T *dst, int r, double add_identity, bool transpose,
                 cudaStream_t st);

}  // namespace ld

// ---------------------------------------------------- the opaque handles
struct ld_precond {
    int64_t n = 0;
    int r = 0;
    int precision = LD_FP32;
    void *Qg = nullptr;       // n x r (T)
    void *CmI = nullptr;      // r x r (T): C_P^-1 - I
    void *CmIT = nullptr;     // r x r (T): C_P^-T - I
    void *dinv_sqrt = nullptr;// n (T)
    double *D = nullptr;      // n
    double *RG = nullptr;     // r x r (upper), G = Qg RG
    double logdet_P = 0.0;
};

namespace ld {
// L^-1 / L^-T apply on float or double handles (precond.cu)
template <typename T>
int precond_apply_impl(const ld_precond *P, bool transpose, const T *V, T *W, int c, double *Td,
                       T *Tt, T *Ut, double *part, cudaStream_t st);
size_t precond_apply_scratch_doubles(const ld_precond *P, int c);
}  // namespace ld
