/*
 * logdet.h -- C ABI of liblogdet.so, a GB300 (sm_103a) implementation of the
 * rational-function log-determinant estimator of Colthurst, Vasudevan, Lottes
 * and Patton, "Fast Approximate Determinants Using Rational Functions"
 * (arXiv 2405.03474):
 *
 *     log det M  =  log det P + tr log(M P^-1)
 *               ~=  log det P + (1/s) sum_i z_i^T r_k(B) z_i ,
 *
 * with r_k (k = 1, 3, 5) from Eq. 1 in the partial-fraction form of Table 1,
 * Rademacher probes z_i (Section 2, Algorithm 1 step 1), B = L^-1 M L^-T
 * (similar to M P^-1; P = L L^T) and P a randomized truncated-SVD
 * preconditioner (Section 2; Appendix "Truncated Randomized SVD").
 *
 * Conventions for every entry point:
 *   - Every block of vectors is ROW-MAJOR n-by-c: element (i, j) at [i*c + j].
 *     X is n-by-d points (float64), probes are n-by-s int8 (+1/-1).
 *   - Pointers named *_dev are device memory, *_host host memory.  The caller
 *     owns all of them; the library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; calls that return host scalars
 *     (ld_result, logdet_P, grad) synchronise that stream before returning.
 *   - `ws`/`ws_bytes`: caller-provided device scratch.  Pass ws = NULL to let
 *     the library cudaMalloc (and free before returning) what it needs;
 *     otherwise ws_bytes must be >= the size the matching *_workspace_size
 *     query returns, else LD_ERR_WORKSPACE.
 *   - Return value: LD_OK (0) or a negative ld_status.  On error nothing is
 *     left allocated; ld_last_error() gives a one-line reason.
 *   - Handles (ld_precond, ld_surrogate) own device memory and are freed with
 *     their *_free function.
 *   - One device: the current CUDA device of the calling thread.
 */
#ifndef LOGDET_H
#define LOGDET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
typedef enum {
    LD_OK = 0,
    LD_ERR_INVALID = -1,        /* bad argument (size, pointer, option)          */
    LD_ERR_NOT_SPD = -2,        /* a Cholesky pivot <= 0 (matrix not SPD)         */
    LD_ERR_NOT_CONVERGED = -3,  /* CG hit max_iters before rel_tol; out is filled */
    LD_ERR_CUDA = -4,           /* a CUDA runtime call failed                     */
    LD_ERR_WORKSPACE = -5,      /* ws_bytes smaller than required                 */
    LD_ERR_UNSUPPORTED = -6,    /* option combination not built                   */
    LD_ERR_DEVICE_TIMEOUT = -7  /* a device-side wait gave up (bounded spin)      */
} ld_status;

/* Kernel families of Section 3 (forms of Rasmussen & Williams):
 *   RBF:        k(r) = v exp(-r^2 / (2 l^2))
 *   MATERN52:   k(r) = v (1 + u + u^2/3) exp(-u),  u = sqrt(5) r / l
 * M = K + noise * I. */
typedef enum { LD_RBF = 0, LD_MATERN52 = 1 } ld_kernel_kind;

/* Arithmetic of the kernel product K V (the O(n^2) step of Algorithm 1):
 *   LD_FP64      SIMT float64 everywhere (parity mode)
 *   LD_FP32      SIMT float32 kernel values and products
 *   LD_BF16_TC   tensor cores (tcgen05), K and V rounded to bf16, fp32 accumulate
 *   LD_F16_TC    tensor cores, K and V rounded to fp16 (V scaled per column)
 *   LD_F16X3_TC  tensor cores, hi/lo fp16 split of K and V, 3 products
 *                (K_hi V_hi + K_hi V_lo + K_lo V_hi), fp32 accumulate
 * Non-FP64 modes keep CG vectors in fp32 and every reduction in fp64. */
typedef enum {
    LD_FP64 = 0,
    LD_FP32 = 1,
    LD_BF16_TC = 2,
    LD_F16_TC = 3,
    LD_F16X3_TC = 4
} ld_precision;

typedef struct {
    int32_t kind;        /* ld_kernel_kind */
    int32_t reserved;
    double lengthscale;  /* l > 0 */
    double variance;     /* v > 0 */
    double noise;        /* nu >= 0, added to the diagonal */
} ld_kernel;

typedef struct {
    int32_t order;           /* k of r_k: 1, 3 or 5 (Eq. 1, Table 1) */
    int32_t num_probes;      /* s, total probes (Algorithm 1 input s) */
    int32_t probes_per_block;/* columns solved together; num_probes % it == 0 */
    int32_t max_iters;       /* cap on Lanczos/CG steps */
    int32_t fixed_iters;     /* > 0: exactly t steps (Algorithm 1 input t);
                                0: iterate until rel_tol */
    int32_t precision;       /* ld_precision */
    int32_t residual_check;  /* 1: fill ld_result.max_resid (one extra K V pass) */
    int32_t dense;           /* 1: materialise M = K + noise I once (n*n words in the
                                workspace) and apply it from HBM (tensor-core
                                precisions: the dense tcgen05 product of
                                ld_dense_kz); 0: matrix-free */
    uint64_t seed;           /* SplitMix64 seed of the probes when probes_dev is NULL */
    double rel_tol;          /* stop when max_i ||r_i|| / ||z_i|| < rel_tol (seed system) */
    int32_t probe_kind;      /* 0: Rademacher (Section 3); 1: N(0, 1) by Box-Muller from the
                                same SplitMix64 stream (counters 2k, 2k+1; device-drawn only);
                                2: normal orthogonal (Appendix, probe types): per block of
                                probes_per_block (<= n) columns, the orthonormal factor (R
                                diagonal > 0) of the Gaussian block of those columns, each
                                column scaled by the norm of Gaussian column 2^30 + its
                                index (a chi_n draw); device-drawn only */
    int32_t probe_col0;      /* >= 0: stream column of this call's first device-drawn probe
                                (probe j uses column probe_col0 + j of the generator above;
                                0 for a whole estimate).  The probes of one estimate can so
                                be split over several calls or processes, each running the
                                same P and its own columns; ld_combine joins their per-probe
                                brackets into the estimate (Algorithm 1's output) */
} ld_options;

typedef struct {
    double logdet;        /* the estimate: logdet_P + trace_est */
    double logdet_P;      /* log det P */
    double trace_est;     /* (1/s) sum_i [b |z_i|^2 + sum_j c_j q_ij] */
    double std_err;       /* sample std of the per-probe brackets / sqrt(s) */
    int32_t iters;        /* max CG steps over the probe blocks */
    int32_t converged;    /* 1 if every column met rel_tol (or fixed_iters ran) */
    double max_resid[5];  /* residual check: max_i ||z_i - (B + sigma_j) x_ij|| / ||z_i||,
                             fp64 norms; entries beyond the order are 0.  The product
                             B x_ij inside it runs in the estimate's precision: fp64
                             in LD_FP64; in the other precisions its relative error
                             (~1e-6 for LD_F16X3_TC and LD_FP32, ~1e-3 for LD_F16_TC,
                             ~1e-2 for LD_BF16_TC) times |B x| / |z| is the floor
                             below which a residual is not resolved */
    double final_rel_resid; /* max_i ||r_i|| / ||z_i|| of the seed system at exit */
    double slq_logdet;    /* stochastic Lanczos quadrature (Ubaru et al., Section 3's
                             comparison method) from the same Lanczos tridiagonals:
                             log det P + (1/s) sum_i |z_i|^2 sum_k q_ik^2 log theta_ik */
} ld_result;

typedef struct ld_precond ld_precond;
typedef struct ld_surrogate ld_surrogate;

/* ------------------------------------------------------------------- misc */
const char *ld_status_string(int status);
/* Reason for the last non-OK status returned on this thread ("" if none). */
const char *ld_last_error(void);
int ld_version(void);

/* Partial fractions of r_k (Table 1, derived here from the Eq. 1 closed forms):
 * r_k(x) = b + sum_{j<k} c[j] / (x + sigma[j]), sigma ascending, c < 0.
 * b, c, sigma are host pointers (c, sigma of length k). */
int ld_rk_coeffs(int32_t order, double *b, double *c, double *sigma);

/* ------------------------------------------------------------ kernel product
 * W = (K(X, X) + noise I) V  -- the matrix-free product Algorithm 1 step 2
 * spends its O(t n^2) time in (Section 2, complexity paragraph).
 * X_dev: n-by-d float64.  V_dev, W_dev: n-by-c row-major, float64 for
 * LD_FP64, float32 otherwise (W_dev must not alias V_dev).  No workspace for
 * FP64/FP32; TC modes need ld_kz_workspace_size(n, d, c, precision) bytes.
 * Sizes: n >= 1, 1 <= c <= 4096, 1 <= d <= 32 (d <= 8 in the tensor-core
 * precisions); anything else, empty inputs included, returns LD_ERR_INVALID
 * before any device work.  ws = NULL: the call allocates and frees its own
 * workspace.  Tensor-core dispatch (all within the call): c <= 48 and n >= 256
 * the symmetric product (each 128 x 128 block evaluated once, the points taken
 * in a Morton order of its own and blocks whose kernel values are all <= 2^-10
 * of the variance rounded once to fp16 in LD_F16X3_TC), 256 < c <= 512 in
 * fp16/bf16 the one-pass wide product, otherwise the general product in chunks
 * of 256 columns. */
size_t ld_kz_workspace_size(int64_t n, int32_t d, int32_t c, int32_t precision);
int ld_kz(const double *X_dev, int64_t n, int32_t d, ld_kernel kern,
          const void *V_dev, void *W_dev, int32_t c, int32_t precision,
          void *ws, size_t ws_bytes, void *stream);

/* The same product with no device allocation at all.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc (a plug-in
 * whose host framework owns all device memory through its own pool, a
 * latency-critical loop where cudaMalloc/cudaFree would synchronise the device,
 * a process under a hard device-memory cap).  Scratch comes from one static
 * __device__ array of ld_kz_static_capacity() bytes (32 MiB) that every GPU
 * loading the library keeps until process exit; sizes whose scratch
 * (ld_kz_workspace_size) exceeds it return LD_ERR_WORKSPACE.  The first call on
 * a device looks up the array's address there (cudaGetSymbolAddress): make that
 * one-time first call before any stream capture begins.  Like ld_kz, a call in
 * a tensor-core precision synchronises `stream` before returning; in FP64 and
 * FP32 the work stays queued on it.  All calls share the array: calls that
 * overlap on the GPU race.  Arguments, size limits (d <= 32; d <= 8 in the
 * tensor-core precisions) and results are those of ld_kz. */
size_t ld_kz_static_capacity(void);
int ld_kz_static(const double *X_dev, int64_t n, int32_t d, ld_kernel kern,
                 const void *V_dev, void *W_dev, int32_t c, int32_t precision,
                 void *stream);

/* Same pass computing both W = K V and W_dl = (dK/dl) V (for the gradient,
 * Section 3's CG-based gradient; derivative forms above).  noise is NOT added
 * to either.  LD_FP64 / LD_FP32: SIMT.  Tensor-core precisions (d <= 8): one
 * tcgen05 pass evaluates k and dk/dl per pair with a shared exponential and
 * accumulates both products in tensor memory, 64 columns per launch, in the
 * precision's rounding of K, dK/dl and V (hi/lo fp16 for LD_F16X3_TC); the call
 * allocates its scratch, synchronises the stream and returns
 * LD_ERR_DEVICE_TIMEOUT if a device-side wait gave up. */
int ld_kz_dl(const double *X_dev, int64_t n, int32_t d, ld_kernel kern,
             const void *V_dev, void *W_dev, void *Wdl_dev, int32_t c,
             int32_t precision, void *stream);

/* Stored dense variant of the same product (Algorithm 1 step 2 with M kept in
 * memory): M = K + noise I written row-major n-by-n (float64 for LD_FP64, float32
 * otherwise; ld_dense_bytes(n, precision) bytes, caller-owned), then W = M V
 * (V, W n-by-c row-major, float64 for LD_FP64, else float32) reading M once per
 * pass over a chunk of columns.  LD_FP64 / LD_FP32: CUDA-core GEMM, asynchronous
 * on the stream.  Tensor-core precisions: chunks of up to 256 columns; a chunk of
 * at most 128 columns with n % 4 == 0, n >= 128 and M 16-byte aligned streams M
 * into shared memory by TMA tensor copies, any other chunk by per-thread loads.
 * Tensor-core precisions (LD_BF16_TC, LD_F16_TC, LD_F16X3_TC; c <= 4096): M is
 * rounded (or split hi/lo) like the computed kernel values of ld_kz after
 * scaling by the power of two that brings max_i |M_ii| into [2^14, 2^15), so M
 * must be positive semidefinite (|M_ij| <= max_i M_ii, true of every K + noise I;
 * an entry beyond about twice that overflows fp16 and makes W non-finite); the call
 * allocates its scratch (the fp16/bf16 image of V), synchronises the stream and
 * returns LD_ERR_DEVICE_TIMEOUT if a device-side wait gave up. */
size_t ld_dense_bytes(int64_t n, int32_t precision);
int ld_dense_materialize(const double *X_dev, int64_t n, int32_t d, ld_kernel kern,
                         int32_t precision, void *M_dev, void *stream);
int ld_dense_kz(const void *M_dev, int64_t n, const void *V_dev, void *W_dev, int32_t c,
                int32_t precision, void *stream);

/* N(0, 1) block (float64, row-major n-by-s): entry (i, j) is
 * sqrt(-2 ln u1) cos(2 pi u2) (Box & Muller 1958) with u1, u2 the (0, 1) uniforms
 * (top 53 bits + 1/2) * 2^-53 of SplitMix64 outputs 2k and 2k + 1, k = (col0 + j) n + i. */
int ld_gaussian(uint64_t seed, int64_t n, int32_t s, int32_t col0, double *Z_dev, void *stream);

/* Rademacher block from the SplitMix64 stream (Steele, Lea & Flood 2014):
 * Z[i, j] (row-major n-by-s int8) uses counter (col0 + j) * n + i and is +1
 * when bit 63 of the output is 0, else -1 (Algorithm 1 step 1 with D the
 * Rademacher distribution of Section 3). */
int ld_rademacher(uint64_t seed, int64_t n, int32_t s, int32_t col0,
                  int8_t *Z_dev, void *stream);

/* --------------------------------------------------------- preconditioner
 * P = D + A A^T by randomized truncated SVD (Section 2 "randomized, truncated
 * SVD" after Halko et al. Alg. 4.1 + 5.3; Section 3: rank, iterations):
 *   Omega = Rademacher(seed) n-by-rank, Y = M Omega,
 *   power_iters times: Y = M orth(Y);  Q = orth(Y);  C = Q^T M Q;
 *   A = Q chol(C);  D = max(diag(M) - rowsumsq(A), max(noise, 1e-12 diag(M))).
 * The handle stores the split factor L = D^1/2 (I + Q_G (C_P - I) Q_G^T) with
 * G = D^-1/2 A = Q_G R_G, C_P C_P^T = I + R_G R_G^T, and
 * log det P = sum log D + 2 sum log diag(C_P).
 * precision: LD_FP64 keeps factors in float64 (products FP64); any other
 * value keeps n-by-rank factors in float32, r-by-r factors in float64, and
 * runs the M products in that precision.
 * rank = 0 gives P = diag(M) (Appendix "Diagonal"); P = NULL in
 * logdet_estimate means P = I (Appendix "Identity").  A NaN or Inf coordinate
 * in X returns LD_ERR_INVALID; a Cholesky pivot <= 0 returns LD_ERR_NOT_SPD. */
size_t precond_workspace_size(int64_t n, int32_t d, int32_t rank, int32_t precision);
int precond_build(const double *X_dev, int64_t n, int32_t d, ld_kernel kern,
                  int32_t rank, int32_t power_iters, uint64_t seed,
                  int32_t precision, void *ws, size_t ws_bytes, void *stream,
                  ld_precond **out);
/* Appendix "Truncated Randomized SVD plus scaling": the same A, with the
 * diagonal replaced by the constant a > 0 (the paper takes a = jitter + noise
 * variance): P = a I + A A^T.  Same workspace as precond_build. */
int precond_build_scaled(const double *X_dev, int64_t n, int32_t d, ld_kernel kern,
                         int32_t rank, int32_t power_iters, uint64_t seed, double a,
                         int32_t precision, void *ws, size_t ws_bytes, void *stream,
                         ld_precond **out);
/* Build the same handle from host A (n-by-rank row-major) and D (n). */
int precond_import(const double *A_host, const double *D_host, int64_t n,
                   int32_t rank, int32_t precision, void *stream,
                   ld_precond **out);
/* Copy A = D^1/2 Q_G R_G (n-by-rank) and D (n) to host; logdet_P optional. */
int precond_export(const ld_precond *P, double *A_host, double *D_host,
                   double *logdet_P, void *stream);
int precond_info(const ld_precond *P, int64_t *n, int32_t *rank,
                 int32_t *precision, double *logdet_P);
/* V_dev (n-by-c) -> W_dev = L^-1 V (transpose = 0) or L^-T V (transpose = 1);
 * float64 for an LD_FP64 handle, float32 otherwise; W may alias V. */
int precond_apply(const ld_precond *P, int32_t transpose, const void *V_dev,
                  void *W_dev, int32_t c, void *stream);
void precond_free(ld_precond *P);

/* --------------------------------------------------------------- estimator
 * Algorithm 1 with the shifted solves done by a block multi-shift CG on
 * B = L^-1 M L^-T (Section 2 multi-shift paragraph, after Jegerlehner): each
 * probe block runs CG on the seed system B + sigma_min I, the Lanczos
 * tridiagonal T is rebuilt from the CG coefficients, and
 * q_ij = |z_i|^2 e_1^T (T_i + (sigma_j - sigma_min) I)^-1 e_1 by a tridiagonal
 * solve (Algorithm 1 step 3, Thomas), giving
 *   logdet = log det P + (1/s) sum_i [ b |z_i|^2 + sum_j c_j q_ij ].
 * P = NULL means P = I.  probes_dev: n-by-num_probes int8 (+-1), or NULL to
 * draw them with ld_rademacher(opt->seed, ...).  per_probe_host: optional
 * (num_probes doubles) receives the bracket per probe.
 * Returns LD_ERR_INVALID for a NaN or Inf coordinate in X (checked on the
 * device first), LD_ERR_NOT_CONVERGED (with *out filled) when rel_tol was not
 * met, and LD_ERR_NOT_SPD (with *out filled) when the estimate is not finite
 * or a CG column met p^T (B + sigma_min) p <= 0 (a matrix that is not SPD; in the
 * reduced precisions this happens when the rounding of K, about 2^-8 (bf16),
 * 2^-11 (fp16), 2^-22 (hi/lo fp16) of each entry times the largest row sum of K,
 * reaches the noise on the diagonal). */
size_t logdet_workspace_size(int64_t n, int32_t d, const ld_precond *P,
                             const ld_options *opt);
int logdet_estimate(const double *X_dev, int64_t n, int32_t d, ld_kernel kern,
                    const ld_precond *P, const ld_options *opt,
                    const int8_t *probes_dev, double *per_probe_host,
                    void *ws, size_t ws_bytes, void *stream, ld_result *out);

/* Algorithm 1's output from per-probe brackets (host only, no device work):
 * logdet = logdet_P + trace_est, trace_est = (1/S) sum_i bracket_i (summed in
 * index order), std_err = sample std of the brackets / sqrt(S); every other
 * field of *out is 0 except logdet_P.  For an estimate whose probe blocks ran
 * in several calls or processes (each with the same P, its own probe_col0 and
 * per_probe_host), the brackets concatenated in probe order give the same
 * value as one call over all probes.  S >= 1; NULL pointers: LD_ERR_INVALID. */
int ld_combine(const double *brackets_host, int32_t num_probes, double logdet_P, ld_result *out);

/* Gradient of the estimator with P and the probes held fixed:
 *   d/dtheta = (1/s) sum_i sum_j (-c_j) y_ij^T (dM/dtheta) y_ij,
 *   y_ij = L^-T x_ij,  x_ij = (B + sigma_j I)^-1 z_i,
 * for theta = (lengthscale, variance, noise) into grad_host[3], plus the
 * estimate itself in *out.  dM/dl = dK/dl, dM/dv = K/v, dM/dnu = I.  Every
 * precision: the derivative pass (K y and dK/dl y for all s m columns) runs as
 * ld_kz_dl does in that precision, the dots y^T (.) y in fp64. */
int logdet_grad(const double *X_dev, int64_t n, int32_t d, ld_kernel kern,
                const ld_precond *P, const ld_options *opt,
                const int8_t *probes_dev, void *ws, size_t ws_bytes,
                void *stream, double *grad_host, ld_result *out);

/* ------------------------------------------------------------- diagnostics
 * Not part of the paper: measurement hooks for benchmarks.
 * ld_launch_count: number of kernels this library has launched in the process.
 * ld_profile_begin / ld_profile_end: between the two calls every launch of the
 * kernel product (the O(n^2) step) is bracketed by CUDA events recorded on its
 * own stream; end synchronises those events and returns the summed device
 * time (ms), the launch count, the kernel evaluations (n^2 per launch; n(n+1)/2
 * for the symmetric product, which evaluates each pair once) and the
 * multiply-add flops (2 n^2 c per product) they did.  Single-threaded use. */
int64_t ld_launch_count(void);
/* Failure-detection self-test: one thread waits on an mbarrier that nothing
 * completes, with the bounded wait the kernel product uses (budget in SM
 * cycles, <= 4e9).  Returns LD_ERR_DEVICE_TIMEOUT once the budget runs out; the
 * context stays usable.  Not part of the paper. */
int ld_selftest_wait_timeout(int64_t budget_cycles, void *stream);
int ld_profile_begin(void);
int ld_profile_end(double *kz_ms, int64_t *kz_launches, double *kz_pairs, double *kz_mma_flops);
/* The same totals of the last closed window for one kernel: 0 the general
 * tensor-core product, 1 the symmetric tensor-core product, 2 the SIMT product,
 * 3 the stored dense product (CUDA-core GEMM or tensor cores), 4 the one-pass wide (256 < c <= 512) tensor-core
 * product, 5 the tensor-core derivative pass of the gradient (K V and dK/dl V).  LD_ERR_INVALID for another
 * id. */
int ld_profile_kernel(int32_t kernel, double *ms, int64_t *launches, double *pairs, double *mma_flops);

/* --------------------------------------------------------------- surrogate
 * MLP 4 -> 128 -> 128 -> 128 -> 1 with exact GELU, fp32, trained by Adam on
 * mean squared error; maps (log l, log v, log nu, log n) to a standardised
 * log det.  Not part of the paper: an addition for hyperparameter search,
 * trained on values logdet_estimate produced.  Parameters are one flat
 * vector: W1 (128x4), b1, W2 (128x128), b2, W3 (128x128), b3, W4 (1x128), b4,
 * each W row-major (out, in): 33793 floats. */
int surrogate_create(uint64_t seed, void *stream, ld_surrogate **out);
int surrogate_set_params(ld_surrogate *S, const float *params_host, void *stream);
int surrogate_get_params(const ld_surrogate *S, float *params_host, void *stream);
/* The affine normalisation the handle applies (set by surrogate_train from its
 * data): 10 floats, input means mu[4], input scales sd[4], target mean, target
 * scale; with the parameters it is the whole state of a trained network (a
 * checkpoint).  set: scales must be > 0 and every entry finite, else
 * LD_ERR_INVALID. */
int surrogate_get_norm(const ld_surrogate *S, float *norm_host, void *stream);
int surrogate_set_norm(ld_surrogate *S, const float *norm_host, void *stream);
/* One full-batch gradient: loss and d loss / d params for (theta_dev N-by-4,
 * y_dev N), written to grad_host (33793) if not NULL. */
int surrogate_loss_grad(ld_surrogate *S, const float *theta_dev, const float *y_dev,
                        int32_t N, double *loss_host, float *grad_host, void *stream);
/* epochs of minibatch Adam (lr, beta1 0.9, beta2 0.999, eps 1e-8) over the
 * N samples in order (batch rows at a time); final full-batch loss returned. */
int surrogate_train(ld_surrogate *S, const float *theta_dev, const float *y_dev,
                    int32_t N, int32_t epochs, int32_t batch, float lr,
                    void *stream, double *final_loss_host);
/* out_dev[Q] = f(q), dout_dev[Q*4] = df/dq (may be NULL). */
int surrogate_infer(const ld_surrogate *S, const float *q_dev, int32_t Q,
                    float *out_dev, float *dout_dev, void *stream);
void surrogate_free(ld_surrogate *S);

#ifdef __cplusplus
}
#endif
#endif /* LOGDET_H */
