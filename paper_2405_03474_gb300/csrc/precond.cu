// Randomized truncated-SVD preconditioner P = D + A A^T (Section 2, after Halko,
// Martinsson & Tropp Algorithms 4.1 and 5.3; Appendix "Truncated Randomized
// SVD") and its split factor L with P = L L^T:
//
//   G = D^-1/2 A = Q_G R_G (thin QR),  C_P C_P^T = I + R_G R_G^T (Cholesky),
//   L^-1 = (I + Q_G (C_P^-1 - I) Q_G^T) D^-1/2,
//   L^-T = D^-1/2 (I + Q_G (C_P^-T - I) Q_G^T),
//   log det P = sum log D + 2 sum log diag C_P   (matrix determinant lemma).
//
// Orthonormalisation is CholeskyQR2 with a tiny relative diagonal shift in
// each pass (Gram in fp64, factors r x r in fp64).  Y = Q R holds exactly for
// any invertible pass factor; the shift only bounds how far Q^T Q may sit from I.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace ld {

namespace {

// D_i = max(diag(M) - rowsumsq(A), floor), or the constant const_d when it is > 0
// (the "plus scaling" variant P = a I + A A^T).
template <typename T>
__global__ void diag_resid_kernel(const T *A, int64_t n, int r, double diagM, double floor, double const_d,
                                  double *D, T *dinv, double *part) {
    __shared__ double red[32];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double lg = 0.0;
    if (i < n) {
        double s = 0.0;
        for (int k = 0; k < r; ++k) {
            double a = (double)A[i * r + k];
            s += a * a;
        }
        double d = const_d > 0.0 ? const_d : fmax(diagM - s, floor);
        D[i] = d;
        dinv[i] = (T)(1.0 / sqrt(d));
        lg = log(d);
    }
    for (int o = 16; o > 0; o >>= 1) lg += __shfl_down_sync(0xffffffffu, lg, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lg;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void sum_serial_kernel(const double *part, int cnt, double *out, double scale,
                                  const double *add_scaled) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < cnt; ++k) s += part[k];
        *out = s + (add_scaled ? scale * (*add_scaled) : 0.0);
    }
}

template <typename T>
__global__ void import_kernel(const double *Ah, const double *D, int64_t n, int r, T *G, T *dinv,
                              double *part) {
    __shared__ double red[32];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double lg = 0.0;
    if (i < n) {
        double d = D[i];
        double is = 1.0 / sqrt(d);
        dinv[i] = (T)is;
        for (int k = 0; k < r; ++k) G[i * r + k] = (T)(Ah[i * r + k] * is);
        lg = log(d);
    }
    for (int o = 16; o > 0; o >>= 1) lg += __shfl_down_sync(0xffffffffu, lg, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lg;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// A = D^1/2 Q_G R_G row i (fp64 out)
template <typename T>
__global__ void export_A_kernel(const T *Qg, const double *RG, const double *D, int64_t n, int r,
                                double *A) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * r) return;
    int64_t i = t / r;
    int k = (int)(t % r);
    double s = 0.0;
    for (int l = 0; l <= k; ++l) s += (double)Qg[i * r + l] * RG[(size_t)l * r + k];
    A[t] = sqrt(D[i]) * s;
}

__global__ void add_identity_kernel(double *A, int r, double a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < r) A[(size_t)i * r + i] += a;
}

__global__ void chol_shift_from_trace(const double *H, int r, double rel, double *shift_out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < r; ++i) t += H[(size_t)i * r + i];
        *shift_out = rel * t / (r > 0 ? r : 1);
    }
}

__global__ void add_identity_dev_kernel(double *A, int r, const double *a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < r) A[(size_t)i * r + i] += *a;
}

inline unsigned nblk(int64_t count, int per = 256) { return (unsigned)((count + per - 1) / per); }

template <typename T>
double qr_shift_rel() {
    return sizeof(T) == 8 ? 1e-15 : 3e-7;
}

// Scratch of one CholeskyQR2 / the r x r cores.
struct Small {
    double *H, *L1, *L1i, *L2, *L2i, *R, *C, *shift, *scal;
    int *status;
    double *part;
};

template <typename T>
int alloc_small(Arena &a, Small &s, int64_t n, int r, int c_max) {
    size_t rr = (size_t)r * r;
    s.H = a.take<double>(rr);
    s.L1 = a.take<double>(rr);
    s.L1i = a.take<double>(rr);
    s.L2 = a.take<double>(rr);
    s.L2i = a.take<double>(rr);
    s.R = a.take<double>(rr);
    s.C = a.take<double>(rr);
    s.shift = a.take<double>(4);
    s.scal = a.take<double>(8);
    s.status = a.take<int>(16);
    size_t np = std::max(gemm_tn_partials(n, r, std::max(r, c_max)), (size_t)((n + 255) / 256 + 1));
    s.part = a.take<double>(np);
    return LD_OK;
}

// Y (n x r) -> Q (n x r) with Y = Q R; tmp is n x r scratch, Tr is r x r scratch (T).
// R (upper, fp64) is left in s.R when want_R.  Chol statuses go to s.status[k0], [k0+1].
template <typename T>
int cholqr2(const T *Y, T *Q, T *tmp, T *Tr, int64_t n, int r, Small &s, int k0, bool want_R,
            cudaStream_t st) {
    const double rel = qr_shift_rel<T>();
    // pass 1
    LD_TRY(gemm_tn<T>(n, r, r, Y, r, Y, r, s.H, s.part, st));
    chol_shift_from_trace<<<1, 1, 0, st>>>(s.H, r, rel, s.shift);
    add_identity_dev_kernel<<<nblk(r), 256, 0, st>>>(s.H, r, s.shift);
    LD_TRY(dense_chol(s.H, r, 0.0, s.status + k0, st));
    std::swap(s.H, s.L1);
    LD_TRY(dense_trinv_lower(s.L1, s.L1i, r, st));
    LD_TRY(dense_export<T>(s.L1i, Tr, r, 0.0, true, st));  // L1^-T
    LD_TRY(gemm_nn<T>(n, r, r, T(1), Y, r, Tr, r, T(0), tmp, r, st));
    // pass 2
    LD_TRY(gemm_tn<T>(n, r, r, tmp, r, tmp, r, s.H, s.part, st));
    chol_shift_from_trace<<<1, 1, 0, st>>>(s.H, r, rel, s.shift);
    add_identity_dev_kernel<<<nblk(r), 256, 0, st>>>(s.H, r, s.shift);
    LD_TRY(dense_chol(s.H, r, 0.0, s.status + k0 + 1, st));
    std::swap(s.H, s.L2);
    LD_TRY(dense_trinv_lower(s.L2, s.L2i, r, st));
    LD_TRY(dense_export<T>(s.L2i, Tr, r, 0.0, true, st));  // L2^-T
    LD_TRY(gemm_nn<T>(n, r, r, T(1), tmp, r, Tr, r, T(0), Q, r, st));
    if (want_R) {
        // R = (L1 L2)^T
        LD_TRY(dense_gemm(r, r, r, 1.0, s.L1, r, false, s.L2, r, false, 0.0, s.C, r, st));
        LD_TRY(dense_export<double>(s.C, s.R, r, 0.0, true, st));
    }
    return check_launch("cholqr2", 4);
}

template <typename T>
size_t build_bytes(int64_t n, int d, int r, int precision) {
    Arena a;
    a.measuring = true;
    a.take<T>((size_t)n * d);
    a.take<int8_t>((size_t)n * r);
    a.take<T>((size_t)n * r);
    a.take<T>((size_t)n * r);
    a.take<T>((size_t)n * r);
    a.take<T>((size_t)r * r);
    Small s;
    alloc_small<T>(a, s, n, r, r);
    a.take<char>(kz_any_workspace<T>(n, d, r, precision));
    return a.off;
}

template <typename T>
int finish_factor(ld_precond *P, T *G, T *Yscratch, T *Tr, Small &s, double *logD_dev,
                  cudaStream_t st) {
    const int64_t n = P->n;
    const int r = P->r;
    T *Qg = static_cast<T *>(P->Qg);
    if (r > 0) {
        LD_TRY(cholqr2<T>(G, Qg, Yscratch, Tr, n, r, s, 4, true, st));
        LD_CHECK_CUDA(cudaMemcpyAsync(P->RG, s.R, sizeof(double) * r * r,
                                      cudaMemcpyDeviceToDevice, st));
        // core I + R_G R_G^T
        LD_TRY(dense_gemm(r, r, r, 1.0, s.R, r, false, s.R, r, true, 0.0, s.C, r, st));
        add_identity_kernel<<<nblk(r), 256, 0, st>>>(s.C, r, 1.0);
        LD_TRY(dense_chol(s.C, r, 0.0, s.status + 6, st));
        LD_TRY(dense_sumlogdiag(s.C, r, s.scal + 1, st));
        LD_TRY(dense_trinv_lower(s.C, s.L1i, r, st));
        LD_TRY(dense_export<T>(s.L1i, static_cast<T *>(P->CmI), r, -1.0, false, st));
        LD_TRY(dense_export<T>(s.L1i, static_cast<T *>(P->CmIT), r, -1.0, true, st));
        sum_serial_kernel<<<1, 1, 0, st>>>(logD_dev, 1, s.scal + 2, 2.0, s.scal + 1);
        LD_TRY(check_launch("finish_factor", 2));
    } else {
        sum_serial_kernel<<<1, 1, 0, st>>>(logD_dev, 1, s.scal + 2, 0.0, nullptr);
        LD_TRY(check_launch("finish_factor", 1));
    }
    int status[16];
    double ld;
    LD_CHECK_CUDA(cudaMemcpyAsync(status, s.status, sizeof(status), cudaMemcpyDeviceToHost, st));
    LD_CHECK_CUDA(cudaMemcpyAsync(&ld, s.scal + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    LD_CHECK_CUDA(cudaStreamSynchronize(st));
    for (int k = 4; k < 7; ++k) {
        if (status[k] != 0) {
            set_error("preconditioner factor: Cholesky pivot %d <= 0 (stage %d)", status[k], k);
            return LD_ERR_NOT_SPD;
        }
    }
    if (!isfinite(ld)) {
        set_error("preconditioner factor: log det P is not finite");
        return LD_ERR_NOT_SPD;
    }
    P->logdet_P = ld;
    return LD_OK;
}

template <typename T>
int alloc_handle(ld_precond *P) {
    size_t nr = (size_t)P->n * P->r, rr = (size_t)P->r * P->r;
    LD_CHECK_CUDA(cudaMalloc(&P->Qg, std::max<size_t>(1, nr) * sizeof(T)));
    LD_CHECK_CUDA(cudaMalloc(&P->CmI, std::max<size_t>(1, rr) * sizeof(T)));
    LD_CHECK_CUDA(cudaMalloc(&P->CmIT, std::max<size_t>(1, rr) * sizeof(T)));
    LD_CHECK_CUDA(cudaMalloc(&P->dinv_sqrt, std::max<int64_t>(1, P->n) * sizeof(T)));
    LD_CHECK_CUDA(cudaMalloc(&P->D, std::max<int64_t>(1, P->n) * sizeof(double)));
    LD_CHECK_CUDA(cudaMalloc(&P->RG, std::max<size_t>(1, rr) * sizeof(double)));
    return LD_OK;
}

void free_handle(ld_precond *P) {
    if (!P) return;
    cudaFree(P->Qg);
    cudaFree(P->CmI);
    cudaFree(P->CmIT);
    cudaFree(P->dinv_sqrt);
    cudaFree(P->D);
    cudaFree(P->RG);
    delete P;
}

template <typename T>
int build_impl(const double *X, int64_t n, int d, const ld_kernel &kern, int r, int q,
               uint64_t seed, int precision, double const_d, void *ws, size_t ws_bytes, cudaStream_t st,
               ld_precond **out) {
    NvtxRange range("ld: preconditioner build");
    Arena a;
    size_t need = build_bytes<T>(n, d, r, precision);
    LD_TRY(arena_open(a, ws, ws_bytes, need));
    ld_precond *P = new ld_precond();
    P->n = n;
    P->r = r;
    P->precision = precision;
    int st_code = alloc_handle<T>(P);
    if (st_code == LD_OK) {
        st_code = [&]() -> int {
            T *Xs = a.take<T>((size_t)n * d);
            int8_t *Om = a.take<int8_t>((size_t)n * r);
            T *Y = a.take<T>((size_t)n * r);
            T *Qb = a.take<T>((size_t)n * r);
            T *tmp = a.take<T>((size_t)n * r);
            T *Tr = a.take<T>((size_t)r * r);
            Small s;
            alloc_small<T>(a, s, n, r, r);
            if (a.overflow) {
                set_error("internal: workspace carve overflow");
                return LD_ERR_WORKSPACE;
            }
            LD_CHECK_CUDA(cudaMemsetAsync(s.status, 0, 16 * sizeof(int), st));
            LD_TRY(check_points_finite(X, n, d, s.status + 15, st));
            LD_TRY(prep_points<T>(X, n, d, point_scale(kern), Xs, st));
            const double diagM = kern.variance + kern.noise;
            const double floor = std::max(kern.noise, 1e-12 * diagM);
            T *A = tmp;
            if (r > 0) {
                // range finder with subspace iteration (Halko et al. 4.1 / 4.4)
                LD_TRY(rademacher(seed, n, r, 0, Om, st));
                LD_TRY(int8_to<T>(Om, Qb, (int64_t)n * r, st));
                LD_TRY(kz_any<T>(Xs, n, d, kern, Qb, Y, r, precision, a, st));
                for (int it = 0; it < q; ++it) {
                    LD_TRY(cholqr2<T>(Y, Qb, tmp, Tr, n, r, s, 0, false, st));
                    LD_TRY(kz_any<T>(Xs, n, d, kern, Qb, Y, r, precision, a, st));
                }
                LD_TRY(cholqr2<T>(Y, Qb, tmp, Tr, n, r, s, 0, false, st));
                LD_TRY(kz_any<T>(Xs, n, d, kern, Qb, Y, r, precision, a, st));
                // core C = Q^T M Q, A = Q chol(C)  (Halko et al. 5.3 with C factored
                // by Cholesky: A A^T = Q C Q^T, the rank-r approximation of M)
                LD_TRY(gemm_tn<T>(n, r, r, Qb, r, Y, r, s.C, s.part, st));
                LD_TRY(dense_symmetrize(s.C, r, st));
                LD_CHECK_CUDA(cudaMemcpyAsync(s.L2, s.C, sizeof(double) * r * r,
                                              cudaMemcpyDeviceToDevice, st));
                LD_TRY(dense_chol(s.C, r, 0.0, s.status + 2, st));
                int stc = 0;
                LD_CHECK_CUDA(cudaMemcpyAsync(&stc, s.status + 2, sizeof(int),
                                              cudaMemcpyDeviceToHost, st));
                LD_CHECK_CUDA(cudaStreamSynchronize(st));
                if (stc != 0) {  // rounding made C indefinite: shift by a tiny multiple of its trace
                    LD_CHECK_CUDA(cudaMemcpyAsync(s.C, s.L2, sizeof(double) * r * r,
                                                  cudaMemcpyDeviceToDevice, st));
                    chol_shift_from_trace<<<1, 1, 0, st>>>(s.C, r, sizeof(T) == 8 ? 1e-13 : 1e-6,
                                                           s.shift);
                    add_identity_dev_kernel<<<nblk(r), 256, 0, st>>>(s.C, r, s.shift);
                    LD_TRY(check_launch("C shift", 2));
                    LD_TRY(dense_chol(s.C, r, 0.0, s.status + 3, st));
                }
                LD_TRY(dense_export<T>(s.C, Tr, r, 0.0, false, st));
                LD_TRY(gemm_nn<T>(n, r, r, T(1), Qb, r, Tr, r, T(0), A, r, st));
            }
            // D = diag(M) - rowsumsq(A), clamped; sum log D
            unsigned nb = nblk(n);
            diag_resid_kernel<T><<<nb, 256, 0, st>>>(A, n, r, diagM, floor, const_d, P->D,
                                                    static_cast<T *>(P->dinv_sqrt), s.part);
            double *logD = s.scal + 0;
            sum_serial_kernel<<<1, 1, 0, st>>>(s.part, (int)nb, logD, 0.0, nullptr);
            LD_TRY(check_launch("diag_resid", 2));
            if (r > 0) {
                LD_TRY(scale_rows<T>(A, static_cast<T *>(P->dinv_sqrt), A, n, r, st));  // G
                int stv[16];
                LD_CHECK_CUDA(cudaMemcpyAsync(stv, s.status, sizeof(stv), cudaMemcpyDeviceToHost, st));
                LD_CHECK_CUDA(cudaStreamSynchronize(st));
                if (stv[0] || stv[1] || (stv[2] && stv[3])) {
                    set_error("randomized SVD: Cholesky failed (statuses %d %d %d %d)", stv[0],
                              stv[1], stv[2], stv[3]);
                    return LD_ERR_NOT_SPD;
                }
            }
            return finish_factor<T>(P, A, Y, Tr, s, logD, st);
        }();
    }
    arena_close(a);
    if (st_code != LD_OK) {
        free_handle(P);
        return st_code;
    }
    *out = P;
    return LD_OK;
}

template <typename T>
int import_impl(const double *A_host, const double *D_host, int64_t n, int r, int precision,
                cudaStream_t st, ld_precond **out) {
    ld_precond *P = new ld_precond();
    P->n = n;
    P->r = r;
    P->precision = precision;
    Arena a;
    int code = alloc_handle<T>(P);
    if (code == LD_OK) {
        Arena meas;
        meas.measuring = true;
        meas.take<double>((size_t)n * r);
        meas.take<T>((size_t)n * r);
        meas.take<T>((size_t)n * r);
        meas.take<T>((size_t)r * r);
        Small sm;
        alloc_small<T>(meas, sm, n, r, r);
        code = arena_open(a, nullptr, 0, meas.off);
    }
    if (code == LD_OK) {
        code = [&]() -> int {
            double *Ad = a.take<double>((size_t)n * r);
            T *G = a.take<T>((size_t)n * r);
            T *Y = a.take<T>((size_t)n * r);
            T *Tr = a.take<T>((size_t)r * r);
            Small s;
            alloc_small<T>(a, s, n, r, r);
            LD_CHECK_CUDA(cudaMemsetAsync(s.status, 0, 16 * sizeof(int), st));
            if (r > 0)
                LD_CHECK_CUDA(cudaMemcpyAsync(Ad, A_host, sizeof(double) * n * r,
                                              cudaMemcpyHostToDevice, st));
            LD_CHECK_CUDA(cudaMemcpyAsync(P->D, D_host, sizeof(double) * n, cudaMemcpyHostToDevice, st));
            unsigned nb = nblk(n);
            import_kernel<T><<<nb, 256, 0, st>>>(Ad, P->D, n, r, G, static_cast<T *>(P->dinv_sqrt),
                                                 s.part);
            sum_serial_kernel<<<1, 1, 0, st>>>(s.part, (int)nb, s.scal + 0, 0.0, nullptr);
            LD_TRY(check_launch("import", 2));
            return finish_factor<T>(P, G, Y, Tr, s, s.scal + 0, st);
        }();
    }
    arena_close(a);
    if (code != LD_OK) {
        free_handle(P);
        return code;
    }
    *out = P;
    return LD_OK;
}

template <typename T>
__global__ void scale_cols_sqrt_kernel(T *Z, int64_t n, int s, const double *norm2) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * s) return;
    Z[t] = (T)((double)Z[t] * sqrt(norm2[t % s]));
}

}  // namespace

// Normal orthogonal probes (the Appendix's "normal orthogonal" probe type, an
// application of Orthogonal Monte Carlo, Yu et al. 2016): W = S Q with Q a random
// matrix with orthonormal columns and S diagonal with chi_n entries.  Q is the
// orthonormal factor of an n x s block of N(0, 1) draws with R's diagonal
// positive (so its columns are Haar distributed), computed by CholeskyQR2; each
// S entry is the norm of an independent n-vector of N(0, 1) draws, which is chi_n
// distributed by definition.  Every column is then marginally N(0, I_n) and the
// s columns are mutually orthogonal.
size_t orth_probe_tail_bytes(int64_t n, int s) {
    Arena a;
    a.measuring = true;
    a.take<double>((size_t)s * s);      // Tr (as double, the larger type)
    a.take<double>((size_t)s + 64);     // squared norms
    Small sm;
    alloc_small<double>(a, sm, n, s, s);
    a.take<double>(coldot_partials(n, s) + 64);
    return a.off;
}

template <typename T>
int orthogonal_probes(uint64_t seed, int64_t n, int s, int col0, T *Z, T *G, T *H, T *tmp, Arena &a,
                      cudaStream_t st) {
    const size_t mark = a.off;
    T *Tr = a.take<T>((size_t)s * s);
    double *norm2 = a.take<double>((size_t)s + 64);
    Small sm;
    alloc_small<T>(a, sm, n, s, s);
    double *cpart = a.take<double>(coldot_partials(n, s) + 64);
    if (a.overflow || !cpart) {
        a.off = mark;
        set_error("orthogonal probes: workspace too small");
        return LD_ERR_WORKSPACE;
    }
    int code = [&]() -> int {
        LD_CHECK_CUDA(cudaMemsetAsync(sm.status, 0, 16 * sizeof(int), st));
        LD_TRY(gaussian<T>(seed, n, s, ORF_NORM_COL0 + col0, H, st));
        LD_TRY(coldot<T>(n, s, H, H, norm2, cpart, st));
        LD_TRY(gaussian<T>(seed, n, s, col0, G, st));
        LD_TRY(cholqr2<T>(G, Z, tmp, Tr, n, s, sm, 0, false, st));
        scale_cols_sqrt_kernel<T><<<nblk(n * s), 256, 0, st>>>(Z, n, s, norm2);
        LD_TRY(check_launch("orthogonal probes"));
        int stv[2] = {0, 0};
        LD_CHECK_CUDA(cudaMemcpyAsync(stv, sm.status, sizeof(stv), cudaMemcpyDeviceToHost, st));
        LD_CHECK_CUDA(cudaStreamSynchronize(st));
        if (stv[0] || stv[1]) {
            set_error("orthogonal probes: CholeskyQR2 failed (statuses %d %d)", stv[0], stv[1]);
            return LD_ERR_NOT_SPD;
        }
        return LD_OK;
    }();
    a.off = mark;
    return code;
}
template int orthogonal_probes<float>(uint64_t, int64_t, int, int, float *, float *, float *, float *, Arena &,
                                      cudaStream_t);
template int orthogonal_probes<double>(uint64_t, int64_t, int, int, double *, double *, double *, double *,
                                       Arena &, cudaStream_t);

// Apply L^-1 (transpose = false) or L^-T to V (n x c) into W (may alias V).
// Scratch: Td (r x c fp64), Tt and Ut (r x c, T), part (gemm_tn partials).
template <typename T>
int precond_apply_impl(const ld_precond *P, bool transpose, const T *V, T *W, int c, double *Td,
                       T *Tt, T *Ut, double *part, cudaStream_t st) {
    const int64_t n = P->n;
    const int r = P->r;
    const T *Qg = static_cast<const T *>(P->Qg);
    const T *dinv = static_cast<const T *>(P->dinv_sqrt);
    if (!transpose) {
        LD_TRY(scale_rows<T>(V, dinv, W, n, c, st));
        if (r == 0) return LD_OK;
        LD_TRY(gemm_tn<T>(n, r, c, Qg, r, W, c, Td, part, st));
        LD_TRY(convert<double, T>(Td, Tt, (int64_t)r * c, st));
        LD_TRY(gemm_nn<T>(r, c, r, T(1), static_cast<const T *>(P->CmI), r, Tt, c, T(0), Ut, c, st));
        LD_TRY(gemm_nn<T>(n, c, r, T(1), Qg, r, Ut, c, T(1), W, c, st));
    } else {
        if (r > 0) {
            LD_TRY(gemm_tn<T>(n, r, c, Qg, r, V, c, Td, part, st));
            LD_TRY(convert<double, T>(Td, Tt, (int64_t)r * c, st));
            LD_TRY(gemm_nn<T>(r, c, r, T(1), static_cast<const T *>(P->CmIT), r, Tt, c, T(0), Ut, c,
                              st));
            if (W != V)
                LD_CHECK_CUDA(cudaMemcpyAsync(W, V, sizeof(T) * n * c, cudaMemcpyDeviceToDevice, st));
            LD_TRY(gemm_nn<T>(n, c, r, T(1), Qg, r, Ut, c, T(1), W, c, st));
            LD_TRY(scale_rows<T>(W, dinv, W, n, c, st));
        } else {
            LD_TRY(scale_rows<T>(V, dinv, W, n, c, st));
        }
    }
    return LD_OK;
}
template int precond_apply_impl<float>(const ld_precond *, bool, const float *, float *, int,
                                       double *, float *, float *, double *, cudaStream_t);
template int precond_apply_impl<double>(const ld_precond *, bool, const double *, double *, int,
                                        double *, double *, double *, double *, cudaStream_t);

size_t precond_apply_scratch_doubles(const ld_precond *P, int c) {
    if (!P) return 0;
    return (size_t)P->r * c + gemm_tn_partials(P->n, P->r, c) + 64;
}

}  // namespace ld

using namespace ld;

extern "C" {

size_t precond_workspace_size(int64_t n, int32_t d, int32_t rank, int32_t precision) {
    if (precision == LD_FP64) return build_bytes<double>(n, d, rank, precision);
    return build_bytes<float>(n, d, rank, precision);
}

int precond_build(const double *X_dev, int64_t n, int32_t d, ld_kernel kern, int32_t rank,
                  int32_t power_iters, uint64_t seed, int32_t precision, void *ws, size_t ws_bytes,
                  void *stream, ld_precond **out) {
    clear_error();
    LD_REQUIRE(out != nullptr, "precond_build: out is NULL");
    LD_REQUIRE(n > 0 && X_dev, "precond_build: need n > 0 points");
    LD_REQUIRE(d >= 1 && d <= 32, "precond_build: d must be in [1, 32]");
    LD_REQUIRE(d <= 8 || precision == LD_FP64 || precision == LD_FP32,
               "precond_build: tensor-core precisions support d <= 8");
    LD_REQUIRE(rank >= 0 && rank <= 1024 && rank <= n, "precond_build: rank must be in [0, min(n, 1024)]");
    LD_REQUIRE(power_iters >= 0 && power_iters <= 64, "precond_build: power_iters in [0, 64]");
    LD_REQUIRE(kern.lengthscale > 0 && kern.variance > 0 && kern.noise >= 0 &&
                   (kern.kind == LD_RBF || kern.kind == LD_MATERN52),
               "precond_build: bad kernel parameters");
    LD_REQUIRE(precision >= LD_FP64 && precision <= LD_F16X3_TC, "precond_build: bad precision");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == LD_FP64)
        return build_impl<double>(X_dev, n, d, kern, rank, power_iters, seed, precision, 0.0, ws, ws_bytes, st, out);
    return build_impl<float>(X_dev, n, d, kern, rank, power_iters, seed, precision, 0.0, ws, ws_bytes, st, out);
}

int precond_build_scaled(const double *X_dev, int64_t n, int32_t d, ld_kernel kern, int32_t rank,
                         int32_t power_iters, uint64_t seed, double a, int32_t precision, void *ws,
                         size_t ws_bytes, void *stream, ld_precond **out) {
    clear_error();
    LD_REQUIRE(a > 0 && isfinite(a), "precond_build_scaled: a must be > 0");
    LD_REQUIRE(out != nullptr && n > 0 && X_dev && d >= 1 && d <= 32, "precond_build_scaled: bad arguments");
    LD_REQUIRE(d <= 8 || precision == LD_FP64 || precision == LD_FP32,
               "precond_build_scaled: tensor-core precisions support d <= 8");
    LD_REQUIRE(rank >= 0 && rank <= 1024 && rank <= n && power_iters >= 0 && power_iters <= 64,
               "precond_build_scaled: bad rank or power_iters");
    LD_REQUIRE(kern.lengthscale > 0 && kern.variance > 0 && kern.noise >= 0 &&
                   (kern.kind == LD_RBF || kern.kind == LD_MATERN52),
               "precond_build_scaled: bad kernel parameters");
    LD_REQUIRE(precision >= LD_FP64 && precision <= LD_F16X3_TC, "precond_build_scaled: bad precision");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == LD_FP64)
        return build_impl<double>(X_dev, n, d, kern, rank, power_iters, seed, precision, a, ws, ws_bytes, st, out);
    return build_impl<float>(X_dev, n, d, kern, rank, power_iters, seed, precision, a, ws, ws_bytes, st, out);
}

int precond_import(const double *A_host, const double *D_host, int64_t n, int32_t rank,
                   int32_t precision, void *stream, ld_precond **out) {
    clear_error();
    LD_REQUIRE(out && D_host && n > 0 && rank >= 0 && rank <= 1024 && rank <= n &&
                   (rank == 0 || A_host),
               "precond_import: bad arguments");
    LD_REQUIRE(precision >= LD_FP64 && precision <= LD_F16X3_TC, "precond_import: bad precision");
    for (int64_t i = 0; i < n; ++i)
        LD_REQUIRE(D_host[i] > 0 && isfinite(D_host[i]), "precond_import: D[%lld] must be > 0", (long long)i);
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == LD_FP64) return import_impl<double>(A_host, D_host, n, rank, precision, st, out);
    return import_impl<float>(A_host, D_host, n, rank, precision, st, out);
}

int precond_export(const ld_precond *P, double *A_host, double *D_host, double *logdet_P,
                   void *stream) {
    clear_error();
    LD_REQUIRE(P != nullptr, "precond_export: NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = P->n;
    const int r = P->r;
    if (A_host && r > 0) {
        double *Ad = nullptr;
        LD_CHECK_CUDA(cudaMalloc(&Ad, sizeof(double) * n * r));
        if (P->precision == LD_FP64)
            export_A_kernel<double><<<nblk(n * r), 256, 0, st>>>(static_cast<const double *>(P->Qg),
                                                               P->RG, P->D, n, r, Ad);
        else
            export_A_kernel<float><<<nblk(n * r), 256, 0, st>>>(static_cast<const float *>(P->Qg),
                                                              P->RG, P->D, n, r, Ad);
        count_launches(1);
        cudaError_t e = cudaMemcpyAsync(A_host, Ad, sizeof(double) * n * r, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(Ad);
        if (e != cudaSuccess) {
            set_error("precond_export: %s", cudaGetErrorString(e));
            return LD_ERR_CUDA;
        }
    }
    if (D_host) {
        LD_CHECK_CUDA(cudaMemcpyAsync(D_host, P->D, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        LD_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    if (logdet_P) *logdet_P = P->logdet_P;
    return LD_OK;
}

int precond_info(const ld_precond *P, int64_t *n, int32_t *rank, int32_t *precision,
                 double *logdet_P) {
    clear_error();
    LD_REQUIRE(P != nullptr, "precond_info: NULL handle");
    if (n) *n = P->n;
    if (rank) *rank = P->r;
    if (precision) *precision = P->precision;
    if (logdet_P) *logdet_P = P->logdet_P;
    return LD_OK;
}

int precond_apply(const ld_precond *P, int32_t transpose, const void *V_dev, void *W_dev,
                  int32_t c, void *stream) {
    clear_error();
    LD_REQUIRE(P && V_dev && W_dev && c > 0, "precond_apply: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    Arena a;
    size_t elt = P->precision == LD_FP64 ? sizeof(double) : sizeof(float);
    size_t need = precond_apply_scratch_doubles(P, c) * sizeof(double) + 2 * (size_t)P->r * c * elt + 1024;
    LD_TRY(arena_open(a, nullptr, 0, need));
    int code;
    double *Td = a.take<double>((size_t)P->r * c);
    double *part = a.take<double>(gemm_tn_partials(P->n, P->r, c) + 64);
    if (P->precision == LD_FP64) {
        double *Tt = a.take<double>((size_t)P->r * c), *Ut = a.take<double>((size_t)P->r * c);
        code = precond_apply_impl<double>(P, transpose != 0, (const double *)V_dev, (double *)W_dev,
                                          c, Td, Tt, Ut, part, st);
    } else {
        float *Tt = a.take<float>((size_t)P->r * c), *Ut = a.take<float>((size_t)P->r * c);
        code = precond_apply_impl<float>(P, transpose != 0, (const float *)V_dev, (float *)W_dev, c,
                                         Td, Tt, Ut, part, st);
    }
    if (code == LD_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("precond_apply: %s", cudaGetErrorString(e));
            code = LD_ERR_CUDA;
        }
    }
    arena_close(a);
    return code;
}

void precond_free(ld_precond *P) { free_handle(P); }

}  // extern "C"
