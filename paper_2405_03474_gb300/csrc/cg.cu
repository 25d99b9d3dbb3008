// The estimator of Algorithm 1 as a block multi-shift conjugate-gradient solve.
//
// Section 2 reads steps 2-3 of Algorithm 1 as a multi-shift solver (after
// Jegerlehner): one Krylov space per probe serves every shifted system
// (B + sigma_j I) x = z.  Here each block of s probes runs CG on the seed
// system B + sigma_min I (B = L^-1 M L^-T), all columns at once so the O(n^2)
// product K V is shared by the block.  CG coefficients (alpha_k, beta_k) give
// the Lanczos tridiagonal of the seed operator,
//     T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1},  T_k,k+1 = sqrt(beta_k)/alpha_k,
// and the quadratic forms of Algorithm 1 step 3 follow from T alone,
//     q_ij = |z_i|^2 e_1^T (T_i + (sigma_j - sigma_min) I)^-1 e_1,
// computed by eliminating the tridiagonal from the bottom (the Thomas
// algorithm specialised to the first component).  The shifted iterates x_ij
// are also carried (Jegerlehner's zeta recurrences) for the residual check
// and the gradient.  All scalar recurrences run in fp64 on the device.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace ld {

namespace {

struct ColState {
    double rho, znorm2, alpha, alpha_prev, beta, beta_prev;
    double zeta[5], zeta_prev[5], zeta_next[5], alpha_s[5], beta_s[5];
    int active, upd, t, live[5];
    int broke;  // p^T (B + sigma_min) p <= 0 was met: the operator is not positive definite
};

struct Shifts {
    int m;
    double delta[5];  // sigma_j - sigma_min
};

__global__ void cg_init_kernel(ColState *cs, const double *rr, int s, int m) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s) return;
    ColState st;
    st.rho = rr[c];
    st.znorm2 = rr[c];
    st.alpha = 0.0;
    st.alpha_prev = 1.0;
    st.beta = 0.0;
    st.beta_prev = 0.0;
    for (int j = 0; j < 5; ++j) {
        st.zeta[j] = 1.0;
        st.zeta_prev[j] = 1.0;
        st.zeta_next[j] = 1.0;
        st.alpha_s[j] = 0.0;
        st.beta_s[j] = 0.0;
        st.live[j] = j < m ? 1 : 0;
    }
    st.active = rr[c] > 0.0 ? 1 : 0;
    st.broke = 0;
    st.upd = 0;
    st.t = 0;
    cs[c] = st;
}

// alpha_k = rho_k / p_k^T (B + sigma_min) p_k, and the shifted alpha^sigma_k.
__global__ void cg_alpha_kernel(ColState *cs, const double *pBp, int s, Shifts sh,
                                double *hist_a, int max_iters) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s) return;
    ColState &st = cs[c];
    st.upd = 0;
    if (!st.active) {
        st.alpha = 0.0;
        for (int j = 0; j < sh.m; ++j) st.alpha_s[j] = 0.0;
        return;
    }
    double a = st.rho / pBp[c];
    if (!(a > 0.0) || !isfinite(a) || st.t >= max_iters) {  // breakdown or cap: stop this column
        // a column whose residual is already at rounding level may meet p^T B p <= 0 harmlessly
        if (st.t < max_iters && st.rho > 1e-28 * st.znorm2) st.broke = 1;
        st.active = 0;
        st.alpha = 0.0;
        for (int j = 0; j < sh.m; ++j) st.alpha_s[j] = 0.0;
        return;
    }
    st.alpha = a;
    st.upd = 1;
    hist_a[(size_t)st.t * s + c] = a;
    for (int j = 0; j < sh.m; ++j) {
        if (!st.live[j]) {
            st.alpha_s[j] = 0.0;
            continue;
        }
        double den = a * st.beta_prev * (st.zeta_prev[j] - st.zeta[j]) +
                     st.zeta_prev[j] * st.alpha_prev * (1.0 + sh.delta[j] * a);
        double zn = st.zeta[j] * st.zeta_prev[j] * st.alpha_prev / den;
        if (!isfinite(zn) || fabs(zn) < 1e-200) zn = 0.0;
        st.zeta_next[j] = zn;
        st.alpha_s[j] = a * zn / st.zeta[j];
    }
}

// beta_k = rho_{k+1} / rho_k, shifted beta^sigma_k, convergence test.
__global__ void cg_beta_kernel(ColState *cs, const double *rr_new, int s, Shifts sh,
                               double *hist_b, double tol2, int fixed_iters, int *n_active) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < s) {
        ColState &st = cs[c];
        if (st.upd) {
            double rn = rr_new[c];
            double b = rn / st.rho;
            if (!isfinite(b)) b = 0.0;
            st.beta = b;
            hist_b[(size_t)st.t * s + c] = b;
            st.t += 1;
            for (int j = 0; j < sh.m; ++j) {
                if (!st.live[j]) {
                    st.beta_s[j] = 0.0;
                    continue;
                }
                double ratio = st.zeta_next[j] / st.zeta[j];
                st.beta_s[j] = b * ratio * ratio;
                st.zeta_prev[j] = st.zeta[j];
                st.zeta[j] = st.zeta_next[j];
            }
            st.alpha_prev = st.alpha;
            st.beta_prev = b;
            st.rho = rn;
            if (rn <= 0.0) st.active = 0;
            if (fixed_iters == 0 && rn < tol2 * st.znorm2) st.active = 0;
            if (fixed_iters > 0 && st.t >= fixed_iters) st.active = 0;
        }
        if (st.active) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(n_active, cnt);
}

// The CG vector updates are flat passes over n x s blocks (HBM-bound).  Each block
// stages the s columns' coefficients in shared memory once (a frozen shift j or a
// column without an update gets a zero flag), then every thread updates G = 4
// consecutive columns of one row with 16-byte accesses when s % 4 == 0 (else G = 1).
constexpr int CG_UPD_THREADS = 256;

template <typename T>
struct CgCoef {
    T alpha[256], beta[256], zeta[5][256], as[5][256], bs[5][256];
    unsigned char upd[256], live[5][256];
};

template <typename T>
__device__ void cg_load_coef(const ColState *cs, int s, int m, CgCoef<T> &k) {
    for (int c = threadIdx.x; c < s; c += blockDim.x) {
        const ColState &st = cs[c];
        k.upd[c] = (unsigned char)st.upd;
        k.alpha[c] = (T)st.alpha;
        k.beta[c] = (T)st.beta;
        for (int j = 0; j < m; ++j) {
            k.live[j][c] = (unsigned char)st.live[j];
            k.as[j][c] = (T)st.alpha_s[j];
            k.bs[j][c] = (T)st.beta_s[j];
            k.zeta[j][c] = (T)st.zeta[j];
        }
    }
    __syncthreads();
}

template <typename T, int G>
struct Vec;
template <typename T>
struct Vec<T, 1> {
    T v[1];
    __device__ void load(const T *p) { v[0] = *p; }
    __device__ void store(T *p) const { *p = v[0]; }
};
template <>
struct Vec<float, 4> {
    float v[4];
    __device__ void load(const float *p) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ void store(float *p) const { *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]); }
};
template <>
struct Vec<double, 4> {
    double v[4];
    __device__ void load(const double *p) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ void store(double *p) const {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
};

// r -= alpha Bp;  x_j += alpha^sigma_j p_j   (columns with upd only)
template <typename T, int G>
__global__ void __launch_bounds__(CG_UPD_THREADS) cg_update_r_kernel(int64_t n, int s, int m, const ColState *cs,
                                                                      const T *Bp, T *r, const T *ps, T *xs) {
    __shared__ CgCoef<T> k;
    cg_load_coef<T>(cs, s, m, k);
    const int sg = s / G;  // groups of G columns per row
    const int64_t total = n * sg;
    const size_t ns = (size_t)n * s;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = q / sg;
        const int c0 = (int)(q - row * sg) * G;
        const size_t e = (size_t)row * s + c0;
        bool any = false;
#pragma unroll
        for (int g = 0; g < G; ++g) any |= k.upd[c0 + g] != 0;
        if (!any) continue;
        Vec<T, G> rv, bv;
        rv.load(r + e);
        bv.load(Bp + e);
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (k.upd[c0 + g]) rv.v[g] -= k.alpha[c0 + g] * bv.v[g];
        rv.store(r + e);
        if (xs) {
            for (int j = 0; j < m; ++j) {
                Vec<T, G> xv, pv;
                xv.load(xs + j * ns + e);
                pv.load(ps + j * ns + e);
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (k.upd[c0 + g] && k.live[j][c0 + g]) xv.v[g] += k.as[j][c0 + g] * pv.v[g];
                xv.store(xs + j * ns + e);
            }
        }
    }
}

// p = r + beta p;  p_j = zeta_j r + beta^sigma_j p_j
template <typename T, int G>
__global__ void __launch_bounds__(CG_UPD_THREADS) cg_update_p_kernel(int64_t n, int s, int m, const ColState *cs,
                                                                      const T *r, T *p, T *ps) {
    __shared__ CgCoef<T> k;
    cg_load_coef<T>(cs, s, m, k);
    const int sg = s / G;
    const int64_t total = n * sg;
    const size_t ns = (size_t)n * s;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = q / sg;
        const int c0 = (int)(q - row * sg) * G;
        const size_t e = (size_t)row * s + c0;
        bool any = false;
#pragma unroll
        for (int g = 0; g < G; ++g) any |= k.upd[c0 + g] != 0;
        if (!any) continue;
        Vec<T, G> rv, pv;
        rv.load(r + e);
        pv.load(p + e);
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (k.upd[c0 + g]) pv.v[g] = rv.v[g] + k.beta[c0 + g] * pv.v[g];
        pv.store(p + e);
        if (ps) {
            for (int j = 0; j < m; ++j) {
                Vec<T, G> qv;
                qv.load(ps + j * ns + e);
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (k.upd[c0 + g] && k.live[j][c0 + g])
                        qv.v[g] = k.zeta[j][c0 + g] * rv.v[g] + k.bs[j][c0 + g] * qv.v[g];
                qv.store(ps + j * ns + e);
            }
        }
    }
}

// grid of the update kernels: a few waves of 256-thread blocks over the G-column groups
inline unsigned cg_upd_grid(int64_t n, int s, int G) {
    const int64_t groups = n * (s / G);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((groups + CG_UPD_THREADS - 1) / CG_UPD_THREADS, 152 * 16));
}

__global__ void cg_freeze_shifts_kernel(ColState *cs, int s, int m) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s) return;
    for (int j = 0; j < m; ++j)
        if (cs[c].live[j] && cs[c].zeta[j] == 0.0) cs[c].live[j] = 0;
}

// q_cj = |z_c|^2 e_1^T (T_c + delta_j I)^-1 e_1 from the recorded CG coefficients;
// bracket_c = b |z_c|^2 + sum_j c_j q_cj.
__global__ void quadrature_kernel(const ColState *cs, const double *hist_a, const double *hist_b,
                                  int s, RkCoeffs rk, double sigma_min, double *q, double *bracket) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s) return;
    const ColState &st = cs[c];
    const int t = st.t;
    double acc = rk.b * st.znorm2;
    for (int j = 0; j < rk.m; ++j) {
        double delta = rk.sigma[j] - sigma_min;
        double qv = 0.0;
        if (t > 0) {
            // bottom-up elimination: d_{t-1} = T_{t-1,t-1} + delta,
            // d_k = T_kk + delta - T_{k,k+1}^2 / d_{k+1};  e_1^T (T+delta)^-1 e_1 = 1 / d_0
            int k = t - 1;
            double ak = hist_a[(size_t)k * s + c];
            double Tkk = 1.0 / ak + (k > 0 ? hist_b[(size_t)(k - 1) * s + c] / hist_a[(size_t)(k - 1) * s + c] : 0.0);
            double dd = Tkk + delta;
            for (k = t - 2; k >= 0; --k) {
                ak = hist_a[(size_t)k * s + c];
                double bk = hist_b[(size_t)k * s + c];
                Tkk = 1.0 / ak + (k > 0 ? hist_b[(size_t)(k - 1) * s + c] / hist_a[(size_t)(k - 1) * s + c] : 0.0);
                double off2 = bk / (ak * ak);
                dd = Tkk + delta - off2 / dd;
            }
            qv = st.znorm2 / dd;
        }
        q[(size_t)c * rk.m + j] = qv;
        acc += rk.c[j] * qv;
    }
    bracket[c] = acc;
}

// Eigenvalues of a symmetric tridiagonal matrix (diag a[0..m), off-diagonal
// b[0..m-1)) and the first components q of its eigenvectors, by implicit
// symmetric QR steps with the Wilkinson shift (Golub & Van Loan, "Matrix
// Computations", symmetric QR algorithm): each step chases a bulge with Givens
// rotations G = [c -s; s c]; only the first row of the accumulated rotations is
// kept, which is what Gauss quadrature needs (Golub & Welsch).  Arrays are
// overwritten (a -> eigenvalues).  Returns false if it did not converge.
__device__ bool tridiag_eig_first_row(double *a, double *b, double *q, int m) {
    for (int i = 0; i < m; ++i) q[i] = i == 0 ? 1.0 : 0.0;
    int h = m - 1, guard = 0;
    while (h > 0) {
        if (++guard > 60 * m) return false;
        if (fabs(b[h - 1]) <= 1e-15 * (fabs(a[h - 1]) + fabs(a[h]))) {
            b[h - 1] = 0.0;
            --h;
            continue;
        }
        int l = h - 1;
        while (l > 0 && fabs(b[l - 1]) > 1e-15 * (fabs(a[l - 1]) + fabs(a[l]))) --l;
        // Wilkinson shift: eigenvalue of the trailing 2x2 block closer to a[h]
        const double dd = 0.5 * (a[h - 1] - a[h]);
        const double bb = b[h - 1];
        const double mu = a[h] - bb * bb / (dd + copysign(hypot(dd, bb), dd));
        double x = a[l] - mu, y = b[l];
        for (int k = l; k < h; ++k) {
            const double r = hypot(x, y);
            const double c = r > 0.0 ? x / r : 1.0, sn = r > 0.0 ? y / r : 0.0;
            if (k > l) b[k - 1] = r;  // the bulge is absorbed
            const double ap = a[k], aq = a[k + 1], bp = b[k];
            a[k] = c * c * ap + 2.0 * c * sn * bp + sn * sn * aq;
            a[k + 1] = sn * sn * ap - 2.0 * c * sn * bp + c * c * aq;
            b[k] = c * sn * (aq - ap) + (c * c - sn * sn) * bp;
            const double qp = q[k], qq = q[k + 1];
            q[k] = c * qp + sn * qq;
            q[k + 1] = -sn * qp + c * qq;
            if (k + 1 < h) {  // new bulge at (k, k + 2)
                y = sn * b[k + 1];
                b[k + 1] *= c;
                x = b[k];
            }
        }
    }
    return true;
}

// Stochastic Lanczos quadrature (Ubaru, Chen & Saad 2017; the comparison method of
// Section 3) from the same CG coefficients: T_B = T_seed - sigma_min I,
// z^T log(B) z ~ |z|^2 sum_k q_k^2 log(theta_k).  scratch: 3 * max_iters per column.
__global__ void slq_kernel(const ColState *cs, const double *hist_a, const double *hist_b, int s,
                           double sigma_min, int max_iters, double *scratch, double *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s) return;
    const ColState &st = cs[c];
    const int t = st.t;
    double *a = scratch + (size_t)c * 3 * max_iters;
    double *b = a + max_iters;
    double *q = b + max_iters;
    if (t == 0) {
        out[c] = 0.0;
        return;
    }
    for (int k = 0; k < t; ++k) {
        const double ak = hist_a[(size_t)k * s + c];
        a[k] = 1.0 / ak + (k > 0 ? hist_b[(size_t)(k - 1) * s + c] / hist_a[(size_t)(k - 1) * s + c] : 0.0) -
               sigma_min;
        if (k + 1 < t) b[k] = sqrt(hist_b[(size_t)k * s + c]) / ak;
    }
    if (!tridiag_eig_first_row(a, b, q, t)) {
        out[c] = nan("");
        return;
    }
    double acc = 0.0;
    for (int k = 0; k < t; ++k) acc += q[k] * q[k] * log(fmax(a[k], 1e-300));
    out[c] = st.znorm2 * acc;
}

// gather probe block columns [col0, col0+s) of an n x S int8 matrix into T
template <typename T>
__global__ void gather_probes_kernel(const int8_t *P, int64_t n, int S, int col0, int s, T *Z) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * s) return;
    int64_t i = t / s;
    int c = (int)(t % s);
    Z[t] = (T)P[i * S + col0 + c];
}

// Xall[i, c*m + j] = x_j[i, c]
template <typename T>
__global__ void interleave_kernel(int64_t n, int s, int m, const T *xs, T *Xall) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * s * m) return;
    int64_t i = t / ((int64_t)s * m);
    int cj = (int)(t % ((int64_t)s * m));
    int c = cj / m, j = cj % m;
    Xall[t] = xs[(size_t)j * n * s + i * s + c];
}

// R[i, c*m+j] = z[i,c] - BX[i,c*m+j] - sigma_j X[i,c*m+j]
template <typename T>
__global__ void residual_kernel(int64_t n, int s, int m, const T *Z, const T *Xall, T *BX,
                                RkCoeffs rk) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * s * m) return;
    int64_t i = t / ((int64_t)s * m);
    int cj = (int)(t % ((int64_t)s * m));
    int c = cj / m, j = cj % m;
    BX[t] = Z[i * s + c] - BX[t] - (T)rk.sigma[j] * Xall[t];
}

inline unsigned nb(int64_t count, int per = 256) { return (unsigned)((count + per - 1) / per); }

template <typename T>
struct Bufs {
    T *Xs, *Z, *r, *p, *Bp, *y, *w, *xs, *ps;
    int8_t *Zi8;
    double *dots, *part, *hist_a, *hist_b, *q, *bracket, *slq_scratch, *slq;
    ColState *cs;
    int *n_active;
    // precond apply scratch
    double *Td, *ppart;
    T *Tt, *Ut;
    // residual / gradient
    T *Xall, *Y, *W1, *W2;
    double *gdots;
    T *M;  // stored dense M = K + noise I (dense mode), else null
};

// Carve (or measure) the estimator's scratch.
template <typename T>
void carve(Arena &a, Bufs<T> &b, int64_t n, int d, const ld_precond *P, int s, int m,
           int max_iters, int precision, bool vectors, bool extra, bool dense) {
    const size_t ns = (size_t)n * s;
    b.M = dense ? a.take<T>((size_t)n * (size_t)n) : nullptr;
    const int sm = s * m;
    b.Xs = a.take<T>((size_t)n * d);
    b.Zi8 = a.take<int8_t>(ns);
    b.Z = a.take<T>(ns);
    b.r = a.take<T>(ns);
    b.p = a.take<T>(ns);
    b.Bp = a.take<T>(ns);
    b.y = a.take<T>(ns);
    b.w = a.take<T>(ns);
    b.xs = vectors ? a.take<T>(ns * m) : nullptr;
    b.ps = vectors ? a.take<T>(ns * m) : nullptr;
    int cw = extra ? std::max(s, sm) : s;
    b.dots = a.take<double>(4 * (size_t)cw + 64);
    b.part = a.take<double>(std::max(coldot_partials(n, s), coldot_partials(n, cw)) + 64);
    b.hist_a = a.take<double>((size_t)max_iters * s + 1);
    b.hist_b = a.take<double>((size_t)max_iters * s + 1);
    b.q = a.take<double>((size_t)s * 5);
    b.bracket = a.take<double>((size_t)s);
    b.slq_scratch = a.take<double>((size_t)s * 3 * max_iters + 1);
    b.slq = a.take<double>((size_t)s);
    b.cs = a.take<ColState>((size_t)s);
    b.n_active = a.take<int>(4);
    const int r = P ? P->r : 0;
    b.Td = a.take<double>((size_t)r * cw + 1);
    // split-K partials are not monotone in the column count: size for each count used
    size_t pp = gemm_tn_partials(n, r, s);
    if (extra) pp = std::max(pp, gemm_tn_partials(n, r, sm));
    b.ppart = a.take<double>(pp + 64);
    b.Tt = a.take<T>((size_t)r * cw + 1);
    b.Ut = a.take<T>((size_t)r * cw + 1);
    if (extra) {
        b.Xall = a.take<T>(ns * m);
        b.Y = a.take<T>(ns * m);
        b.W1 = a.take<T>(ns * m);
        b.W2 = a.take<T>(ns * m);
        b.gdots = a.take<double>(8 * (size_t)sm + 64);
    } else {
        b.Xall = b.Y = b.W1 = b.W2 = nullptr;
        b.gdots = nullptr;
    }
}

// carve() plus the tail the kernel product takes for itself (it carves from the
// arena's remaining space and gives it back after each call)
template <typename T>
size_t run_bytes(int64_t n, int d, const ld_precond *P, int s, int m, int max_iters, int precision,
                 bool vectors, bool extra, bool dense) {
    Arena meas;
    meas.measuring = true;
    Bufs<T> b;
    carve<T>(meas, b, n, d, P, s, m, max_iters, precision, vectors, extra, dense);
    // the free tail serves the kernel product and, before the CG starts, the
    // orthogonal-probe cores
    size_t tail = orth_probe_tail_bytes(n, s);
    const int cw = extra ? std::max(s, s * m) : s;
    if (!dense) tail = std::max(tail, kz_any_workspace<T>(n, d, cw, precision));
    // the gradient's derivative pass on the tensor cores
    if (extra && std::is_same<T, float>::value && is_tc_precision(precision))
        tail = std::max(tail, kz_dl_tc_workspace(n, d, precision));
    else if (std::is_same<T, float>::value && is_tc_precision(precision))
        tail = std::max(tail, dense_tc_workspace(n, cw, precision));
    meas.take<char>(tail);
    return meas.off;
}

// W = (B + shift) V for a block of c columns.  B = L^-1 (K + noise I) L^-T.
template <typename T>
int apply_B(const ld_precond *P, Bufs<T> &b, const T *Xs, int64_t n, int d, const ld_kernel &k,
            const T *V, T *out, T *tmp1, T *tmp2, int c, double shift, int precision, Arena &a,
            cudaStream_t st) {
    auto product = [&](const T *in, T *o) -> int {
        if (b.M) {
            if constexpr (std::is_same<T, float>::value) {
                if (is_tc_precision(precision)) return dense_tc(b.M, n, in, o, c, precision, a, st);
            }
            return dense_product<T>(b.M, n, in, o, c, st);
        }
        return kz_any<T>(Xs, n, d, k, in, o, c, precision, a, st);
    };
    if (P) {
        LD_TRY(precond_apply_impl<T>(P, true, V, tmp1, c, b.Td, b.Tt, b.Ut, b.ppart, st));
        LD_TRY(product(tmp1, tmp2));
        LD_TRY(precond_apply_impl<T>(P, false, tmp2, out, c, b.Td, b.Tt, b.Ut, b.ppart, st));
    } else {
        LD_TRY(product(V, out));
    }
    if (shift != 0.0) LD_TRY(axpy<T>((int64_t)n * c, (T)shift, V, out, st));
    return LD_OK;
}

struct RunOut {
    std::vector<double> brackets, slq;
    int iters = 0;
    bool converged = true;
    int broke = 0;  // columns whose CG met p^T (B + sigma_min) p <= 0
    double final_rel = 0.0;
    double max_resid[5] = {0, 0, 0, 0, 0};
    double grad[3] = {0, 0, 0};
};

template <typename T>
int run_impl(const double *X, int64_t n, int d, const ld_kernel &kern, const ld_precond *P,
             const ld_options &o, const int8_t *probes, void *ws, size_t ws_bytes, cudaStream_t st,
             bool want_grad, RunOut &out) {
    RkCoeffs rk;
    LD_TRY(rk_coeffs(o.order, rk));
    const int s = o.probes_per_block;
    const int m = rk.m;
    const int nblocks = o.num_probes / s;
    const bool vectors = o.residual_check || want_grad;
    const int max_iters = o.fixed_iters > 0 ? std::min(o.fixed_iters, o.max_iters) : o.max_iters;
    Bufs<T> b;
    Arena a;
    const bool dense = o.dense != 0;
    LD_TRY(arena_open(a, ws, ws_bytes, run_bytes<T>(n, d, P, s, m, max_iters, o.precision, vectors, vectors, dense)));
    int code = [&]() -> int {
        carve<T>(a, b, n, d, P, s, m, max_iters, o.precision, vectors, vectors, dense);
        if (a.overflow) {
            set_error("internal: estimator workspace overflow");
            return LD_ERR_WORKSPACE;
        }
        LD_TRY(check_points_finite(X, n, d, b.n_active, st));
        LD_TRY(prep_points<T>(X, n, d, point_scale(kern), b.Xs, st));
        if (dense) LD_TRY(dense_materialize<T>(b.Xs, n, d, kern, b.M, st));
        const size_t ns = (size_t)n * s;
        const double smin = rk.sigma[0];
        Shifts sh;
        sh.m = m;
        for (int j = 0; j < 5; ++j) sh.delta[j] = j < m ? rk.sigma[j] - smin : 0.0;
        const double tol2 = o.rel_tol * o.rel_tol;
        out.brackets.assign(o.num_probes, 0.0);
        out.slq.assign(o.num_probes, 0.0);
        for (int blk = 0; blk < nblocks; ++blk) {
            // probes (Algorithm 1 step 1)
            if (probes) {
                gather_probes_kernel<T><<<nb(ns), 256, 0, st>>>(probes, n, o.num_probes, blk * s, s, b.Z);
                LD_TRY(check_launch("gather_probes"));
            } else if (o.probe_kind == 1) {
                LD_TRY(gaussian<T>(o.seed, n, s, o.probe_col0 + blk * s, b.Z, st));
            } else if (o.probe_kind == 2) {
                LD_TRY(orthogonal_probes<T>(o.seed, n, s, o.probe_col0 + blk * s, b.Z, b.Bp, b.y, b.w, a, st));
            } else {
                LD_TRY(rademacher(o.seed, n, s, o.probe_col0 + blk * s, b.Zi8, st));
                LD_TRY(int8_to<T>(b.Zi8, b.Z, (int64_t)ns, st));
            }
            LD_CHECK_CUDA(cudaMemcpyAsync(b.r, b.Z, ns * sizeof(T), cudaMemcpyDeviceToDevice, st));
            LD_CHECK_CUDA(cudaMemcpyAsync(b.p, b.Z, ns * sizeof(T), cudaMemcpyDeviceToDevice, st));
            if (vectors) {
                LD_CHECK_CUDA(cudaMemsetAsync(b.xs, 0, ns * m * sizeof(T), st));
                for (int j = 0; j < m; ++j)
                    LD_CHECK_CUDA(cudaMemcpyAsync(b.ps + j * ns, b.Z, ns * sizeof(T),
                                                  cudaMemcpyDeviceToDevice, st));
            }
            LD_TRY(coldot<T>(n, s, b.r, b.r, b.dots, b.part, st));
            cg_init_kernel<<<nb(s, 128), 128, 0, st>>>(b.cs, b.dots, s, m);
            LD_TRY(check_launch("cg_init"));
            int it = 0;
            for (; it < max_iters; ++it) {
                NvtxRange range("ld: CG iteration");
                // Bp = (B + sigma_min I) p   (the O(n^2) step)
                LD_TRY(apply_B<T>(P, b, b.Xs, n, d, kern, b.p, b.Bp, b.y, b.w, s, smin, o.precision, a, st));
                LD_TRY(coldot<T>(n, s, b.p, b.Bp, b.dots, b.part, st));
                cg_alpha_kernel<<<nb(s, 128), 128, 0, st>>>(b.cs, b.dots, s, sh, b.hist_a, max_iters);
                if (s % 4 == 0)
                    cg_update_r_kernel<T, 4><<<cg_upd_grid(n, s, 4), CG_UPD_THREADS, 0, st>>>(n, s, m, b.cs, b.Bp, b.r,
                                                                                             b.ps, b.xs);
                else
                    cg_update_r_kernel<T, 1><<<cg_upd_grid(n, s, 1), CG_UPD_THREADS, 0, st>>>(n, s, m, b.cs, b.Bp, b.r,
                                                                                             b.ps, b.xs);
                LD_TRY(coldot<T>(n, s, b.r, b.r, b.dots + s, b.part, st));
                LD_CHECK_CUDA(cudaMemsetAsync(b.n_active, 0, sizeof(int), st));
                cg_beta_kernel<<<nb(s, 128), 128, 0, st>>>(b.cs, b.dots + s, s, sh, b.hist_b, tol2,
                                                          o.fixed_iters, b.n_active);
                if (s % 4 == 0)
                    cg_update_p_kernel<T, 4><<<cg_upd_grid(n, s, 4), CG_UPD_THREADS, 0, st>>>(n, s, m, b.cs, b.r, b.p,
                                                                                             b.ps);
                else
                    cg_update_p_kernel<T, 1><<<cg_upd_grid(n, s, 1), CG_UPD_THREADS, 0, st>>>(n, s, m, b.cs, b.r, b.p,
                                                                                             b.ps);
                cg_freeze_shifts_kernel<<<nb(s, 128), 128, 0, st>>>(b.cs, s, m);
                LD_TRY(check_launch("cg iteration", 5));
                int n_active = 0;
                LD_CHECK_CUDA(cudaMemcpyAsync(&n_active, b.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
                LD_CHECK_CUDA(cudaStreamSynchronize(st));
                if (n_active == 0) {
                    ++it;
                    break;
                }
            }
            out.iters = std::max(out.iters, it);
            quadrature_kernel<<<nb(s, 128), 128, 0, st>>>(b.cs, b.hist_a, b.hist_b, s, rk, smin, b.q,
                                                         b.bracket);
            LD_TRY(check_launch("quadrature"));
            slq_kernel<<<nb(s, 64), 64, 0, st>>>(b.cs, b.hist_a, b.hist_b, s, smin, max_iters, b.slq_scratch, b.slq);
            LD_TRY(check_launch("slq"));
            std::vector<ColState> cs(s);
            LD_CHECK_CUDA(cudaMemcpyAsync(out.brackets.data() + (size_t)blk * s, b.bracket,
                                          sizeof(double) * s, cudaMemcpyDeviceToHost, st));
            LD_CHECK_CUDA(cudaMemcpyAsync(out.slq.data() + (size_t)blk * s, b.slq, sizeof(double) * s,
                                          cudaMemcpyDeviceToHost, st));
            LD_CHECK_CUDA(cudaMemcpyAsync(cs.data(), b.cs, sizeof(ColState) * s, cudaMemcpyDeviceToHost, st));
            LD_CHECK_CUDA(cudaStreamSynchronize(st));
            for (int c = 0; c < s; ++c) {
                double rel = cs[c].znorm2 > 0 ? sqrt(std::max(cs[c].rho, 0.0) / cs[c].znorm2) : 0.0;
                out.final_rel = std::max(out.final_rel, rel);
                if (o.fixed_iters == 0 && !(cs[c].rho < tol2 * cs[c].znorm2) && cs[c].rho > 0)
                    out.converged = false;
                out.broke += cs[c].broke;
            }
            if (!vectors) continue;
            const int sm = s * m;
            const size_t nsm = ns * m;
            interleave_kernel<T><<<nb(nsm), 256, 0, st>>>(n, s, m, b.xs, b.Xall);
            LD_TRY(check_launch("interleave"));
            if (o.residual_check) {
                NvtxRange range("ld: residual check");
                // ||z - (B + sigma_j) x_j|| / ||z||, one extra pass over all s*m columns
                LD_TRY(apply_B<T>(P, b, b.Xs, n, d, kern, b.Xall, b.W1, b.Y, b.W2, sm, 0.0, o.precision, a, st));
                residual_kernel<T><<<nb(nsm), 256, 0, st>>>(n, s, m, b.Z, b.Xall, b.W1, rk);
                LD_TRY(check_launch("residual"));
                LD_TRY(coldot<T>(n, sm, b.W1, b.W1, b.gdots, b.part, st));
                std::vector<double> rn(sm);
                LD_CHECK_CUDA(cudaMemcpyAsync(rn.data(), b.gdots, sizeof(double) * sm, cudaMemcpyDeviceToHost, st));
                LD_CHECK_CUDA(cudaStreamSynchronize(st));
                for (int c = 0; c < s; ++c)
                    for (int j = 0; j < m; ++j)
                        out.max_resid[j] = std::max(out.max_resid[j], sqrt(rn[c * m + j] / cs[c].znorm2));
            }
            if (want_grad) {
                NvtxRange range("ld: adjoint");
                // y = L^-T x;  dest/dtheta = (1/s) sum (-c_j) y^T dM y
                if (P) {
                    LD_TRY(precond_apply_impl<T>(P, true, b.Xall, b.Y, sm, b.Td, b.Tt, b.Ut, b.ppart, st));
                } else {
                    LD_CHECK_CUDA(cudaMemcpyAsync(b.Y, b.Xall, nsm * sizeof(T), cudaMemcpyDeviceToDevice, st));
                }
                bool dl_done = false;
                if constexpr (std::is_same<T, float>::value) {
                    if (is_tc_precision(o.precision)) {
                        LD_TRY(kz_dl_tc(b.Xs, n, d, kern.kind, kern.lengthscale, kern.variance, b.Y, b.W1, b.W2,
                                        sm, o.precision, a, st));
                        dl_done = true;
                    }
                }
                if (!dl_done)
                    LD_TRY(kz_dl_simt<T>(b.Xs, n, d, kern.kind, kern.lengthscale, kern.variance, b.Y, b.W1,
                                         b.W2, sm, st));
                LD_TRY(coldot<T>(n, sm, b.Y, b.W2, b.gdots, b.part, st));
                LD_TRY(coldot<T>(n, sm, b.Y, b.W1, b.gdots + sm, b.part, st));
                LD_TRY(coldot<T>(n, sm, b.Y, b.Y, b.gdots + 2 * sm, b.part, st));
                std::vector<double> g(3 * sm);
                LD_CHECK_CUDA(cudaMemcpyAsync(g.data(), b.gdots, sizeof(double) * 3 * sm, cudaMemcpyDeviceToHost, st));
                LD_CHECK_CUDA(cudaStreamSynchronize(st));
                for (int c = 0; c < s; ++c)
                    for (int j = 0; j < m; ++j) {
                        double w = -rk.c[j] / o.num_probes;
                        out.grad[0] += w * g[c * m + j];
                        out.grad[1] += w * g[sm + c * m + j] / kern.variance;
                        out.grad[2] += w * g[2 * sm + c * m + j];
                    }
            }
        }
        return LD_OK;
    }();
    arena_close(a);
    return code;
}

int validate(const double *X, int64_t n, int d, const ld_kernel &k, const ld_precond *P,
             const ld_options *o, bool grad) {
    LD_REQUIRE(o != nullptr, "options are NULL");
    LD_REQUIRE(X != nullptr && n > 0, "need n > 0 points");
    LD_REQUIRE(d >= 1 && d <= 32, "d must be in [1, 32]");
    LD_REQUIRE(d <= 8 || o->precision == LD_FP64 || o->precision == LD_FP32 || o->dense,
               "tensor-core precisions support d <= 8");
    LD_REQUIRE(k.lengthscale > 0 && k.variance > 0 && k.noise >= 0 &&
                   (k.kind == LD_RBF || k.kind == LD_MATERN52),
               "bad kernel parameters");
    LD_REQUIRE(o->order == 1 || o->order == 3 || o->order == 5, "order must be 1, 3 or 5");
    LD_REQUIRE(o->probes_per_block >= 1 && o->probes_per_block <= 256,
               "probes_per_block must be in [1, 256]");
    LD_REQUIRE(o->num_probes >= o->probes_per_block && o->num_probes % o->probes_per_block == 0,
               "num_probes must be a positive multiple of probes_per_block");
    LD_REQUIRE(o->max_iters >= 1 && o->max_iters <= 100000, "max_iters must be in [1, 100000]");
    LD_REQUIRE(o->fixed_iters >= 0, "fixed_iters must be >= 0");
    LD_REQUIRE(o->fixed_iters > 0 || o->rel_tol > 0, "rel_tol must be > 0 without fixed_iters");
    LD_REQUIRE(o->precision >= LD_FP64 && o->precision <= LD_F16X3_TC, "bad precision");
    LD_REQUIRE(o->dense == 0 || o->dense == 1, "dense must be 0 or 1");
    LD_REQUIRE(o->probe_kind >= 0 && o->probe_kind <= 2,
               "probe_kind must be 0 (Rademacher), 1 (Gaussian) or 2 (normal orthogonal)");
    LD_REQUIRE(o->probe_col0 >= 0 && (int64_t)o->probe_col0 + o->num_probes < ORF_NORM_COL0,
               "probe_col0 must be >= 0 with probe_col0 + num_probes < 2^30");
    LD_REQUIRE(o->probe_kind != 2 || o->probes_per_block <= n, "orthogonal probes need probes_per_block <= n");
    LD_REQUIRE(o->dense == 0 || n <= (int64_t)1 << 18, "dense mode keeps n*n words: n <= 262144");
    if (P) {
        LD_REQUIRE(P->n == n, "preconditioner built for n = %lld, not %lld", (long long)P->n, (long long)n);
        LD_REQUIRE((P->precision == LD_FP64) == (o->precision == LD_FP64),
                   "preconditioner and estimate must both be FP64 or both be non-FP64");
    }
    return LD_OK;
}

// Algorithm 1's output: log det P + the Hutchinson mean of the per-probe brackets
// (summed in index order), and the standard error of that mean.
void combine_brackets(const double *br, int S, double ldP, ld_result *out) {
    double mean = 0.0;
    for (int i = 0; i < S; ++i) mean += br[i];
    mean /= S;
    double var = 0.0;
    for (int i = 0; i < S; ++i) var += (br[i] - mean) * (br[i] - mean);
    var = S > 1 ? var / (S - 1) : 0.0;
    out->logdet = ldP + mean;
    out->logdet_P = ldP;
    out->trace_est = mean;
    out->std_err = sqrt(var / S);
}

void fill_result(const RunOut &r, const ld_precond *P, const ld_options &o, ld_result *out,
                 double *per_probe) {
    const int S = (int)r.brackets.size();
    const double ldP = P ? P->logdet_P : 0.0;
    combine_brackets(r.brackets.data(), S, ldP, out);
    out->iters = r.iters;
    out->converged = r.converged ? 1 : 0;
    for (int j = 0; j < 5; ++j) out->max_resid[j] = r.max_resid[j];
    out->final_rel_resid = r.final_rel;
    double slq = 0.0;
    for (double v : r.slq) slq += v;
    out->slq_logdet = ldP + slq / S;
    if (per_probe)
        for (int i = 0; i < S; ++i) per_probe[i] = r.brackets[i];
    (void)o;
}

}  // namespace

}  // namespace ld

using namespace ld;

extern "C" {

size_t logdet_workspace_size(int64_t n, int32_t d, const ld_precond *P, const ld_options *opt) {
    if (!opt) return 0;
    RkCoeffs rk;
    if (rk_coeffs(opt->order, rk) != LD_OK) return 0;
    const int max_iters = opt->fixed_iters > 0 ? std::min(opt->fixed_iters, opt->max_iters) : opt->max_iters;
    const bool vectors = true;  // enough for residual check and gradient
    if (opt->precision == LD_FP64)
        return run_bytes<double>(n, d, P, opt->probes_per_block, rk.m, max_iters, opt->precision, vectors, vectors,
                                 opt->dense != 0);
    return run_bytes<float>(n, d, P, opt->probes_per_block, rk.m, max_iters, opt->precision, vectors, vectors,
                            opt->dense != 0);
}

int logdet_estimate(const double *X_dev, int64_t n, int32_t d, ld_kernel kern, const ld_precond *P,
                    const ld_options *opt, const int8_t *probes_dev, double *per_probe_host,
                    void *ws, size_t ws_bytes, void *stream, ld_result *out) {
    clear_error();
    LD_REQUIRE(out != nullptr, "logdet_estimate: out is NULL");
    LD_TRY(validate(X_dev, n, d, kern, P, opt, false));
    LD_REQUIRE(!(probes_dev && opt->probe_kind != 0),
               "Gaussian and orthogonal probes are drawn on the device (probes_dev = NULL)");
    RunOut r;
    cudaStream_t st = (cudaStream_t)stream;
    int code = opt->precision == LD_FP64
                   ? run_impl<double>(X_dev, n, d, kern, P, *opt, probes_dev, ws, ws_bytes, st, false, r)
                   : run_impl<float>(X_dev, n, d, kern, P, *opt, probes_dev, ws, ws_bytes, st, false, r);
    if (code != LD_OK) return code;
    fill_result(r, P, *opt, out, per_probe_host);
    if (!isfinite(out->logdet)) {
        // NaN / Inf guard: a non-finite point or parameter, or an operator that is not SPD
        set_error("non-finite estimate (logdet_P %g, trace %g): the points or kernel parameters do not give a "
                  "finite SPD matrix", out->logdet_P, out->trace_est);
        return LD_ERR_NOT_SPD;
    }
    if (r.broke) {
        set_error("CG breakdown in %d column(s): p^T (B + sigma) p <= 0, the operator in this precision is not "
                  "positive definite (the rounding of K exceeds the noise; use a wider precision)", r.broke);
        return LD_ERR_NOT_SPD;
    }
    if (!r.converged) {
        set_error("CG did not reach rel_tol %.3g in %d iterations (final %.3g)", opt->rel_tol,
                  opt->max_iters, r.final_rel);
        return LD_ERR_NOT_CONVERGED;
    }
    return LD_OK;
}

int ld_combine(const double *brackets_host, int32_t num_probes, double logdet_P, ld_result *out) {
    clear_error();
    LD_REQUIRE(brackets_host != nullptr && out != nullptr, "ld_combine: NULL pointer");
    LD_REQUIRE(num_probes >= 1, "ld_combine: need at least one probe");
    *out = ld_result{};
    combine_brackets(brackets_host, num_probes, logdet_P, out);
    return LD_OK;
}

int logdet_grad(const double *X_dev, int64_t n, int32_t d, ld_kernel kern, const ld_precond *P,
                const ld_options *opt, const int8_t *probes_dev, void *ws, size_t ws_bytes,
                void *stream, double *grad_host, ld_result *out) {
    clear_error();
    LD_REQUIRE(out != nullptr && grad_host != nullptr, "logdet_grad: out/grad are NULL");
    LD_TRY(validate(X_dev, n, d, kern, P, opt, true));
    RunOut r;
    cudaStream_t st = (cudaStream_t)stream;
    int code = opt->precision == LD_FP64
                   ? run_impl<double>(X_dev, n, d, kern, P, *opt, probes_dev, ws, ws_bytes, st, true, r)
                   : run_impl<float>(X_dev, n, d, kern, P, *opt, probes_dev, ws, ws_bytes, st, true, r);
    if (code != LD_OK) return code;
    fill_result(r, P, *opt, out, nullptr);
    for (int a = 0; a < 3; ++a) grad_host[a] = r.grad[a];
    if (!isfinite(out->logdet) || !isfinite(r.grad[0]) || !isfinite(r.grad[1]) || !isfinite(r.grad[2])) {
        set_error("non-finite estimate or gradient: the points or kernel parameters do not give a finite SPD "
                  "matrix");
        return LD_ERR_NOT_SPD;
    }
    if (r.broke) {
        set_error("CG breakdown in %d column(s): p^T (B + sigma) p <= 0, the operator in this precision is not "
                  "positive definite", r.broke);
        return LD_ERR_NOT_SPD;
    }
    if (!r.converged) {
        set_error("CG did not reach rel_tol %.3g in %d iterations", opt->rel_tol, opt->max_iters);
        return LD_ERR_NOT_CONVERGED;
    }
    return LD_OK;
}

}  // extern "C"
