// Error state, workspace arena, status strings and the r_k coefficients.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace ld {

static thread_local char g_err[512] = {0};

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char *last_error() { return g_err; }
void clear_error() { g_err[0] = 0; }

int arena_open(Arena &a, void *ws, size_t ws_bytes, size_t need) {
    a.off = 0;
    a.overflow = false;
    a.measuring = false;
    if (ws) {
        if (ws_bytes < need) {
            set_error("workspace too small: %zu bytes given, %zu needed", ws_bytes, need);
            return LD_ERR_WORKSPACE;
        }
        if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
            set_error("workspace must be 256-byte aligned");
            return LD_ERR_INVALID;
        }
        a.base = static_cast<char *>(ws);
        a.cap = ws_bytes;
        a.owned = false;
        return LD_OK;
    }
    a.cap = need;
    a.owned = true;
    if (need == 0) {
        a.base = nullptr;
        return LD_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu) for workspace failed: %s", need, cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    a.base = static_cast<char *>(p);
    return LD_OK;
}

void arena_close(Arena &a) {
    if (a.owned && a.base) cudaFree(a.base);
    a.base = nullptr;
    a.owned = false;
}

// r_k of Eq. 1 as N(z)/D(z); its partial fractions (Table 1) from the closed-form
// roots of D:  r_1: D = z + 1.  r_3: D = (z + 1)(z^2 + 14 z + 1), roots -1 and
// -7 +- 4 sqrt 3.  r_5: D = (z + 1)(z^4 + 44 z^3 + 166 z^2 + 44 z + 1); the quartic
// is palindromic, so w = z + 1/z solves w^2 + 44 w + 164 = 0, w = -22 +- 8 sqrt 5,
// and z solves z^2 - w z + 1 = 0 (product of the two roots is 1).
// Residues c_j = N(-sigma_j) / D'(-sigma_j), evaluated in long double.
int rk_coeffs(int order, RkCoeffs &out) {
    typedef long double Ld;
    const Ld n1[] = {2, -2}, d1[] = {1, 1};
    const Ld n3[] = {14, 54, -54, -14}, d3[] = {3, 45, 45, 3};  // (2/3)(..)/(..) scaled by 3
    const Ld n5[] = {86, 1650, 2300, -2300, -1650, -86};
    const Ld d5[] = {15, 675, 3150, 3150, 675, 15};              // (2/15)(..)/(..) scaled by 15
    const Ld *N, *Dn;
    Ld roots[5];
    int m;
    if (order == 1) {
        N = n1; Dn = d1; m = 1;
        roots[0] = -1;
    } else if (order == 3) {
        N = n3; Dn = d3; m = 3;
        Ld s3 = sqrtl((Ld)3);
        roots[0] = -7 + 4 * s3;
        roots[1] = -1;
        roots[2] = -7 - 4 * s3;
        // -7 + 4 sqrt 3 loses digits to cancellation: use the reciprocal of its partner
        roots[0] = 1 / roots[2];
    } else if (order == 5) {
        N = n5; Dn = d5; m = 5;
        Ld s5 = sqrtl((Ld)5);
        Ld w[2] = {-22 + 8 * s5, -22 - 8 * s5};
        Ld zs[4];
        for (int a = 0; a < 2; ++a) {
            Ld big = (w[a] - sqrtl(w[a] * w[a] - 4)) / 2;  // no cancellation, w < 0
            zs[2 * a] = big;
            zs[2 * a + 1] = 1 / big;
        }
        roots[0] = zs[0]; roots[1] = zs[1]; roots[2] = -1; roots[3] = zs[2]; roots[4] = zs[3];
    } else {
        set_error("order must be 1, 3 or 5 (got %d)", order);
        return LD_ERR_INVALID;
    }
    // sort by increasing sigma = -root
    std::sort(roots, roots + m, [](Ld a, Ld b) { return a > b; });
    out.m = m;
    out.b = (double)(N[0] / Dn[0]);
    for (int j = 0; j < m; ++j) {
        Ld x = roots[j];
        Ld nv = 0, dv = 0;
        for (int i = 0; i <= m; ++i) nv = nv * x + N[i];
        for (int i = 0; i < m; ++i) dv = dv * x + Dn[i] * (Ld)(m - i);
        out.sigma[j] = (double)(-x);
        out.c[j] = (double)(nv / dv);
    }
    return LD_OK;
}

double point_scale(const ld_kernel &k) {
    if (k.kind == LD_RBF) return 1.0 / (k.lengthscale * sqrt(2.0));
    return sqrt(5.0) / k.lengthscale;
}

}  // namespace ld

extern "C" {

const char *ld_status_string(int status) {
    switch (status) {
        case LD_OK: return "ok";
        case LD_ERR_INVALID: return "invalid argument";
        case LD_ERR_NOT_SPD: return "matrix not positive definite";
        case LD_ERR_NOT_CONVERGED: return "not converged";
        case LD_ERR_CUDA: return "CUDA error";
        case LD_ERR_WORKSPACE: return "workspace too small";
        case LD_ERR_UNSUPPORTED: return "unsupported option";
        case LD_ERR_DEVICE_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char *ld_last_error(void) { return ld::last_error(); }

int ld_version(void) { return 1; }

int ld_rk_coeffs(int32_t order, double *b, double *c, double *sigma) {
    ld::RkCoeffs rk;
    int st = ld::rk_coeffs(order, rk);
    if (st != LD_OK) return st;
    if (b) *b = rk.b;
    for (int j = 0; j < rk.m; ++j) {
        if (c) c[j] = rk.c[j];
        if (sigma) sigma[j] = rk.sigma[j];
    }
    return LD_OK;
}

}  // extern "C"
