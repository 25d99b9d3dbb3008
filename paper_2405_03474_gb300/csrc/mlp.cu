// Surrogate MLP for log det over kernel hyperparameters (an addition to the
// paper's method, for hyperparameter search): 4 -> 128 -> 128 -> 128 -> 1,
// exact GELU (x Phi(x)) after each hidden layer, fp32, trained by Adam on the
// mean squared error of values the estimator produced.
//
// Parameters are one flat vector (33793 floats): W1 (128x4), b1, W2 (128x128),
// b2, W3 (128x128), b3, W4 (1x128), b4; each W row-major (out, in).  The handle
// also holds an affine normalisation of inputs and target (identity after
// create; surrogate_train sets it from its training data): the network sees
// (theta - mu) / sd and predicts (y - ymu) / ysd.
//
// Kernels are plain SIMT: one thread per output of a layer (forward, input
// backward) or per weight (weight gradient, summed over the batch in a fixed
// order).  The work is tiny next to one estimate (65536 queries: 4.4 GFLOP).
#include <math.h>

#include <vector>

#include "common.cuh"

namespace {

constexpr int L0 = 4, L1 = 128, L2 = 128, L3 = 128, L4 = 1;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + L1 * L0, OFF_W2 = OFF_B1 + L1, OFF_B2 = OFF_W2 + L2 * L1,
              OFF_W3 = OFF_B2 + L2, OFF_B3 = OFF_W3 + L3 * L2, OFF_W4 = OFF_B3 + L3,
              OFF_B4 = OFF_W4 + L4 * L3, NPARAM = OFF_B4 + L4;
static_assert(NPARAM == 33793, "parameter count");

struct Layer {
    int in, out, w, b;
};
constexpr Layer LAYERS[4] = {{L0, L1, OFF_W1, OFF_B1}, {L1, L2, OFF_W2, OFF_B2}, {L2, L3, OFF_W3, OFF_B3},
                             {L3, L4, OFF_W4, OFF_B4}};

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

// z[s, o] = sum_i in[s, i] W[o, i] + b[o];  h = gelu(z) when act
__global__ void fwd_kernel(const float *in, int B, int I, int O, const float *W, const float *b, float *z,
                           float *h, int act) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)B * O) return;
    const int s = (int)(t / O), o = (int)(t % O);
    const float *x = in + (size_t)s * I;
    const float *w = W + (size_t)o * I;
    float acc = b[o];
    for (int i = 0; i < I; ++i) acc = fmaf(x[i], w[i], acc);
    z[t] = acc;
    if (h) h[t] = act ? gelu(acc) : acc;
}

// normalised input: xn = (theta - mu) / sd
__global__ void norm_in_kernel(const float *theta, int B, const float *mu, const float *sd, float *xn) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * L0) return;
    const int a = t % L0;
    xn[t] = (theta[t] - mu[a]) / sd[a];
}

// dz4[s] = (2/N) (pred[s] - (y[s] - ymu)/ysd); loss partial per block (fp64)
__global__ void loss_kernel(const float *pred, const float *y, int B, int Ntot, const float *ymu,
                            const float *ysd, float *dz, double *part) {
    __shared__ double red[32];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (s < B) {
        const float r = pred[s] - (y[s] - ymu[0]) / ysd[0];
        dz[s] = 2.0f * r / (float)Ntot;
        l = (double)r * r;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void fill_kernel(float *p, int n, float v) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) p[t] = v;
}

// din[s, i] = sum_o dz[s, o] W[o, i];  if zprev: din *= gelu'(zprev[s, i])
__global__ void bwd_in_kernel(const float *dz, int B, int I, int O, const float *W, const float *zprev,
                              float *din) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)B * I) return;
    const int s = (int)(t / I), i = (int)(t % I);
    const float *g = dz + (size_t)s * O;
    float acc = 0.f;
    for (int o = 0; o < O; ++o) acc = fmaf(g[o], W[(size_t)o * I + i], acc);
    din[t] = zprev ? acc * gelu_grad(zprev[t]) : acc;
}

// dW[o, i] = sum_s dz[s, o] in[s, i];  db[o] = sum_s dz[s, o]   (fixed order)
__global__ void bwd_w_kernel(const float *dz, const float *in, int B, int I, int O, float *dW, float *db) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= O * (I + 1)) return;
    const int o = t / (I + 1), i = t % (I + 1);
    double acc = 0.0;
    if (i < I) {
        for (int s = 0; s < B; ++s) acc += (double)dz[(size_t)s * O + o] * in[(size_t)s * I + i];
        dW[(size_t)o * I + i] = (float)acc;
    } else {
        for (int s = 0; s < B; ++s) acc += dz[(size_t)s * O + o];
        db[o] = (float)acc;
    }
}

// Adam (Kingma & Ba): m, v moments, bias-corrected step
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

// mean and std over rows of a (B x c) block, fp64 sums, one block per column
__global__ void moments_kernel(const float *a, int B, int c, float *mu, float *sd) {
    __shared__ double s1[256], s2[256];
    const int col = blockIdx.x;
    double x1 = 0.0, x2 = 0.0;
    for (int s = threadIdx.x; s < B; s += blockDim.x) {
        const double v = a[(size_t)s * c + col];
        x1 += v;
        x2 += v * v;
    }
    s1[threadIdx.x] = x1;
    s2[threadIdx.x] = x2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            t1 += s1[k];
            t2 += s2[k];
        }
        const double m = t1 / B;
        const double var = fmax(t2 / B - m * m, 0.0);
        const double sdv = sqrt(var);
        mu[col] = (float)m;
        sd[col] = sdv > 1e-12 * fmax(1.0, fabs(m)) ? (float)sdv : 1.0f;  // constant input: no scaling
    }
}

// Glorot-uniform weights from SplitMix64 (counter = parameter index), zero biases
__device__ __forceinline__ uint64_t mix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void init_kernel(float *p, uint64_t seed) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NPARAM) return;
    // layer of parameter t: (fan_in + fan_out, first bias index)
    int fans, bias0;
    if (t < OFF_W2) { fans = L0 + L1; bias0 = OFF_B1; }
    else if (t < OFF_W3) { fans = L1 + L2; bias0 = OFF_B2; }
    else if (t < OFF_W4) { fans = L2 + L3; bias0 = OFF_B3; }
    else { fans = L3 + L4; bias0 = OFF_B4; }
    if (t >= bias0) {
        p[t] = 0.f;
        return;
    }
    const float a = sqrtf(6.0f / (float)fans);
    const double u = (double)(mix64(seed, (uint64_t)t) >> 11) * (1.0 / 9007199254740992.0);  // [0,1)
    p[t] = (float)((2.0 * u - 1.0) * a);
}

// out = pred * ysd + ymu;  dout[s, a] = dnet/dxn[s, a] * ysd / sd[a]
__global__ void denorm_kernel(const float *pred, const float *dxn, int B, const float *sd, const float *ymu,
                              const float *ysd, float *out, float *dout) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < B) out[t] = pred[t] * ysd[0] + ymu[0];
    if (dout && t < B * L0) dout[t] = dxn[t] * ysd[0] / sd[t % L0];
}

inline unsigned nb(int64_t n, int per = 256) { return (unsigned)((n + per - 1) / per); }

}  // namespace

struct ld_surrogate {
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    float *norm = nullptr;  // mu[4], sd[4], ymu, ysd
    int step = 0;
};

namespace {

// per-batch scratch for a forward/backward pass over B rows
struct Scratch {
    float *xn, *z[4], *h[3], *dz[4], *dxn;
    double *part;
};

int alloc_scratch(ld::Arena &a, Scratch &s, int B) {
    s.xn = a.take<float>((size_t)B * L0);
    for (int l = 0; l < 4; ++l) s.z[l] = a.take<float>((size_t)B * LAYERS[l].out);
    for (int l = 0; l < 3; ++l) s.h[l] = a.take<float>((size_t)B * LAYERS[l].out);
    for (int l = 0; l < 4; ++l) s.dz[l] = a.take<float>((size_t)B * LAYERS[l].out);
    s.dxn = a.take<float>((size_t)B * L0);
    s.part = a.take<double>((size_t)nb(B) + 16);
    return LD_OK;
}

size_t scratch_bytes(int B) {
    ld::Arena a;
    a.measuring = true;
    Scratch s;
    alloc_scratch(a, s, B);
    return a.off;
}

// forward over B normalised rows already in s.xn; prediction in s.z[3]
int forward(const ld_surrogate *S, Scratch &s, int B, cudaStream_t st) {
    const float *in = s.xn;
    for (int l = 0; l < 4; ++l) {
        const Layer L = LAYERS[l];
        fwd_kernel<<<nb((int64_t)B * L.out), 256, 0, st>>>(in, B, L.in, L.out, S->params + L.w, S->params + L.b,
                                                            s.z[l], l < 3 ? s.h[l] : nullptr, l < 3 ? 1 : 0);
        if (l < 3) in = s.h[l];
    }
    return ld::check_launch("surrogate forward", 4);
}

// backward from s.dz[3] (B x 1): parameter gradient into S->grad (when want_w),
// and the gradient with respect to the normalised input into s.dxn (when want_x)
int backward(ld_surrogate *S, Scratch &s, int B, bool want_w, bool want_x, cudaStream_t st) {
    int launches = 0;
    for (int l = 3; l >= 0; --l) {
        const Layer L = LAYERS[l];
        const float *in = l > 0 ? s.h[l - 1] : s.xn;
        if (want_w) {
            bwd_w_kernel<<<nb(L.out * (L.in + 1)), 256, 0, st>>>(s.dz[l], in, B, L.in, L.out, S->grad + L.w,
                                                                  S->grad + L.b);
            ++launches;
        }
        if (l > 0) {
            bwd_in_kernel<<<nb((int64_t)B * L.in), 256, 0, st>>>(s.dz[l], B, L.in, L.out, S->params + L.w,
                                                                  s.z[l - 1], s.dz[l - 1]);
            ++launches;
        } else if (want_x) {
            bwd_in_kernel<<<nb((int64_t)B * L.in), 256, 0, st>>>(s.dz[0], B, L.in, L.out, S->params + L.w,
                                                                  nullptr, s.dxn);
            ++launches;
        }
    }
    return ld::check_launch("surrogate backward", launches);
}

// loss (mean over Ntot) of rows [0, B) of (theta, y); sets s.dz[3]; optional host loss
int loss_and_grad(ld_surrogate *S, Scratch &s, const float *theta, const float *y, int B, int Ntot,
                  double *loss_host, cudaStream_t st) {
    norm_in_kernel<<<nb(B * L0), 256, 0, st>>>(theta, B, S->norm, S->norm + 4, s.xn);
    LD_TRY(ld::check_launch("surrogate norm"));
    LD_TRY(forward(S, s, B, st));
    loss_kernel<<<nb(B), 256, 0, st>>>(s.z[3], y, B, Ntot, S->norm + 8, S->norm + 9, s.dz[3], s.part);
    LD_TRY(ld::check_launch("surrogate loss"));
    LD_TRY(backward(S, s, B, true, false, st));
    if (loss_host) {
        std::vector<double> part(nb(B));
        LD_CHECK_CUDA(cudaMemcpyAsync(part.data(), s.part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st));
        LD_CHECK_CUDA(cudaStreamSynchronize(st));
        double t = 0.0;
        for (double v : part) t += v;
        *loss_host = t / Ntot;
    }
    return LD_OK;
}

int check_handle(const ld_surrogate *S) {
    if (!S) {
        ld::set_error("surrogate handle is NULL");
        return LD_ERR_INVALID;
    }
    return LD_OK;
}

}  // namespace

extern "C" {

int surrogate_create(uint64_t seed, void *stream, ld_surrogate **out) {
    ld::clear_error();
    LD_REQUIRE(out != nullptr, "surrogate_create: out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    ld_surrogate *S = new ld_surrogate();
    auto fail = [&](cudaError_t e) {
        ld::set_error("surrogate_create: %s", cudaGetErrorString(e));
        cudaFree(S->params);
        cudaFree(S->grad);
        cudaFree(S->m);
        cudaFree(S->v);
        cudaFree(S->norm);
        delete S;
        return LD_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&S->params, NPARAM * sizeof(float))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&S->grad, NPARAM * sizeof(float))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&S->m, NPARAM * sizeof(float))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&S->v, NPARAM * sizeof(float))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&S->norm, 16 * sizeof(float))) != cudaSuccess) return fail(e);
    init_kernel<<<nb(NPARAM), 256, 0, st>>>(S->params, seed);
    fill_kernel<<<nb(NPARAM), 256, 0, st>>>(S->m, NPARAM, 0.f);
    fill_kernel<<<nb(NPARAM), 256, 0, st>>>(S->v, NPARAM, 0.f);
    fill_kernel<<<1, 32, 0, st>>>(S->norm, 4, 0.f);      // mu
    fill_kernel<<<1, 32, 0, st>>>(S->norm + 4, 4, 1.f);  // sd
    fill_kernel<<<1, 32, 0, st>>>(S->norm + 8, 1, 0.f);  // ymu
    fill_kernel<<<1, 32, 0, st>>>(S->norm + 9, 1, 1.f);  // ysd
    if (ld::check_launch("surrogate_create", 7) != LD_OK || (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(cudaGetLastError());
    *out = S;
    return LD_OK;
}

int surrogate_set_params(ld_surrogate *S, const float *params_host, void *stream) {
    ld::clear_error();
    LD_TRY(check_handle(S));
    LD_REQUIRE(params_host != nullptr, "surrogate_set_params: NULL params");
    cudaStream_t st = (cudaStream_t)stream;
    LD_CHECK_CUDA(cudaMemcpyAsync(S->params, params_host, NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    LD_CHECK_CUDA(cudaStreamSynchronize(st));
    return LD_OK;
}

int surrogate_get_params(const ld_surrogate *S, float *params_host, void *stream) {
    ld::clear_error();
    LD_TRY(check_handle(S));
    LD_REQUIRE(params_host != nullptr, "surrogate_get_params: NULL params");
    cudaStream_t st = (cudaStream_t)stream;
    LD_CHECK_CUDA(cudaMemcpyAsync(params_host, S->params, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st));
    LD_CHECK_CUDA(cudaStreamSynchronize(st));
    return LD_OK;
}

int surrogate_get_norm(const ld_surrogate *S, float *norm_host, void *stream) {
    ld::clear_error();
    LD_TRY(check_handle(S));
    LD_REQUIRE(norm_host != nullptr, "surrogate_get_norm: NULL norm");
    cudaStream_t st = (cudaStream_t)stream;
    LD_CHECK_CUDA(cudaMemcpyAsync(norm_host, S->norm, 10 * sizeof(float), cudaMemcpyDeviceToHost, st));
    LD_CHECK_CUDA(cudaStreamSynchronize(st));
    return LD_OK;
}

int surrogate_set_norm(ld_surrogate *S, const float *norm_host, void *stream) {
    ld::clear_error();
    LD_TRY(check_handle(S));
    LD_REQUIRE(norm_host != nullptr, "surrogate_set_norm: NULL norm");
    for (int k = 0; k < 10; ++k) {
        const bool scale = (k >= 4 && k < 8) || k == 9;  // sd[4] and ysd
        LD_REQUIRE(isfinite(norm_host[k]) && (!scale || norm_host[k] > 0.f),
                   "surrogate_set_norm: entry %d must be finite (and > 0 for a scale)", k);
    }
    cudaStream_t st = (cudaStream_t)stream;
    LD_CHECK_CUDA(cudaMemcpyAsync(S->norm, norm_host, 10 * sizeof(float), cudaMemcpyHostToDevice, st));
    LD_CHECK_CUDA(cudaStreamSynchronize(st));
    return LD_OK;
}

int surrogate_loss_grad(ld_surrogate *S, const float *theta_dev, const float *y_dev, int32_t N,
                        double *loss_host, float *grad_host, void *stream) {
    ld::clear_error();
    LD_TRY(check_handle(S));
    LD_REQUIRE(theta_dev && y_dev && N > 0, "surrogate_loss_grad: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    ld::Arena a;
    LD_TRY(ld::arena_open(a, nullptr, 0, scratch_bytes(N)));
    Scratch s;
    alloc_scratch(a, s, N);
    int code = loss_and_grad(S, s, theta_dev, y_dev, N, N, loss_host, st);
    if (code == LD_OK && grad_host) {
        cudaError_t e = cudaMemcpyAsync(grad_host, S->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            ld::set_error("surrogate_loss_grad: %s", cudaGetErrorString(e));
            code = LD_ERR_CUDA;
        }
    }
    ld::arena_close(a);
    return code;
}

int surrogate_train(ld_surrogate *S, const float *theta_dev, const float *y_dev, int32_t N, int32_t epochs,
                    int32_t batch, float lr, void *stream, double *final_loss_host) {
    ld::clear_error();
    LD_TRY(check_handle(S));
    LD_REQUIRE(theta_dev && y_dev && N > 0 && epochs >= 0 && batch > 0 && lr > 0,
               "surrogate_train: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int B = batch < N ? batch : N;
    ld::Arena a;
    LD_TRY(ld::arena_open(a, nullptr, 0, scratch_bytes(N)));
    Scratch s;
    alloc_scratch(a, s, N);
    int code = [&]() -> int {
        // normalisation from the training data (inputs and target)
        moments_kernel<<<L0, 256, 0, st>>>(theta_dev, N, L0, S->norm, S->norm + 4);
        moments_kernel<<<1, 256, 0, st>>>(y_dev, N, 1, S->norm + 8, S->norm + 9);
        LD_TRY(ld::check_launch("surrogate moments", 2));
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        for (int ep = 0; ep < epochs; ++ep) {
            for (int r0 = 0; r0 < N; r0 += B) {
                const int Bc = (N - r0) < B ? (N - r0) : B;
                LD_TRY(loss_and_grad(S, s, theta_dev + (size_t)r0 * L0, y_dev + r0, Bc, Bc, nullptr, st));
                S->step += 1;
                const float c1 = 1.f - powf(b1, (float)S->step), c2 = 1.f - powf(b2, (float)S->step);
                adam_kernel<<<nb(NPARAM), 256, 0, st>>>(S->params, S->grad, S->m, S->v, NPARAM, lr, b1, b2, eps, c1,
                                                         c2);
                LD_TRY(ld::check_launch("surrogate adam"));
            }
        }
        double loss = 0.0;
        LD_TRY(loss_and_grad(S, s, theta_dev, y_dev, N, N, &loss, st));
        if (final_loss_host) *final_loss_host = loss;
        return LD_OK;
    }();
    ld::arena_close(a);
    return code;
}

int surrogate_infer(const ld_surrogate *S, const float *q_dev, int32_t Q, float *out_dev, float *dout_dev,
                    void *stream) {
    ld::clear_error();
    LD_TRY(check_handle(S));
    LD_REQUIRE(q_dev && out_dev && Q > 0, "surrogate_infer: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    ld::Arena a;
    LD_TRY(ld::arena_open(a, nullptr, 0, scratch_bytes(Q)));
    Scratch s;
    alloc_scratch(a, s, Q);
    ld_surrogate *Sm = const_cast<ld_surrogate *>(S);  // backward writes only scratch when want_w = false
    int code = [&]() -> int {
        norm_in_kernel<<<nb(Q * L0), 256, 0, st>>>(q_dev, Q, S->norm, S->norm + 4, s.xn);
        LD_TRY(ld::check_launch("surrogate norm"));
        LD_TRY(forward(S, s, Q, st));
        if (dout_dev) {
            fill_kernel<<<nb(Q), 256, 0, st>>>(s.dz[3], Q, 1.f);
            LD_TRY(ld::check_launch("surrogate seed"));
            LD_TRY(backward(Sm, s, Q, false, true, st));
        }
        denorm_kernel<<<nb(Q * L0), 256, 0, st>>>(s.z[3], s.dxn, Q, S->norm + 4, S->norm + 8, S->norm + 9,
                                                   out_dev, dout_dev);
        LD_TRY(ld::check_launch("surrogate denorm"));
        LD_CHECK_CUDA(cudaStreamSynchronize(st));
        return LD_OK;
    }();
    ld::arena_close(a);
    return code;
}

void surrogate_free(ld_surrogate *S) {
    if (!S) return;
    cudaFree(S->params);
    cudaFree(S->grad);
    cudaFree(S->m);
    cudaFree(S->v);
    cudaFree(S->norm);
    delete S;
}

}  // extern "C"
