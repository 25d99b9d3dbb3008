// ld_kz_static: the kernel product W = (K + noise I) V with no device
// allocation at all.
//
// Some callers cannot call cudaMalloc: a plug-in running inside a host
// framework that owns every byte of device memory through its own pool, a
// latency-critical loop where cudaMalloc/cudaFree would synchronise the device,
// or a process started under a hard device-memory cap.  For them the scratch
// the product needs (scaled points, the fp16 operand image of V, per-column
// scales and partial maxima, an error word) is carved from one file-scope
// __device__ array of fixed size.  Every GPU that loads this library reserves
// that array until the process exits.
//
// The array's device address is looked up once per device, with that device
// current, the first time this entry point runs on it (cudaGetSymbolAddress);
// make that first call on each device before any stream capture begins.  Like
// ld_kz, a call in a tensor-core precision synchronises its stream before it
// returns (it reads the product's error word); in FP64 and FP32 the work stays
// queued on the stream.  All calls share the one array and it keeps the
// previous call's contents: the product rewrites everything it reads and clears
// its error word itself, but two calls whose work overlaps on the GPU
// (different streams, or host threads) race on the array.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t KZ_STATIC_BYTES = size_t(32) << 20;  // 32 MiB per device
constexpr int MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_kz_static_scratch[KZ_STATIC_BYTES];

std::mutex g_mu;
void *g_scratch[MAX_DEVICES] = {nullptr};

// Device address of the static scratch on the current device (set up once).
int static_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        ld::set_error("ld_kz_static: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    if (dev < 0 || dev >= MAX_DEVICES) {
        ld::set_error("ld_kz_static: device ordinal %d out of range", dev);
        return LD_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_kz_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            ld::set_error("ld_kz_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return LD_ERR_CUDA;
        }
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return LD_OK;
}

}  // namespace

extern "C" {

size_t ld_kz_static_capacity(void) { return KZ_STATIC_BYTES; }

int ld_kz_static(const double *X_dev, int64_t n, int32_t d, ld_kernel kern, const void *V_dev,
                 void *W_dev, int32_t c, int32_t precision, void *stream) {
    using namespace ld;
    clear_error();
    LD_REQUIRE(X_dev && V_dev && W_dev && n > 0 && c > 0, "ld_kz_static: bad pointers or sizes");
    LD_REQUIRE(V_dev != W_dev, "ld_kz_static: W must not alias V");
    LD_REQUIRE(d >= 1 && d <= 32, "ld_kz_static: d must be in [1, 32]");
    LD_REQUIRE(d <= 8 || precision == LD_FP64 || precision == LD_FP32,
               "ld_kz_static: tensor-core precisions support d <= 8");
    LD_REQUIRE(c <= 4096, "ld_kz_static: at most 4096 columns");
    LD_REQUIRE(kern.lengthscale > 0 && kern.variance > 0 && kern.noise >= 0 &&
                   (kern.kind == LD_RBF || kern.kind == LD_MATERN52),
               "ld_kz_static: bad kernel parameters");
    LD_REQUIRE(precision >= LD_FP64 && precision <= LD_F16X3_TC, "ld_kz_static: bad precision");
    const size_t need = ld_kz_workspace_size(n, d, c, precision);
    if (need > KZ_STATIC_BYTES) {
        set_error("ld_kz_static: this size needs %zu bytes of scratch, more than the %zu-byte static "
                  "array; use ld_kz with a caller workspace",
                  need, KZ_STATIC_BYTES);
        return LD_ERR_WORKSPACE;
    }
    void *base = nullptr;
    LD_TRY(static_scratch(&base));
    cudaStream_t st = (cudaStream_t)stream;
    Arena a;
    LD_TRY(arena_open(a, base, KZ_STATIC_BYTES, need));  // caller-scratch mode: no allocation
    if (precision == LD_FP64) {
        double *Xs = a.take<double>((size_t)n * d);
        LD_TRY(prep_points<double>(X_dev, n, d, point_scale(kern), Xs, st));
        return kz_any<double>(Xs, n, d, kern, (const double *)V_dev, (double *)W_dev, c, precision, a, st);
    }
    float *Xs = a.take<float>((size_t)n * d);
    LD_TRY(prep_points<float>(X_dev, n, d, point_scale(kern), Xs, st));
    return kz_any<float>(Xs, n, d, kern, (const float *)V_dev, (float *)W_dev, c, precision, a, st);
}

}  // extern "C"
