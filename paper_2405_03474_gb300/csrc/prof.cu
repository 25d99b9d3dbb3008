// Launch accounting and event timing of the kernel-product launches.
#include <atomic>
#include <vector>

#include "common.cuh"

namespace ld {

namespace {
std::atomic<long long> g_launches{0};
struct Rec {
    cudaEvent_t a = nullptr, b = nullptr;
    double pairs = 0, flops = 0;
    int kernel = 0;
};
struct Total {
    double ms = 0, pairs = 0, flops = 0;
    int64_t launches = 0;
};
bool g_on = false;
std::vector<Rec> g_recs;
Total g_last[PROF_KERNELS];  // per kernel, of the last closed profile window
}  // namespace

void count_launches(int k) { g_launches += k; }

int prof_begin_launch(cudaStream_t st, int kernel, double pairs, double mma_flops) {
    if (!g_on) return -1;
    Rec r;
    if (cudaEventCreate(&r.a) != cudaSuccess) return -1;
    if (cudaEventCreate(&r.b) != cudaSuccess) {
        cudaEventDestroy(r.a);
        return -1;
    }
    r.pairs = pairs;
    r.flops = mma_flops;
    r.kernel = kernel >= 0 && kernel < PROF_KERNELS ? kernel : 0;
    cudaEventRecord(r.a, st);
    g_recs.push_back(r);
    return (int)g_recs.size() - 1;
}

void prof_end_launch(cudaStream_t st, int slot) {
    if (slot < 0 || slot >= (int)g_recs.size()) return;
    cudaEventRecord(g_recs[slot].b, st);
}

}  // namespace ld

extern "C" {

int64_t ld_launch_count(void) { return (int64_t)ld::g_launches.load(); }

int ld_profile_begin(void) {
    ld::clear_error();
    for (auto &r : ld::g_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    ld::g_recs.clear();
    ld::g_on = true;
    return LD_OK;
}

int ld_profile_end(double *kz_ms, int64_t *kz_launches, double *kz_pairs, double *kz_mma_flops) {
    ld::clear_error();
    ld::g_on = false;
    double ms = 0, pairs = 0, flops = 0;
    int code = LD_OK;
    for (auto &t : ld::g_last) t = ld::Total();
    for (auto &r : ld::g_recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
            ld::set_error("ld_profile_end: event timing failed");
            code = LD_ERR_CUDA;
        }
        ms += t;
        pairs += r.pairs;
        flops += r.flops;
        ld::Total &k = ld::g_last[r.kernel];
        k.ms += t;
        k.pairs += r.pairs;
        k.flops += r.flops;
        k.launches += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    if (kz_ms) *kz_ms = ms;
    if (kz_launches) *kz_launches = (int64_t)ld::g_recs.size();
    if (kz_pairs) *kz_pairs = pairs;
    if (kz_mma_flops) *kz_mma_flops = flops;
    ld::g_recs.clear();
    return code;
}

int ld_profile_kernel(int32_t kernel, double *ms, int64_t *launches, double *pairs, double *mma_flops) {
    ld::clear_error();
    if (kernel < 0 || kernel >= ld::PROF_KERNELS) {
        ld::set_error("ld_profile_kernel: kernel id %d out of range", kernel);
        return LD_ERR_INVALID;
    }
    const ld::Total &k = ld::g_last[kernel];
    if (ms) *ms = k.ms;
    if (launches) *launches = k.launches;
    if (pairs) *pairs = k.pairs;
    if (mma_flops) *mma_flops = k.flops;
    return LD_OK;
}

}  // extern "C"
