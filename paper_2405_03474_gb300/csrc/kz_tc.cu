// Tensor-core (tcgen05) kernel product: placeholder until the kernel lands.
#include "common.cuh"

namespace ld {
size_t kz_tc_workspace(int64_t, int, int, int) { return 0; }
int kz_tc(const float *, int64_t, int, int, double, double, const float *, float *, int, int,
          Arena &, cudaStream_t) {
    set_error("tensor-core precisions are not built yet");
    return LD_ERR_UNSUPPORTED;
}
}  // namespace ld
