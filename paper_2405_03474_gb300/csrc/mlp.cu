// Surrogate MLP: placeholder entry points until the kernels land.
#include "common.cuh"

extern "C" {
int surrogate_create(uint64_t, void *, ld_surrogate **) { ld::set_error("surrogate not built yet"); return LD_ERR_UNSUPPORTED; }
int surrogate_set_params(ld_surrogate *, const float *, void *) { return LD_ERR_UNSUPPORTED; }
int surrogate_get_params(const ld_surrogate *, float *, void *) { return LD_ERR_UNSUPPORTED; }
int surrogate_loss_grad(ld_surrogate *, const float *, const float *, int32_t, double *, float *, void *) { return LD_ERR_UNSUPPORTED; }
int surrogate_train(ld_surrogate *, const float *, const float *, int32_t, int32_t, int32_t, float, void *, double *) { return LD_ERR_UNSUPPORTED; }
int surrogate_infer(const ld_surrogate *, const float *, int32_t, float *, float *, void *) { return LD_ERR_UNSUPPORTED; }
void surrogate_free(ld_surrogate *) {}
}
