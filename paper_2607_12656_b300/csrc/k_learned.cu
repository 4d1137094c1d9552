// Learned-model decode (placeholder until the kernels land).
#include <vector>
#include "sgs_internal.h"
namespace sgs {
size_t learned_work_bytes(const sgs_scene_info &) { return 0; }
cudaError_t launch_learned_decode(const uint8_t *, const sgs_scene_info &, const sgs_scene_out &,
                                  uint8_t *, int *, cudaStream_t) { return cudaErrorNotSupported; }
int learned_token_fc(sgs_ctx *, const uint8_t *, const uint8_t *, uint32_t, uint32_t,
                     std::vector<uint32_t> &, std::vector<uint32_t> &) { return SGS_E_UNSUPPORTED; }
}  // namespace sgs
extern "C" int sgs_train(sgs_ctx *, const uint8_t *, uint32_t, uint32_t, const sgs_train_params *,
                         uint32_t, float *, float *, float *) { return SGS_E_UNSUPPORTED; }
extern "C" int sgs_train_grad(sgs_ctx *, const uint8_t *, uint32_t, uint32_t, const int64_t *,
                              uint32_t, const float *, float *, float *) { return SGS_E_UNSUPPORTED; }
extern "C" int sgs_freeze(const float *, const uint8_t *, uint32_t, uint32_t, uint32_t, uint8_t *) {
    return SGS_E_UNSUPPORTED;
}
