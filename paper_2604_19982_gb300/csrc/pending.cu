// Entry points whose kernels are not built yet; they fail loudly.
#include <string>

#include "internal.h"

namespace pj {

pj_status join_streamed(pj_ctx* ctx, const pj_set*, const pj_set*, const pj_query*, pj_result*, cudaStream_t,
                        std::string&) {
  ctx->last_error = "streamed join not built yet";
  return PJ_EINVAL;
}

}  // namespace pj

extern "C" {
pj_status pj_mlp_train(pj_ctx* ctx, const float*, const float*, int64_t, int, uint64_t) {
  if (ctx) ctx->last_error = "MLP not built yet";
  return PJ_EINVAL;
}
pj_status pj_mlp_save(const pj_ctx*, const char*) { return PJ_EINVAL; }
pj_status pj_mlp_load(pj_ctx*, const char*) { return PJ_EINVAL; }
pj_status pj_mlp_set_weights(pj_ctx*, const float*, const float*, const float*, const float*, const float*,
                             const float*) {
  return PJ_EINVAL;
}
pj_status pj_mlp_get_weights(const pj_ctx*, float*, float*, float*, float*, float*, float*) { return PJ_EINVAL; }
pj_status pj_mlp_forward(pj_ctx*, const float*, int64_t, float*, void*) { return PJ_EINVAL; }
pj_status pj_mlp_grad(pj_ctx*, const float*, const float*, int64_t, float*, float*, float*, float*, float*, float*,
                      float*, void*) {
  return PJ_EINVAL;
}
pj_status pj_pair_features(pj_ctx*, const pj_set*, const pj_set*, const int32_t*, const int32_t*, int64_t,
                           float*) {
  return PJ_EINVAL;
}
}
