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

