// Single-precision refinement kernels: k_refine<float>, k_refine2 and
// k_cross_fix<float> (see refine_kern.cuh).
#include "refine_kern.cuh"

namespace pj {

void launch_refine_f32(pj_ctx* ctx, RefineArgs& a, int64_t n_tiles, bool full, int variant, cudaStream_t st) {
  if (variant == 1) {
    if (full) launch_refine<float, true>(ctx, a, n_tiles, st);
    else launch_refine<float, false>(ctx, a, n_tiles, st);
  } else {
    if (full) launch_refine2<true>(ctx, a, n_tiles, st);
    else launch_refine2<false>(ctx, a, n_tiles, st);
  }
}

}  // namespace pj
