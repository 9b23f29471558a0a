// Double-precision refinement kernels: k_refine<double> and
// k_cross_fix<double> (see refine_kern.cuh).
#include "refine_kern.cuh"

namespace pj {

void launch_refine_f64(pj_ctx* ctx, RefineArgs& a, int64_t n_tiles, bool full, cudaStream_t st) {
  if (full) launch_refine<double, true>(ctx, a, n_tiles, st);
  else launch_refine<double, false>(ctx, a, n_tiles, st);
}

}  // namespace pj
