// FMA-throughput micro-benchmark: the measured FP32 / FP64 arithmetic peak
// used as the roofline denominator of the refinement kernels (the
// geometry is plain ALU arithmetic, not a tensor-core contraction).
#include "internal.h"

namespace pj {

// 8 independent FMA chains per thread keep every FMA pipe busy.
template <class T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T seed, T* sink) {
  T a0 = seed + threadIdx.x, a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
  T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
  const T m = T(0.999999), c = T(1e-7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = a0 * m + c;
      a1 = a1 * m + c;
      a2 = a2 * m + c;
      a3 = a3 * m + c;
      a4 = a4 * m + c;
      a5 = a5 * m + c;
      a6 = a6 * m + c;
      a7 = a7 * m + c;
    }
  }
  T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == T(-1234.5)) sink[blockIdx.x] = s;   // never true; keeps the chains live
}

}  // namespace pj

using namespace pj;

extern "C" pj_status pj_fma_peak(pj_ctx* ctx, int fp64, double* gflops) {
  if (!ctx || !gflops) return PJ_EINVAL;
  try {
    PJ_CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int blocks = ctx->sm_count * 8, threads = 256;
    const int iters = fp64 ? 64 : 2048;
    void* sink = ws_get(ctx, WS_MISC5, (size_t)blocks * 8, st);
    cudaEvent_t e0 = ctx->ev[62], e1 = ctx->ev[63];
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      PJ_CK(cudaEventRecord(e0, st));
      if (fp64) k_fma_peak<double><<<blocks, threads, 0, st>>>(iters, 1.0, (double*)sink);
      else k_fma_peak<float><<<blocks, threads, 0, st>>>(iters, 1.0f, (float*)sink);
      PJ_CK(cudaGetLastError());
      PJ_COUNT_LAUNCH;
      PJ_CK(cudaEventRecord(e1, st));
      PJ_CK(cudaEventSynchronize(e1));
      float ms = 0;
      PJ_CK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && ms < best) best = ms;
    }
    double flops = 2.0 * 8.0 * 16.0 * (double)iters * blocks * threads;
    *gflops = flops / (best * 1e-3) / 1e9;
    return PJ_OK;
  } catch (const CudaError& e) {
    ctx->last_error = std::string(e.what) + ": " + cudaGetErrorString(e.e);
    return PJ_ECUDA;
  }
}
