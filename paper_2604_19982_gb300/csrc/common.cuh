// Device-side utilities shared by the kernels of the join library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pj {

// Device error word bits (ORed by kernels, read by the host after a join).
enum : int {
  ERR_MBAR_TIMEOUT = 1,   // an mbarrier wait hit its iteration limit
  ERR_BOUNDS = 2,         // an index outside its buffer was skipped
  ERR_NONFINITE = 4,      // NaN / Inf input data
  ERR_CAPACITY = 8        // an output list would have overflowed its buffer
};

constexpr int CHUNK = 256;       // facets per chunk (coarse pruning box)
constexpr int BLK = 32;          // facets per block (side of a refinement unit)
constexpr int REFINE_THREADS = 384;   // 12 warps: one CTA per SM (shared memory of the stages)

__device__ __forceinline__ void set_err(int* err, int bit) {
  if (err) atomicOr(err, bit);
}

// ---------------------------------------------------------------- mbarrier
// One-shot TMA staging: thread 0 arms the barrier with the byte count and
// issues the bulk copy; every thread then waits on the phase parity.  Waits
// are bounded: after `limit` polls the caller gets `false` and reports
// ERR_MBAR_TIMEOUT instead of spinning forever.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// 1-D bulk copy global -> shared (non-multicast), completion on `bar`.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}

// ---------------------------------------------------------------- ordered bits
// Non-negative IEEE floats compare like their unsigned bit patterns, so a
// per-pair minimum can be kept with integer atomicMin.

__device__ __forceinline__ unsigned f2bits(float x) { return __float_as_uint(x); }
__device__ __forceinline__ unsigned long long d2bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}
__device__ __forceinline__ float bits2f(unsigned b) { return __uint_as_float(b); }
__device__ __forceinline__ double bits2d(unsigned long long b) {
  return __longlong_as_double(static_cast<long long>(b));
}

template <class T>
struct Bits;
template <>
struct Bits<float> {
  using U = unsigned;
  __device__ static U enc(float x) { return f2bits(x); }
  __device__ static float dec(U b) { return bits2f(b); }
};
template <>
struct Bits<double> {
  using U = unsigned long long;
  __device__ static U enc(double x) { return d2bits(x); }
  __device__ static double dec(U b) { return bits2d(b); }
};

// ---------------------------------------------------------------- warp mins
template <class T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace pj
