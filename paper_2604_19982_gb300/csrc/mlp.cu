// Learned proposal: a 16 -> 64 -> 64 -> 1 ReLU network in bf16 on the
// tensor cores (mma.sync m16n8k16, fp32 accumulation) that predicts
// log(1 + d) of a candidate pair from box and coarse-LoD features.  It only
// orders the k-NN refinement and picks the starting LoD of a pair; results
// never depend on it.  (The paper has no learned component.)
//
// A warp handles 16 rows: layer 1 is 8 MMAs (n = 64), its accumulators are
// repacked in registers as the A fragments of layer 2 (32 MMAs), the last
// layer is a 64-wide dot product.  The backward pass forms dL/dz2 and
// dL/dz1 in the same fragment layout, dL/dh1 = dz2 W2 on the tensor cores,
// and the weight gradients dz^T h (K = the 16 rows) after a transpose
// through the warp's shared-memory slice; per-block gradient sums live in
// shared memory and are added to the global gradient once per block.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pj {

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int MLP_WARPS = 4;

struct MlpSmem {
  __nv_bfloat16 w1[64 * 16];   // [n][k]
  __nv_bfloat16 w2[64 * 64];   // [n][k]
  __nv_bfloat16 w2t[64 * 64];  // [k][n]
  float b1[64], b2[64], w3[64], b3;
};

__device__ void load_weights(MlpSmem& s, const float* W) {
  for (int i = threadIdx.x; i < 64 * 16; i += blockDim.x) s.w1[i] = __float2bfloat16_rn(W[MLP_W1 + i]);
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    s.w2[i] = __float2bfloat16_rn(W[MLP_W2 + i]);
    int n = i / 64, k = i % 64;
    s.w2t[k * 64 + n] = __float2bfloat16_rn(W[MLP_W2 + i]);
  }
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    s.b1[i] = W[MLP_B1 + i];
    s.b2[i] = W[MLP_B2 + i];
    s.w3[i] = W[MLP_W3 + i];
  }
  if (threadIdx.x == 0) s.b3 = W[MLP_B3];
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// forward of one 16-row tile: X fragments in, z1/z2 accumulators (after
// bias, before ReLU) and y for rows g and g + 8 (valid in lanes t == 0)
struct Tile16 {
  uint32_t ax[4];
  float z1[8][4], z2[8][4];
  float y0, y1;
};

__device__ __forceinline__ void load_x(Tile16& T, const float* X, const int32_t* idx, int64_t row0, int64_t n,
                                       int lane) {
  const int g = lane >> 2, t = lane & 3;
  float v[2][4];
  for (int h = 0; h < 2; ++h) {
    int64_t r = row0 + g + 8 * h;
    if (r < n) {
      int64_t rr = idx ? idx[r] : r;
      const float* x = X + 16 * rr;
      v[h][0] = x[2 * t];
      v[h][1] = x[2 * t + 1];
      v[h][2] = x[2 * t + 8];
      v[h][3] = x[2 * t + 9];
    } else {
      v[h][0] = v[h][1] = v[h][2] = v[h][3] = 0.f;
    }
  }
  T.ax[0] = pack_bf16(v[0][0], v[0][1]);
  T.ax[1] = pack_bf16(v[1][0], v[1][1]);
  T.ax[2] = pack_bf16(v[0][2], v[0][3]);
  T.ax[3] = pack_bf16(v[1][2], v[1][3]);
}

__device__ __forceinline__ void forward_tile(Tile16& T, const MlpSmem& s, int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    T.z1[j][0] = T.z1[j][1] = T.z1[j][2] = T.z1[j][3] = 0.f;
    uint32_t b[2] = {ld_pair(&s.w1[(8 * j + g) * 16 + 2 * t]), ld_pair(&s.w1[(8 * j + g) * 16 + 2 * t + 8])};
    mma16816(T.z1[j], T.ax, b);
    float c0 = s.b1[8 * j + 2 * t], c1 = s.b1[8 * j + 2 * t + 1];
    T.z1[j][0] += c0;
    T.z1[j][1] += c1;
    T.z1[j][2] += c0;
    T.z1[j][3] += c1;
  }
  uint32_t a2[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    a2[kk][0] = pack_bf16(fmaxf(T.z1[2 * kk][0], 0.f), fmaxf(T.z1[2 * kk][1], 0.f));
    a2[kk][1] = pack_bf16(fmaxf(T.z1[2 * kk][2], 0.f), fmaxf(T.z1[2 * kk][3], 0.f));
    a2[kk][2] = pack_bf16(fmaxf(T.z1[2 * kk + 1][0], 0.f), fmaxf(T.z1[2 * kk + 1][1], 0.f));
    a2[kk][3] = pack_bf16(fmaxf(T.z1[2 * kk + 1][2], 0.f), fmaxf(T.z1[2 * kk + 1][3], 0.f));
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    T.z2[j][0] = T.z2[j][1] = T.z2[j][2] = T.z2[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t b[2] = {ld_pair(&s.w2[(8 * j + g) * 64 + 16 * kk + 2 * t]),
                       ld_pair(&s.w2[(8 * j + g) * 64 + 16 * kk + 2 * t + 8])};
      mma16816(T.z2[j], a2[kk], b);
    }
    float c0 = s.b2[8 * j + 2 * t], c1 = s.b2[8 * j + 2 * t + 1];
    T.z2[j][0] += c0;
    T.z2[j][1] += c1;
    T.z2[j][2] += c0;
    T.z2[j][3] += c1;
  }
  float p0 = 0.f, p1 = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float w0 = s.w3[8 * j + 2 * t], w1 = s.w3[8 * j + 2 * t + 1];
    p0 += fmaxf(T.z2[j][0], 0.f) * w0 + fmaxf(T.z2[j][1], 0.f) * w1;
    p1 += fmaxf(T.z2[j][2], 0.f) * w0 + fmaxf(T.z2[j][3], 0.f) * w1;
  }
  p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
  p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
  T.y0 = p0 + s.b3;
  T.y1 = p1 + s.b3;
}

__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_fwd(const float* W, const float* X, int64_t n, float* y) {
  __shared__ MlpSmem s;
  load_weights(s, W);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t tiles = (n + 15) / 16;
  for (int64_t tile = blockIdx.x * MLP_WARPS + warp; tile < tiles; tile += (int64_t)gridDim.x * MLP_WARPS) {
    Tile16 T;
    load_x(T, X, nullptr, tile * 16, n, lane);
    forward_tile(T, s, lane);
    if (t == 0) {
      int64_t r0 = tile * 16 + g, r1 = r0 + 8;
      if (r0 < n) y[r0] = T.y0;
      if (r1 < n) y[r1] = T.y1;
    }
  }
}

// gradient of L = sum over rows of scale * (y - target)^2 / 2
__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_grad(const float* W, const float* X, const float* target,
                                                             const int32_t* idx, int64_t n, float scale,
                                                             float* grad, float* loss) {
  __shared__ MlpSmem s;
  extern __shared__ __align__(16) unsigned char dyn[];
  // dynamic: gradient sums, then per warp the staging tiles of dz / h1 / x
  float* sg = reinterpret_cast<float*>(dyn);
  __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(dyn + ((MLP_NW * 4 + 15) / 16) * 16);
  __shared__ float sloss;
  load_weights(s, W);
  for (int i = threadIdx.x; i < MLP_NW; i += blockDim.x) sg[i] = 0.f;
  if (threadIdx.x == 0) sloss = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  __nv_bfloat16* T1 = stage + warp * (2 * 16 * 64 + 16 * 16);
  __nv_bfloat16* T2 = T1 + 16 * 64;
  __nv_bfloat16* TX = T2 + 16 * 64;
  float gw3[16], gb2[16], gb1[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) gw3[i] = gb2[i] = gb1[i] = 0.f;
  float gb3 = 0.f, lsum = 0.f;
  const int64_t tiles = (n + 15) / 16;
  for (int64_t tile = blockIdx.x * MLP_WARPS + warp; tile < tiles; tile += (int64_t)gridDim.x * MLP_WARPS) {
    Tile16 T;
    const int64_t row0 = tile * 16;
    load_x(T, X, idx, row0, n, lane);
    forward_tile(T, s, lane);
    // residual and dL/dy of rows g, g + 8 (padding rows contribute 0)
    float r0 = 0.f, r1 = 0.f;
    if (t == 0) {
      if (row0 + g < n) r0 = T.y0 - target[idx ? idx[row0 + g] : row0 + g];
      if (row0 + g + 8 < n) r1 = T.y1 - target[idx ? idx[row0 + g + 8] : row0 + g + 8];
      lsum += 0.5f * scale * (r0 * r0 + r1 * r1);
      gb3 += scale * (r0 + r1);
    }
    const float dy0 = scale * __shfl_sync(0xffffffffu, r0, lane & ~3);
    const float dy1 = scale * __shfl_sync(0xffffffffu, r1, lane & ~3);
    // dz2 = dy w3 * [z2 > 0]; gradient of w3 and b2
    float dz2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * j + 2 * t;
      float h[4] = {fmaxf(T.z2[j][0], 0.f), fmaxf(T.z2[j][1], 0.f), fmaxf(T.z2[j][2], 0.f), fmaxf(T.z2[j][3], 0.f)};
      gw3[2 * j] += h[0] * dy0 + h[2] * dy1;
      gw3[2 * j + 1] += h[1] * dy0 + h[3] * dy1;
      dz2[j][0] = T.z2[j][0] > 0.f ? dy0 * s.w3[c] : 0.f;
      dz2[j][1] = T.z2[j][1] > 0.f ? dy0 * s.w3[c + 1] : 0.f;
      dz2[j][2] = T.z2[j][2] > 0.f ? dy1 * s.w3[c] : 0.f;
      dz2[j][3] = T.z2[j][3] > 0.f ? dy1 * s.w3[c + 1] : 0.f;
      gb2[2 * j] += dz2[j][0] + dz2[j][2];
      gb2[2 * j + 1] += dz2[j][1] + dz2[j][3];
    }
    // dh1 = dz2 W2 (tensor cores), dz1 = dh1 * [z1 > 0]
    uint32_t a[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      a[kk][0] = pack_bf16(dz2[2 * kk][0], dz2[2 * kk][1]);
      a[kk][1] = pack_bf16(dz2[2 * kk][2], dz2[2 * kk][3]);
      a[kk][2] = pack_bf16(dz2[2 * kk + 1][0], dz2[2 * kk + 1][1]);
      a[kk][3] = pack_bf16(dz2[2 * kk + 1][2], dz2[2 * kk + 1][3]);
    }
    float dz1[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      dz1[j][0] = dz1[j][1] = dz1[j][2] = dz1[j][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        uint32_t b[2] = {ld_pair(&s.w2t[(8 * j + g) * 64 + 16 * kk + 2 * t]),
                         ld_pair(&s.w2t[(8 * j + g) * 64 + 16 * kk + 2 * t + 8])};
        mma16816(dz1[j], a[kk], b);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) dz1[j][q] = T.z1[j][q] > 0.f ? dz1[j][q] : 0.f;
      gb1[2 * j] += dz1[j][0] + dz1[j][2];
      gb1[2 * j + 1] += dz1[j][1] + dz1[j][3];
    }
    // stage dz2, h1 (for gW2) and dz1 is staged after; rows g, g + 8
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * j + 2 * t;
      T2[g * 64 + c] = __float2bfloat16_rn(dz2[j][0]);
      T2[g * 64 + c + 1] = __float2bfloat16_rn(dz2[j][1]);
      T2[(g + 8) * 64 + c] = __float2bfloat16_rn(dz2[j][2]);
      T2[(g + 8) * 64 + c + 1] = __float2bfloat16_rn(dz2[j][3]);
      T1[g * 64 + c] = __float2bfloat16_rn(fmaxf(T.z1[j][0], 0.f));
      T1[g * 64 + c + 1] = __float2bfloat16_rn(fmaxf(T.z1[j][1], 0.f));
      T1[(g + 8) * 64 + c] = __float2bfloat16_rn(fmaxf(T.z1[j][2], 0.f));
      T1[(g + 8) * 64 + c + 1] = __float2bfloat16_rn(fmaxf(T.z1[j][3], 0.f));
    }
    // x tile for gW1 (the A fragments hold it: rows g, g+8, cols 2t.., 2t+8..)
    {
      const __nv_bfloat162* ax = reinterpret_cast<const __nv_bfloat162*>(T.ax);
      TX[g * 16 + 2 * t] = ax[0].x;
      TX[g * 16 + 2 * t + 1] = ax[0].y;
      TX[(g + 8) * 16 + 2 * t] = ax[1].x;
      TX[(g + 8) * 16 + 2 * t + 1] = ax[1].y;
      TX[g * 16 + 2 * t + 8] = ax[2].x;
      TX[g * 16 + 2 * t + 9] = ax[2].y;
      TX[(g + 8) * 16 + 2 * t + 8] = ax[3].x;
      TX[(g + 8) * 16 + 2 * t + 9] = ax[3].y;
    }
    __syncwarp();
    // gW2[m][k] = sum over rows of dz2[row][m] h1[row][k]: M = 64, N = 64, K = 16 rows
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t aa[4] = {pack2(T2[(2 * t) * 64 + 16 * i + g], T2[(2 * t + 1) * 64 + 16 * i + g]),
                        pack2(T2[(2 * t) * 64 + 16 * i + g + 8], T2[(2 * t + 1) * 64 + 16 * i + g + 8]),
                        pack2(T2[(2 * t + 8) * 64 + 16 * i + g], T2[(2 * t + 9) * 64 + 16 * i + g]),
                        pack2(T2[(2 * t + 8) * 64 + 16 * i + g + 8], T2[(2 * t + 9) * 64 + 16 * i + g + 8])};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t bb[2] = {pack2(T1[(2 * t) * 64 + 8 * j + g], T1[(2 * t + 1) * 64 + 8 * j + g]),
                          pack2(T1[(2 * t + 8) * 64 + 8 * j + g], T1[(2 * t + 9) * 64 + 8 * j + g])};
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, aa, bb);
        const int m = 16 * i + g, k = 8 * j + 2 * t;
        atomicAdd(&sg[MLP_W2 + m * 64 + k], c[0]);
        atomicAdd(&sg[MLP_W2 + m * 64 + k + 1], c[1]);
        atomicAdd(&sg[MLP_W2 + (m + 8) * 64 + k], c[2]);
        atomicAdd(&sg[MLP_W2 + (m + 8) * 64 + k + 1], c[3]);
      }
    }
    __syncwarp();
    // dz1 staged in T2 (dz2 no longer needed), then gW1 = dz1^T x: M = 64, N = 16, K = 16
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * j + 2 * t;
      T2[g * 64 + c] = __float2bfloat16_rn(dz1[j][0]);
      T2[g * 64 + c + 1] = __float2bfloat16_rn(dz1[j][1]);
      T2[(g + 8) * 64 + c] = __float2bfloat16_rn(dz1[j][2]);
      T2[(g + 8) * 64 + c + 1] = __float2bfloat16_rn(dz1[j][3]);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t aa[4] = {pack2(T2[(2 * t) * 64 + 16 * i + g], T2[(2 * t + 1) * 64 + 16 * i + g]),
                        pack2(T2[(2 * t) * 64 + 16 * i + g + 8], T2[(2 * t + 1) * 64 + 16 * i + g + 8]),
                        pack2(T2[(2 * t + 8) * 64 + 16 * i + g], T2[(2 * t + 9) * 64 + 16 * i + g]),
                        pack2(T2[(2 * t + 8) * 64 + 16 * i + g + 8], T2[(2 * t + 9) * 64 + 16 * i + g + 8])};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        uint32_t bb[2] = {pack2(TX[(2 * t) * 16 + 8 * j + g], TX[(2 * t + 1) * 16 + 8 * j + g]),
                          pack2(TX[(2 * t + 8) * 16 + 8 * j + g], TX[(2 * t + 9) * 16 + 8 * j + g])};
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, aa, bb);
        const int m = 16 * i + g, k = 8 * j + 2 * t;
        atomicAdd(&sg[MLP_W1 + m * 16 + k], c[0]);
        atomicAdd(&sg[MLP_W1 + m * 16 + k + 1], c[1]);
        atomicAdd(&sg[MLP_W1 + (m + 8) * 16 + k], c[2]);
        atomicAdd(&sg[MLP_W1 + (m + 8) * 16 + k + 1], c[3]);
      }
    }
    __syncwarp();
  }
  // per-lane column partials: sum over the 8 row groups, then into shared
#pragma unroll
  for (int i = 0; i < 16; ++i) {
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      gw3[i] += __shfl_xor_sync(0xffffffffu, gw3[i], o);
      gb2[i] += __shfl_xor_sync(0xffffffffu, gb2[i], o);
      gb1[i] += __shfl_xor_sync(0xffffffffu, gb1[i], o);
    }
  }
  if (g == 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * j + 2 * t;
      atomicAdd(&sg[MLP_W3 + c], gw3[2 * j]);
      atomicAdd(&sg[MLP_W3 + c + 1], gw3[2 * j + 1]);
      atomicAdd(&sg[MLP_B2 + c], gb2[2 * j]);
      atomicAdd(&sg[MLP_B2 + c + 1], gb2[2 * j + 1]);
      atomicAdd(&sg[MLP_B1 + c], gb1[2 * j]);
      atomicAdd(&sg[MLP_B1 + c + 1], gb1[2 * j + 1]);
    }
  }
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) {
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  }
  if (lane == 0) {
    atomicAdd(&sg[MLP_B3], gb3);
    atomicAdd(&sloss, lsum);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < MLP_NW; i += blockDim.x)
    if (sg[i] != 0.f) atomicAdd(&grad[i], sg[i]);
  if (threadIdx.x == 0 && loss) atomicAdd(loss, sloss);
}

// Adam step on the float master weights
__global__ void k_adam(float* w, float* m, float* v, const float* g, float lr, float b1, float b2, float c1, float c2,
                       int nw) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

// ------------------------------------------------------------------ features

// 16 features of a candidate pair (box, anchor and coarse-LoD quantities):
//  0 log1p(box MINDIST)        1 log1p(anchor distance)   2 log1p(centre distance)
//  3 log1p(diag r)             4 log1p(diag s)            5..7 centre offset / summed half extents per axis
//  8 log1p(max hd r, LoD 0)    9 log1p(max hd s, LoD 0)   10 log(facets r) / 10    11 log(facets s) / 10
// 12 log1p(min chunk-pair box gap at LoD 0)               13 MINDIST / (anchor distance + 1e-6)
// 14 log1p(max ph r + max ph s, LoD 0)                    15 1
__global__ void k_pair_features(int64_t n, const int32_t* pr, const int32_t* ps, const float* mbbR, const float* mbbS,
                                const float* ancR, const float* ancS, const float4* chR, const int64_t* coffR,
                                const float4* chS, const int64_t* coffS, const int64_t* foffR, const int64_t* foffS,
                                float* out, const int64_t* n_live) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (n_live && p >= *n_live) {   // padding of a fixed-capacity (graph) join: no pair ids there
    for (int k = 0; k < 16; ++k) out[16 * p + k] = 0.f;
    return;
  }
  const int r = pr[p], s = ps[p];
  const float* a = mbbR + 6LL * r;
  const float* b = mbbS + 6LL * s;
  float f[16];
  double md2 = 0, ad2 = 0, cd2 = 0, da = 0, db = 0;
  for (int k = 0; k < 3; ++k) {
    double g = fmax(0.0, fmax((double)b[k] - a[3 + k], (double)a[k] - b[3 + k]));
    md2 += g * g;
    double q = (double)ancR[3LL * r + k] - ancS[3LL * s + k];
    ad2 += q * q;
    double ca = 0.5 * ((double)a[k] + a[3 + k]), cb = 0.5 * ((double)b[k] + b[3 + k]);
    cd2 += (ca - cb) * (ca - cb);
    da += ((double)a[3 + k] - a[k]) * ((double)a[3 + k] - a[k]);
    db += ((double)b[3 + k] - b[k]) * ((double)b[3 + k] - b[k]);
    double hx = 0.5 * (((double)a[3 + k] - a[k]) + ((double)b[3 + k] - b[k]));
    f[5 + k] = (float)fmin(4.0, fabs(ca - cb) / (hx + 1e-9));
  }
  const double md = sqrt(md2), ad = sqrt(ad2);
  f[0] = (float)log1p(md);
  f[1] = (float)log1p(ad);
  f[2] = (float)log1p(sqrt(cd2));
  f[3] = (float)log1p(sqrt(da));
  f[4] = (float)log1p(sqrt(db));
  float hr = 0.f, hs = 0.f, pr_ = 0.f, ps_ = 0.f;
  for (int64_t c = coffR[r]; c < coffR[r + 1]; ++c) {
    hr = fmaxf(hr, chR[3 * c].w);
    pr_ = fmaxf(pr_, chR[3 * c + 1].w);
  }
  for (int64_t c = coffS[s]; c < coffS[s + 1]; ++c) {
    hs = fmaxf(hs, chS[3 * c].w);
    ps_ = fmaxf(ps_, chS[3 * c + 1].w);
  }
  f[8] = log1pf(hr);
  f[9] = log1pf(hs);
  f[10] = logf((float)(foffR[r + 1] - foffR[r]) + 1.f) / 10.f;
  f[11] = logf((float)(foffS[s + 1] - foffS[s]) + 1.f) / 10.f;
  float gmin = INFINITY;
  for (int64_t c = coffR[r]; c < coffR[r + 1]; ++c)
    for (int64_t e = coffS[s]; e < coffS[s + 1]; ++e) {
      float g2 = 0.f;
      for (int k = 0; k < 3; ++k) {
        float lo1 = (&chR[3 * c].x)[k], hi1 = (&chR[3 * c + 1].x)[k];
        float lo2 = (&chS[3 * e].x)[k], hi2 = (&chS[3 * e + 1].x)[k];
        float gg = fmaxf(0.f, fmaxf(lo2 - hi1, lo1 - hi2));
        g2 += gg * gg;
      }
      gmin = fminf(gmin, g2);
    }
  f[12] = log1pf(sqrtf(gmin < INFINITY ? gmin : 0.f));
  f[13] = (float)(md / (ad + 1e-6));
  f[14] = log1pf(pr_ + ps_);
  f[15] = 1.f;
  for (int k = 0; k < 16; ++k) out[16 * p + k] = f[k];
}

void pair_features(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr, const int32_t* ps, int64_t n,
                   float* out, cudaStream_t st, const int64_t* n_live) {
  if (n == 0) return;
  const LodData& a = R->lod[0];
  const LodData& b = S->lod[0];
  int th = 128;
  k_pair_features<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, pr, ps, R->mbb, S->mbb, R->anchor, S->anchor,
                                                                a.chunk, a.coff, b.chunk, b.coff, R->lod[R->L - 1].foff,
                                                                S->lod[S->L - 1].foff, out, n_live);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

void mlp_forward(pj_ctx* ctx, const float* feats, int64_t n, float* out, cudaStream_t st) {
  if (n == 0) return;
  if (!ctx->mlp_ready) throw ApiError{PJ_EINVAL, "the MLP has no weights (train or load it first)"};
  int64_t tiles = (n + 15) / 16;
  unsigned g = (unsigned)std::min<int64_t>((tiles + MLP_WARPS - 1) / MLP_WARPS, (int64_t)ctx->sm_count * 8);
  k_mlp_fwd<<<g, MLP_WARPS * 32, 0, st>>>(ctx->mlp_w, feats, n, out);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

constexpr size_t MLP_GRAD_DYN = ((MLP_NW * 4 + 15) / 16) * 16 + MLP_WARPS * (2 * 16 * 64 + 16 * 16) * 2;

static void mlp_grad_launch(pj_ctx* ctx, const float* w, const float* X, const float* t, const int32_t* idx,
                            int64_t n, float scale, float* grad, float* loss, cudaStream_t st) {
  int64_t tiles = (n + 15) / 16;
  unsigned g = (unsigned)std::min<int64_t>((tiles + MLP_WARPS - 1) / MLP_WARPS, (int64_t)ctx->sm_count * 2);
  if (g < 1) g = 1;
  PJ_CK(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_GRAD_DYN));
  k_mlp_grad<<<g, MLP_WARPS * 32, MLP_GRAD_DYN, st>>>(w, X, t, idx, n, scale, grad, loss);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

static void mlp_init_host(std::vector<float>& W, uint64_t seed) {
  W.assign(MLP_NW, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> n1(0.0, std::sqrt(2.0 / 16)), n2(0.0, std::sqrt(2.0 / 64)),
      n3(0.0, std::sqrt(1.0 / 64));
  for (int i = 0; i < 64 * 16; ++i) W[MLP_W1 + i] = (float)n1(rng);
  for (int i = 0; i < 64 * 64; ++i) W[MLP_W2 + i] = (float)n2(rng);
  for (int i = 0; i < 64; ++i) W[MLP_W3 + i] = (float)n3(rng);
}

static void ensure_weights(pj_ctx* ctx) {
  if (!ctx->mlp_w) {
    note_alloc();
    PJ_CK(cudaMalloc((void**)&ctx->mlp_w, MLP_NW * sizeof(float)));
  }
}

// Adam over shuffled mini-batches of device-resident features X [n][16] and
// targets T [n].  The per-epoch permutation is drawn on the host.
static void mlp_train_dev(pj_ctx* ctx, const float* X, const float* T, int64_t n, int epochs, uint64_t seed,
                          cudaStream_t st) {
  ensure_weights(ctx);
  if (!ctx->mlp_ready) {
    std::vector<float> W;
    mlp_init_host(W, seed);
    PJ_CK(cudaMemcpyAsync(ctx->mlp_w, W.data(), MLP_NW * 4, cudaMemcpyHostToDevice, st));
    PJ_CK(cudaStreamSynchronize(st));
    ctx->mlp_ready = true;
  }
  float* opt = (float*)ws_get(ctx, WS_MLP3, (3 * MLP_NW + 1) * sizeof(float), st);
  float* grad = opt;
  float* m = opt + MLP_NW;
  float* v = opt + 2 * MLP_NW;
  PJ_CK(cudaMemsetAsync(m, 0, 2 * MLP_NW * sizeof(float), st));
  int32_t* idx = (int32_t*)ws_get(ctx, WS_FEAT, (size_t)n * 4, st);
  std::vector<int32_t> perm(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  std::mt19937_64 rng(seed ^ 0x9e3779b97f4a7c15ULL);
  const int64_t batch = std::min<int64_t>(n, 2048);
  const float lr = 3e-3f, b1 = 0.9f, b2 = 0.999f;
  int64_t step = 0;
  for (int e = 0; e < epochs; ++e) {
    std::shuffle(perm.begin(), perm.end(), rng);
    PJ_CK(cudaMemcpyAsync(idx, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st));
    PJ_CK(cudaStreamSynchronize(st));   // perm is reused by the next epoch
    for (int64_t b0 = 0; b0 < n; b0 += batch) {
      const int64_t cnt = std::min(batch, n - b0);
      PJ_CK(cudaMemsetAsync(grad, 0, MLP_NW * sizeof(float), st));
      mlp_grad_launch(ctx, ctx->mlp_w, X, T, idx + b0, cnt, 1.f / (float)cnt, grad, nullptr, st);
      ++step;
      const float c1 = 1.f / (1.f - std::pow(b1, (float)step)), c2 = 1.f / (1.f - std::pow(b2, (float)step));
      k_adam<<<(MLP_NW + 255) / 256, 256, 0, st>>>(ctx->mlp_w, m, v, grad, lr, b1, b2, c1, c2, MLP_NW);
      PJ_CK(cudaGetLastError());
      count_launch(ctx);
    }
  }
  PJ_CK(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ proposal
// The network predicts y = log1p(d) of a candidate pair from its features.

const float* propose(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, cudaStream_t st,
                     const int64_t* n_live) {
  float* X = (float*)ws_get(ctx, WS_FEAT, (size_t)n * 64, st);
  float* y = (float*)ws_get(ctx, WS_PRED, (size_t)n * 4, st);
  pair_features(ctx, R, S, (const int32_t*)ctx->ws[WS_PR].p, (const int32_t*)ctx->ws[WS_PS].p, n, X, st, n_live);
  mlp_forward(ctx, X, n, y, st);
  return y;
}

struct LodMax {
  const float4* chunkR[PJ_MAX_LODS];
  const int64_t* coffR[PJ_MAX_LODS];
  const float4* chunkS[PJ_MAX_LODS];
  const int64_t* coffS[PJ_MAX_LODS];
};

__device__ __forceinline__ float obj_hd_ph(const float4* ch, const int64_t* coff, int o) {
  float m = 0.f;
  for (int64_t c = coff[o]; c < coff[o + 1]; ++c) m = fmaxf(m, ch[3 * c].w + ch[3 * c + 1].w);
  return m;
}

// Start LoD of the undecided pairs.  Section 3.1 refines every pair LoD by
// LoD from the coarsest; skipping the coarse steps a pair cannot pass is
// this library's addition, driven by the prediction.  Step l can decide
// a pair only when its distance is far enough from tau compared with the
// Hausdorff terms of that LoD; with the per-object maxima w_l (hd + ph of r
// plus hd + ph of s), |d - tau| > w_l decides it for certain.  The pair
// starts at the coarsest step with max |x - tau| >= margin * w_l over the
// prediction interval x in [expm1(y - u), expm1(y + u)], else at full
// resolution.  Skipping steps never changes a result.
__global__ void k_start_lod(int64_t n, const int32_t* pr, const int32_t* ps, const uint8_t* status,
                            const float* pred, double tau, LodMax M, int offR, int offS, int Lmax, float margin,
                            float u, uint8_t* lod0) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (status[p] != UNDECIDED) return;
  const double y = pred[p];
  const double lo = fmax(0.0, expm1(y - u)), hi = expm1(y + u);
  const double gap = fmax(fabs(lo - tau), fabs(hi - tau));
  const int r = pr[p], s = ps[p];
  int start = Lmax - 1;
  for (int l = 0; l < Lmax - 1; ++l) {
    const int lr = max(0, l - offR), ls = max(0, l - offS);
    const float w = obj_hd_ph(M.chunkR[lr], M.coffR[lr], r) + obj_hd_ph(M.chunkS[ls], M.coffS[ls], s);
    if (gap >= (double)margin * w) {
      start = l;
      break;
    }
  }
  lod0[p] = (uint8_t)start;
}

void start_lod(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const float* pred, double tau,
               cudaStream_t st) {
  if (n == 0) return;
  LodMax M;
  for (int l = 0; l < PJ_MAX_LODS; ++l) {
    M.chunkR[l] = l < R->L ? R->lod[l].chunk : nullptr;
    M.coffR[l] = l < R->L ? R->lod[l].coff : nullptr;
    M.chunkS[l] = l < S->L ? S->lod[l].chunk : nullptr;
    M.coffS[l] = l < S->L ? S->lod[l].coff : nullptr;
  }
  const int Lmax = std::max(R->L, S->L);
  int th = 256;
  k_start_lod<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(
      n, (const int32_t*)ctx->ws[WS_PR].p, (const int32_t*)ctx->ws[WS_PS].p, (const uint8_t*)ctx->ws[WS_STATUS].p,
      pred, tau, M, Lmax - R->L, Lmax - S->L, Lmax, START_MARGIN, PRED_BAND, (uint8_t*)ctx->ws[WS_LOD0].p);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

// Training targets: y = log1p of the full-resolution distance (midpoint of
// the single-precision bracket, whose width is a few ulps).
__global__ void k_targets(int64_t n, const float* lb, const float* ub, float* t) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) t[p] = log1pf(0.5f * (lb[p] + ub[p]));
}

__global__ void k_sq_err(int64_t n, const float* y, const float* t, double* acc) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double e = 0;
  if (p < n) e = (double)(y[p] - t[p]) * (y[p] - t[p]);
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0 && e != 0) atomicAdd(acc, e);
}

}  // namespace pj

using namespace pj;

static pj_status mlp_fail(pj_ctx* ctx, pj_status s, const std::string& m) {
  if (ctx) ctx->last_error = m;
  return s;
}

#define MLP_TRY try {
#define MLP_CATCH(ctx)                                                                                    \
  }                                                                                                       \
  catch (const CudaError& e) {                                                                            \
    return mlp_fail(ctx, PJ_ECUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));                \
  }                                                                                                       \
  catch (const ApiError& e) {                                                                             \
    return mlp_fail(ctx, e.st, e.msg);                                                                    \
  }

extern "C" {

pj_status pj_mlp_set_weights(pj_ctx* ctx, const float* w1, const float* b1, const float* w2, const float* b2,
                             const float* w3, const float* b3) {
  if (!ctx || !w1 || !b1 || !w2 || !b2 || !w3 || !b3) return mlp_fail(ctx, PJ_EINVAL, "null weight");
  MLP_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  std::vector<float> W(MLP_NW);
  memcpy(&W[MLP_W1], w1, 64 * 16 * 4);
  memcpy(&W[MLP_B1], b1, 64 * 4);
  memcpy(&W[MLP_W2], w2, 64 * 64 * 4);
  memcpy(&W[MLP_B2], b2, 64 * 4);
  memcpy(&W[MLP_W3], w3, 64 * 4);
  W[MLP_B3] = b3[0];
  for (float x : W)
    if (!std::isfinite(x)) return mlp_fail(ctx, PJ_ENONFINITE, "non-finite weight");
  ensure_weights(ctx);
  PJ_CK(cudaMemcpy(ctx->mlp_w, W.data(), MLP_NW * 4, cudaMemcpyHostToDevice));
  ctx->mlp_ready = true;
  return PJ_OK;
  MLP_CATCH(ctx)
}

pj_status pj_mlp_get_weights(const pj_ctx* ctx, float* w1, float* b1, float* w2, float* b2, float* w3, float* b3) {
  if (!ctx || !ctx->mlp_ready) return PJ_EINVAL;
  std::vector<float> W(MLP_NW);
  if (cudaMemcpy(W.data(), ctx->mlp_w, MLP_NW * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PJ_ECUDA;
  if (w1) memcpy(w1, &W[MLP_W1], 64 * 16 * 4);
  if (b1) memcpy(b1, &W[MLP_B1], 64 * 4);
  if (w2) memcpy(w2, &W[MLP_W2], 64 * 64 * 4);
  if (b2) memcpy(b2, &W[MLP_B2], 64 * 4);
  if (w3) memcpy(w3, &W[MLP_W3], 64 * 4);
  if (b3) b3[0] = W[MLP_B3];
  return PJ_OK;
}

pj_status pj_mlp_save(const pj_ctx* ctx, const char* path) {
  if (!ctx || !path || !ctx->mlp_ready) return PJ_EINVAL;
  std::vector<float> W(MLP_NW);
  if (cudaMemcpy(W.data(), ctx->mlp_w, MLP_NW * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PJ_ECUDA;
  FILE* f = fopen(path, "wb");
  if (!f) return PJ_EINVAL;
  const char magic[8] = {'P', 'J', 'M', 'L', 'P', '1', 0, 0};
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(W.data(), 4, MLP_NW, f) == (size_t)MLP_NW;
  fclose(f);
  return ok ? PJ_OK : PJ_EINVAL;
}

pj_status pj_mlp_load(pj_ctx* ctx, const char* path) {
  if (!ctx || !path) return PJ_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return mlp_fail(ctx, PJ_EINVAL, "cannot open the weight file");
  char magic[8];
  std::vector<float> W(MLP_NW);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "PJMLP1", 6) == 0 &&
            fread(W.data(), 4, MLP_NW, f) == (size_t)MLP_NW;
  fclose(f);
  if (!ok) return mlp_fail(ctx, PJ_EINVAL, "not a weight file of this library");
  return pj_mlp_set_weights(ctx, &W[MLP_W1], &W[MLP_B1], &W[MLP_W2], &W[MLP_B2], &W[MLP_W3], &W[MLP_B3]);
}

pj_status pj_mlp_forward(pj_ctx* ctx, const float* feats, int64_t n, float* out, void* cuda_stream) {
  if (!ctx || n < 0 || (n > 0 && (!feats || !out))) return mlp_fail(ctx, PJ_EINVAL, "bad mlp_forward arguments");
  MLP_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  mlp_forward(ctx, feats, n, out, st);
  PJ_CK(cudaStreamSynchronize(st));
  return PJ_OK;
  MLP_CATCH(ctx)
}

pj_status pj_mlp_grad(pj_ctx* ctx, const float* feats, const float* target, int64_t n, float* loss, float* g_w1,
                      float* g_b1, float* g_w2, float* g_b2, float* g_w3, float* g_b3, void* cuda_stream) {
  if (!ctx || n <= 0 || !feats || !target) return mlp_fail(ctx, PJ_EINVAL, "bad mlp_grad arguments");
  if (!ctx->mlp_ready) return mlp_fail(ctx, PJ_EINVAL, "the MLP has no weights");
  MLP_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  float* grad = (float*)ws_get(ctx, WS_MLP3, (MLP_NW + 1) * sizeof(float), st);
  PJ_CK(cudaMemsetAsync(grad, 0, (MLP_NW + 1) * sizeof(float), st));
  mlp_grad_launch(ctx, ctx->mlp_w, feats, target, nullptr, n, 1.f / (float)n, grad, grad + MLP_NW, st);
  if (loss) PJ_CK(cudaMemcpyAsync(loss, grad + MLP_NW, 4, cudaMemcpyDeviceToDevice, st));
  struct {
    float* dst;
    int off, cnt;
  } parts[6] = {{g_w1, MLP_W1, 1024}, {g_b1, MLP_B1, 64}, {g_w2, MLP_W2, 4096},
                {g_b2, MLP_B2, 64},   {g_w3, MLP_W3, 64},  {g_b3, MLP_B3, 1}};
  for (auto& p : parts)
    if (p.dst) PJ_CK(cudaMemcpyAsync(p.dst, grad + p.off, p.cnt * 4, cudaMemcpyDeviceToDevice, st));
  PJ_CK(cudaStreamSynchronize(st));
  return PJ_OK;
  MLP_CATCH(ctx)
}

pj_status pj_mlp_train(pj_ctx* ctx, const float* feats, const float* target, int64_t n, int epochs, uint64_t seed) {
  if (!ctx || n <= 0 || !feats || !target || epochs < 1) return mlp_fail(ctx, PJ_EINVAL, "bad mlp_train arguments");
  MLP_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  for (int64_t i = 0; i < 16 * n; ++i)
    if (!std::isfinite(feats[i])) return mlp_fail(ctx, PJ_ENONFINITE, "non-finite feature");
  float* X = (float*)ws_get(ctx, WS_MLP, (size_t)n * 16 * 4, st);
  float* T = (float*)ws_get(ctx, WS_MLP2, (size_t)n * 4, st);
  PJ_CK(cudaMemcpyAsync(X, feats, (size_t)n * 64, cudaMemcpyHostToDevice, st));
  PJ_CK(cudaMemcpyAsync(T, target, (size_t)n * 4, cudaMemcpyHostToDevice, st));
  mlp_train_dev(ctx, X, T, n, epochs, seed, st);
  return PJ_OK;
  MLP_CATCH(ctx)
}

// Each pair's threshold set to its anchor distance (an upper bound of d,
// rounded up): units and facet pairs farther apart cannot hold the minimum.
__global__ void k_thr_from_ub(int64_t n, const double* anc_ub, float* thr) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) thr[p] = __double2float_ru(anc_ub[p]);
}

pj_status pj_mlp_fit(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, int64_t max_pairs,
                     int epochs, uint64_t seed, double* rmse) {
  if (!ctx || !R || !S || !q || max_pairs < 16 || epochs < 1) return mlp_fail(ctx, PJ_EINVAL, "bad mlp_fit arguments");
  if (R->streamed || S->streamed) return mlp_fail(ctx, PJ_EINVAL, "streamed sets are not addressable");
  if (q->pred == PJ_KNN && (q->k < 1 || q->k > 32)) return mlp_fail(ctx, PJ_EINVAL, "k out of range");
  if (q->pred == PJ_WITHIN && !(q->tau >= 0.0)) return mlp_fail(ctx, PJ_EINVAL, "tau must be >= 0");
  MLP_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  (void)cudaGetLastError();
  cudaStream_t st = ctx->stream;
  PJ_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  FilterOut fo = q->pred == PJ_KNN ? filter_knn(ctx, R, S, q->k, st)
                                   : filter_within(ctx, R, S, q->pred == PJ_INTERSECT ? 0.0 : q->tau, st);
  const int64_t nc = fo.n_pairs;
  if (nc < 16) return mlp_fail(ctx, PJ_EINVAL, "the query has fewer than 16 candidate pairs to learn from");
  // a seeded sample of the candidates (all of them when they fit)
  std::vector<int32_t> hr(nc), hs(nc);
  PJ_CK(cudaMemcpyAsync(hr.data(), ctx->ws[WS_PR].p, nc * 4, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaMemcpyAsync(hs.data(), ctx->ws[WS_PS].p, nc * 4, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaStreamSynchronize(st));
  std::mt19937_64 rng(seed * 0x2545f4914f6cdd1dULL + 1);
  std::vector<int64_t> pick(nc);
  for (int64_t i = 0; i < nc; ++i) pick[i] = i;
  std::shuffle(pick.begin(), pick.end(), rng);
  const int64_t n = std::min(nc, max_pairs);
  std::vector<int32_t> sr(n), ss(n);
  for (int64_t i = 0; i < n; ++i) {
    sr[i] = hr[pick[i]];
    ss[i] = hs[pick[i]];
  }
  auto dpr = (int32_t*)ws_get(ctx, WS_PR, n * 4, st);
  auto dps = (int32_t*)ws_get(ctx, WS_PS, n * 4, st);
  PJ_CK(cudaMemcpyAsync(dpr, sr.data(), n * 4, cudaMemcpyHostToDevice, st));
  PJ_CK(cudaMemcpyAsync(dps, ss.data(), n * 4, cudaMemcpyHostToDevice, st));
  // labels: full-resolution distances from the refinement kernel, with
  // units pruned against each pair's anchor distance (the minimum lies in
  // a unit within it)
  setup_pairs(ctx, R, S, n, 0.0, false, st);
  {
    const int th = 256;
    k_thr_from_ub<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, (const double*)ctx->ws[WS_ANCUB].p,
                                                                 (float*)ctx->ws[WS_THR].p);
    PJ_CK(cudaGetLastError());
    count_launch(ctx);
  }
  StepSpec sp;
  sp.lodR = R->L - 1;
  sp.lodS = S->L - 1;
  sp.full = true;
  sp.fp64 = false;
  sp.cull = true;
  sp.want = UNDECIDED;
  sp.step = STEP_ALL;
  sp.exact_cross = true;
  init_bounds(ctx, n, sp, st);
  UnitCount uc = build_tiles(ctx, R, S, n, sp, st);
  run_refine(ctx, R, S, uc, sp, st);
  float* X = (float*)ws_get(ctx, WS_MLP, (size_t)n * 64, st);
  float* T = (float*)ws_get(ctx, WS_MLP2, (size_t)n * 4, st);
  pair_features(ctx, R, S, dpr, dps, n, X, st);
  int th = 256;
  k_targets<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, (const float*)ctx->ws[WS_LB].p,
                                                          (const float*)ctx->ws[WS_UB].p, T);
  PJ_CK(cudaGetLastError());
  count_launch(ctx);
  int herr = 0;
  PJ_CK(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaStreamSynchronize(st));
  if (herr & ERR_MBAR_TIMEOUT) return mlp_fail(ctx, PJ_ETIMEOUT, "a device wait hit its limit");
  // train on the first 90 %, report the RMSE (log1p units) on the rest
  const int64_t nv = std::max<int64_t>(1, n / 10), ntr = n - nv;
  ctx->mlp_ready = false;   // fresh weights for this workload
  mlp_train_dev(ctx, X, T, ntr, epochs, seed, st);
  float* yv = (float*)ws_get(ctx, WS_PRED, (size_t)nv * 4, st);
  mlp_forward(ctx, X + 16 * ntr, nv, yv, st);
  double* acc = (double*)ws_get(ctx, WS_MISC5, 8, st);
  PJ_CK(cudaMemsetAsync(acc, 0, 8, st));
  k_sq_err<<<(unsigned)((nv + th - 1) / th), th, 0, st>>>(nv, yv, T + ntr, acc);
  PJ_CK(cudaGetLastError());
  count_launch(ctx);
  double se = 0;
  PJ_CK(cudaMemcpyAsync(&se, acc, 8, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaStreamSynchronize(st));
  if (rmse) *rmse = std::sqrt(se / (double)nv);
  return PJ_OK;
  MLP_CATCH(ctx)
}

pj_status pj_pair_features(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr, const int32_t* ps,
                           int64_t n, float* out_dev) {
  if (!ctx || !R || !S || n < 0 || (n > 0 && (!pr || !ps || !out_dev)))
    return mlp_fail(ctx, PJ_EINVAL, "bad pair_features arguments");
  for (int64_t i = 0; i < n; ++i)
    if (pr[i] < 0 || pr[i] >= R->n || ps[i] < 0 || ps[i] >= S->n) return mlp_fail(ctx, PJ_EBOUNDS, "pair id out of range");
  if (n == 0) return PJ_OK;
  MLP_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  int32_t* dpr = (int32_t*)ws_get(ctx, WS_MLP, (size_t)n * 8, st);
  int32_t* dps = dpr + n;
  PJ_CK(cudaMemcpyAsync(dpr, pr, n * 4, cudaMemcpyHostToDevice, st));
  PJ_CK(cudaMemcpyAsync(dps, ps, n * 4, cudaMemcpyHostToDevice, st));
  pair_features(ctx, R, S, dpr, dps, n, out_dev, st);
  PJ_CK(cudaStreamSynchronize(st));
  return PJ_OK;
  MLP_CATCH(ctx)
}

}  // extern "C"
