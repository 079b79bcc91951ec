// Shared device helpers of the rmc library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>

namespace rmc {

constexpr int kWarp = 32;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = kWarp / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = kWarp / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Double-float ("double-FP32") arithmetic: a value is the unevaluated sum
// hi + lo of two floats (48 significant bits).  A product's rounding error is
// recovered exactly with an FMA (Dekker's product, FMA form) and an addition
// into an accumulator keeps its error by Knuth's TwoSum, so one multiply-add
// takes 12 FP32 instructions; the lo*lo term is dropped (2^-48 relative).
__device__ __forceinline__ float2 df_split(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}
__device__ __forceinline__ double df_value(float2 v) { return (double)v.x + (double)v.y; }

// (s, t) += a * b
__device__ __forceinline__ void df_mac(float& s, float& t, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float u = s + p;
  const float bp = u - s;
  const float err = (s - (u - bp)) + (p - bp);
  s = u;
  t += err + e;
}

// Block-wide sum; `scratch` holds >= 32 elements; all threads get the result.
template <typename T>
__device__ T block_sum(T v, T* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  T r = (threadIdx.x < nw) ? scratch[threadIdx.x] : T(0);
  if (wid == 0) r = warp_sum(r);
  if (threadIdx.x == 0) scratch[0] = r;
  __syncthreads();
  r = scratch[0];
  __syncthreads();
  return r;
}

template <typename T>
__device__ T block_max(T v, T* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  T r = (threadIdx.x < nw) ? scratch[threadIdx.x] : T(-INFINITY);
  if (wid == 0) r = warp_max(r);
  if (threadIdx.x == 0) scratch[0] = r;
  __syncthreads();
  r = scratch[0];
  __syncthreads();
  return r;
}

inline unsigned ceil_div(long a, long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace rmc
