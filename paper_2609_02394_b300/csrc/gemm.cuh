// Tiled SIMT GEMM template with pluggable epilogues (FP32 FMA / FP64 DFMA).
//
//   acc[m][n] = sum_k op(A)[m][k] * op(B)[k][n]     (per batch z, per K split)
//
// op(A)[m][k] = A[m*lda + k] (TA = false) or A[k*lda + m] (TA = true);
// op(B)[k][n] = B[k*ldb + n] (TB = false) or B[n*ldb + k] (TB = true).
// The epilogue functor receives (batch, split, m, n, acc) for every in-range
// output and decides where and how to write it, so permuted layouts (the two
// stages of the Kronecker product), scaled accumulations and split-K partial
// buffers all use the same main loop.  Out-of-range tile elements are zero
// filled, so any M, N, K (ragged tails included) is valid.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace rmc {

struct GemmShape {
  int M, N, K;
  long lda, ldb;
  long batch_stride_a, batch_stride_b;
  int k_splits;  // >= 1; split s covers K range [s*Ks, (s+1)*Ks)
  const int* skip = nullptr;  // if non-null and *skip != 0 the launch does nothing
};

// With DF (T = double only) the tiles are held as (hi, lo) float pairs and
// the products are accumulated in double-float arithmetic on the FP32 pipe
// (see common.cuh); the epilogue receives hi + lo as a double.
template <typename T, int BM, int BN, int BK, int TM, int TN, bool TA, bool TB, class Epi, bool DF = false>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_kernel(const T* __restrict__ A, const T* __restrict__ B, GemmShape s, Epi epi) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int RY = BM / TM;  // thread rows
  constexpr int RX = BN / TN;  // thread cols
  static_assert(!DF || sizeof(T) == 8, "double-float products take FP64 data");
  using ST = std::conditional_t<DF, float2, T>;
  if (s.skip && *s.skip) return;
  __shared__ ST As[BK][BM + 1];
  __shared__ ST Bs[BK][BN + 1];

  const int batch = blockIdx.z / s.k_splits;
  const int split = blockIdx.z % s.k_splits;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int Ks = (s.K + s.k_splits - 1) / s.k_splits;
  const int kbeg = split * Ks;
  const int kend = min(s.K, kbeg + Ks);
  A += (long)batch * s.batch_stride_a;
  B += (long)batch * s.batch_stride_b;

  const int tid = threadIdx.x;
  const int ty = tid / RX, tx = tid % RX;
  using AT = std::conditional_t<DF, float, T>;
  AT acc[TM][TN], acc_lo[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = acc_lo[i][j] = AT(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // A tile: BM x BK
#pragma unroll
    for (int e = tid; e < BM * BK; e += NT) {
      int mm, kk;
      if (TA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      T v = T(0);
      if (gm < s.M && gk < kend) v = TA ? A[(long)gk * s.lda + gm] : A[(long)gm * s.lda + gk];
      if constexpr (DF) As[kk][mm] = df_split(v);
      else As[kk][mm] = v;
    }
    // B tile: BK x BN
#pragma unroll
    for (int e = tid; e < BN * BK; e += NT) {
      int nn, kk;
      if (TB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      const int gn = n0 + nn, gk = k0 + kk;
      T v = T(0);
      if (gn < s.N && gk < kend) v = TB ? B[(long)gn * s.ldb + gk] : B[(long)gk * s.ldb + gn];
      if constexpr (DF) Bs[kk][nn] = df_split(v);
      else Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      ST a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * RY];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * RX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          if constexpr (DF) df_mac(acc[i][j], acc_lo[i][j], a[i], b[j]);
          else acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + i * RY;
    if (gm >= s.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + j * RX;
      if (gn >= s.N) continue;
      if constexpr (DF) epi(batch, split, gm, gn, (T)((double)acc[i][j] + (double)acc_lo[i][j]));
      else epi(batch, split, gm, gn, acc[i][j]);
    }
  }
}

// Plain store epilogue: C[batch*sc + m*ldc + n] = alpha*acc + beta*C (beta == 0
// never reads C).  With k_splits > 1 the caller passes a partial buffer and
// split stride instead and reduces afterwards.
template <typename T>
struct EpiStore {
  T* C;
  long ldc, batch_stride, split_stride;
  T alpha, beta;
  __device__ void operator()(int b, int sp, int m, int n, T acc) const {
    T* p = C + (long)b * batch_stride + (long)sp * split_stride + (long)m * ldc + n;
    *p = (beta == T(0)) ? alpha * acc : alpha * acc + beta * (*p);
  }
};

// Sum `splits` partial M x N buffers (stride split_stride) into C with
// C = alpha * sum + beta * C.  Also used with splits == 1 as a scaled copy.
template <typename T>
__global__ void reduce_splits_kernel(const T* __restrict__ P, int splits, long split_stride,
                                     int M, int N, T* C, long ldc, T alpha, T beta, int symmetrize) {
  const long total = (long)M * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int m = (int)(e / N), n = (int)(e % N);
    T acc = T(0);
    for (int sp = 0; sp < splits; ++sp) acc += P[sp * split_stride + e];
    if (symmetrize && m != n) {
      T acc2 = T(0);
      const long e2 = (long)n * N + m;
      for (int sp = 0; sp < splits; ++sp) acc2 += P[sp * split_stride + e2];
      acc = T(0.5) * (acc + acc2);
    }
    T* p = C + (long)m * ldc + n;
    *p = (beta == T(0)) ? alpha * acc : alpha * acc + beta * (*p);
  }
}

// Launch helper.  Tile presets: FP32 64x64x16 / 4x4, FP64 64x64x8 / 4x4,
// small 32x32 / 2x2 (for the b x b products of the Rayleigh-Ritz steps).
template <typename T, int BM, int BN, int BK, int TM, int TN, bool TA, bool TB, class Epi, bool DF = false>
inline void launch_gemm(const T* A, const T* B, const GemmShape& s, int batches, const Epi& epi,
                        cudaStream_t st) {
  dim3 grid(ceil_div(s.N, BN), ceil_div(s.M, BM), batches * s.k_splits);
  gemm_kernel<T, BM, BN, BK, TM, TN, TA, TB, Epi, DF><<<grid, (BM / TM) * (BN / TN), 0, st>>>(A, B, s, epi);
}

}  // namespace rmc
