// Fused Kronecker-form products with H_eff (Eq. (7)) for blocks whose vectors
// fit in shared memory: the whole Chebyshev filter of one subspace iteration
// (Zhou and Saad's scaled three-term recurrence), or one plain product H X,
// in a single launch.
//
// Each vector of the block is a kA x kB matrix and every step of the filter
// acts on the vectors independently, so a CTA owns `vpc` vectors for the
// whole polynomial: the two most recent terms of the recurrence and the
// stage-1 intermediate stay in shared memory, the operators are staged there
// once (FP32) or read through L1/L2 (FP64), and only the input block and the
// normalised result cross HBM.  The multi-launch form (two GEMM launches per
// degree, each term written to and read back from HBM) remains for blocks
// that do not fit and for the deflated filter of the locked iteration.
//
// Per vector v and step, with Y the current term:
//   stage 1: T[(j, a), (v, b)] = sum_b' Y[v][a][b'] B_j[b][b']
//   stage 2: (H Y)[v][a][b]    = (EA[a] + EB[b]) Y[v][a][b] + sum_{j,a'} Acat[a][(j,a')] T[(j,a'), (v,b)]
// where Acat folds the coupling coefficients into the A-side operators.
#pragma once

#include "common.cuh"

namespace rmc {

constexpr int kFusedThreads = 256;                // 16 x 16 threads, 4 x 4 outputs each per 64 x 64 tile
constexpr size_t kFusedSmemLimit = 200u * 1024u;  // dynamic shared memory of one CTA

struct FusedArgs {
  int kA, kB, n_ops, nv;  // block of nv vectors of length kA * kB
  int vpc;                // vectors per CTA
  int deg;                // polynomial degree (>= 1) of the filter; 0: plain product
  int compute_hx;         // 1: H X is formed in the kernel, HX is not read
  int ops_in_smem;        // operators staged in shared memory
  double e, c, sigma1;    // filter: half width and centre of the damped interval, e / (theta0 - c)
};

// C(m, n) = sum_k A(m, k) B(k, n) for an M x N output, A(m, k) = A[m*sam + k*sak],
// B(k, n) = B[k*sbk + n*sbn], by all threads of the CTA (16 x 16 thread grid,
// 4 x 4 register tile per thread per 64 x 64 output tile).  Out-of-range rows
// and columns read a clamped in-range element and are not stored.
template <typename T, class Epi>
__device__ __forceinline__ void cta_gemm(int M, int N, int K, const T* A, int sam, int sak, const T* B, int sbk,
                                         int sbn, const Epi& epi) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int m0 = 0; m0 < M; m0 += 64) {
    for (int n0 = 0; n0 < N; n0 += 64) {
      int ar[4], bc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ar[i] = min(m0 + ty + 16 * i, M - 1) * sam;
        bc[i] = min(n0 + tx + 16 * i, N - 1) * sbn;
      }
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
      for (int k = 0; k < K; ++k) {
        T a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = A[ar[i] + k * sak];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = B[k * sbk + bc[j]];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = n0 + tx + 16 * j;
          if (n < N) epi(m, n, acc[i][j]);
        }
      }
    }
  }
}

// Stage-1 epilogue: T[((j*kA + a)*nvl + v)*kB + b] for m = v*kA + a, n = j*kB + b.
template <typename T>
struct FusedEpi1 {
  T* Ts;
  int kA, kB, nvl;
  __device__ void operator()(int m, int n, T acc) const {
    const int v = m / kA, a = m - v * kA, j = n / kB, b = n - j * kB;
    Ts[((j * kA + a) * nvl + v) * kB + b] = acc;
  }
};

// Stage-2 epilogue of a recurrence step: with x = Ycur and z = Yold at the
// same element, Yold <- alpha * (acc + (EA[a] + EB[b]) x) + beta * x + gamma * z
// (the new term overwrites the one two steps back; gamma = 0 ignores z).
template <typename T>
struct FusedEpi2 {
  const T* Ycur;
  T* Yold;
  const T* EA;
  const T* EB;
  int kA, kB;
  T alpha, beta, gamma;
  __device__ void operator()(int a, int n, T acc) const {
    const int v = n / kB, b = n - v * kB;
    const int idx = (v * kA + a) * kB + b;
    const T x = Ycur[idx];
    T y = alpha * (acc + (EA[a] + EB[b]) * x) + beta * x;
    if (gamma != T(0)) y += gamma * Yold[idx];
    Yold[idx] = y;
  }
};

template <typename T>
__device__ __forceinline__ void fused_product(const FusedArgs& p, int nvl, const T* Ysrc, T* Ts, const T* Aop,
                                              const T* Bop, int bsk, int bsn, const FusedEpi2<T>& e2) {
  const int kA = p.kA, kB = p.kB, no = p.n_ops;
  if (no > 0) {
    cta_gemm<T>(nvl * kA, no * kB, kB, Ysrc, kB, 1, Bop, bsk, bsn, FusedEpi1<T>{Ts, kA, kB, nvl});
    __syncthreads();
  }
  cta_gemm<T>(kA, nvl * kB, no * kA, Aop, no * kA, 1, Ts, nvl * kB, 1, e2);
  __syncthreads();
}

// One launch: Out = normalised p(H) X (deg >= 1) or Out = H X (deg == 0).
// X and Out may be the same array (each CTA reads its vectors before it
// writes them).  HX is read only when compute_hx == 0 and deg >= 1.
template <typename T>
__global__ void __launch_bounds__(kFusedThreads)
    cheb_fused_kernel(const T* X, const T* __restrict__ HX, const T* __restrict__ EA, const T* __restrict__ EB,
                      const T* __restrict__ Acat, const T* __restrict__ Bcat, T* Out, FusedArgs p) {
  extern __shared__ __align__(16) unsigned char fused_smem[];
  T* sm = reinterpret_cast<T*>(fused_smem);
  const int kA = p.kA, kB = p.kB, no = p.n_ops;
  const int n = kA * kB;
  const int v0 = blockIdx.x * p.vpc;
  const int nvl = min(p.vpc, p.nv - v0);
  if (nvl <= 0) return;
  T* Yp = sm;                      // term k-1 (starts as X)
  T* Yc = Yp + (size_t)p.vpc * n;  // term k
  T* Ts = Yc + (size_t)p.vpc * n;  // stage-1 intermediate, n_ops * vpc * n
  T* As = Ts + (size_t)no * p.vpc * n;
  T* Bt = As + (size_t)kA * no * kA;
  T* red = p.ops_in_smem ? Bt + (size_t)kB * no * kB : As;
  const long base = (long)v0 * n;
  const int cnt = nvl * n;
  const T s1e = T(p.sigma1 / p.e);
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const T x = X[base + i];
    Yp[i] = x;
    if (!p.compute_hx && p.deg >= 1) Yc[i] = s1e * (HX[base + i] - T(p.c) * x);
  }
  const T* Aop = Acat;
  const T* Bop = Bcat;
  int bsk = 1, bsn = kB;  // B(k, n') = Bcat[n' * kB + k]
  if (p.ops_in_smem && no > 0) {
    for (int i = threadIdx.x; i < kA * no * kA; i += blockDim.x) As[i] = Acat[i];
    for (int i = threadIdx.x; i < no * kB * kB; i += blockDim.x) {
      const int r = i / kB, k = i - r * kB;  // Bcat[r][k] -> Bt[k][r]
      Bt[k * (no * kB) + r] = Bcat[i];
    }
    Aop = As;
    Bop = Bt;
    bsk = no * kB;
    bsn = 1;
  }
  __syncthreads();
  if (p.compute_hx || p.deg == 0) {
    // Yc = a1 * (H Yp) + b1 * Yp: the first filter term, or the plain product
    const T a1 = p.deg == 0 ? T(1) : s1e;
    const T b1 = p.deg == 0 ? T(0) : T(-p.c) * s1e;
    fused_product<T>(p, nvl, Yp, Ts, Aop, Bop, bsk, bsn, FusedEpi2<T>{Yp, Yc, EA, EB, kA, kB, a1, b1, T(0)});
  }
  double sigma = p.sigma1;
  const double tau = 2.0 / p.sigma1;
  for (int d = 2; d <= p.deg; ++d) {
    const double s1 = 1.0 / (tau - sigma);
    fused_product<T>(p, nvl, Yc, Ts, Aop, Bop, bsk, bsn,
                     FusedEpi2<T>{Yc, Yp, EA, EB, kA, kB, T(2 * s1 / p.e), T(-2 * s1 * p.c / p.e), T(-sigma * s1)});
    T* t = Yp;  // the new term was written over the old one
    Yp = Yc;
    Yc = t;
    sigma = s1;
  }
  if (p.deg == 0) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) Out[base + i] = Yc[i];
    return;
  }
  for (int v = 0; v < nvl; ++v) {
    const T* y = Yc + (size_t)v * n;
    T s = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += y[i] * y[i];
    s = block_sum(s, red);
    const T inv = s > T(0) ? T(1) / sqrt(s) : T(0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) Out[base + (long)v * n + i] = y[i] * inv;
  }
}


// ---------------------------------------------------------------------------
// FP32 fused filter with k-major operands and 128-bit shared-memory loads.
//
// In cta_gemm above a thread's four rows are 16 apart, so every multiply-add
// step reads eight scalars (and the rows' stride puts two of them in one bank)
// for sixteen FMAs: the kernel is bound by shared-memory wavefronts at a
// fraction of the FMA pipe.  Here every operand is stored k-major (row k holds
// the whole m or n range), a thread owns a block of adjacent rows and columns,
// and one k step is one vector load of A^T, one of B and a block of FMAs
// (cta_gemm_v4).  Layouts (floats, row strides padded to multiples of 4 so every float4
// is 16-byte aligned; a stride that is a multiple of 32 gets 4 more, which
// spreads the transposing loads and stores over the banks):
//   Y  [b][M1p]            vector v's element (a, b) at b * M1p + v * kA + a
//   Ts [(j, a)][N2p]       stage-1 output, column v * kB + b
//   As [(j, a')][kAp]      coef_j A_j[a][a'] at row j * kA + a', column a
//   Bt [b'][N1p]           B_j[b][b'] at column j * kB + b
// ---------------------------------------------------------------------------
struct V4Layout {
  int M1p, N1p, N2p, kAp;
  size_t y, ts, as, bt;  // floats per buffer
  size_t bytes;          // whole dynamic shared memory, reduction scratch included
};

__host__ __device__ inline int v4_pad(int x) {
  int p = (x + 3) & ~3;
  if ((p & 31) == 0) p += 4;
  return p;
}

__host__ __device__ inline V4Layout v4_layout(int kA, int kB, int no, int vpc) {
  V4Layout L;
  L.M1p = v4_pad(vpc * kA);
  L.N1p = v4_pad(no * kB);
  L.N2p = v4_pad(vpc * kB);
  L.kAp = (kA + 3) & ~3;
  L.y = (size_t)kB * L.M1p;
  L.ts = (size_t)no * kA * L.N2p;
  L.as = (size_t)no * kA * L.kAp;
  L.bt = (size_t)kB * L.N1p;
  L.bytes = sizeof(float) * (2 * L.y + L.ts + L.as + L.bt + 32);
  return L;
}

// C(m, n) = sum_k At[k * lda + m] * Bk[k * ldb + n] for an M x N output, by the
// kV4Threads = 512 threads of the CTA in 64 x 64 tiles: a warp owns four
// adjacent rows (one float4 of A^T a step, the same for every lane: a
// broadcast), its lanes two adjacent columns each (one float2 of B; the warp
// reads 256 contiguous bytes).  Sixteen warps a CTA hide the shared-memory and
// FMA latency that eight could not.  lda and ldb are multiples of 4; a vector
// whose first row (column) is in range lies wholly inside the padded row, and
// out-of-range blocks read zeros.
constexpr int kV4Threads = 512;

template <class Epi>
__device__ __forceinline__ void cta_gemm_v4(int M, int N, int K, const float* At, int lda, const float* Bk, int ldb,
                                            const Epi& epi) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int m0 = 0; m0 < M; m0 += 64) {
    for (int n0 = 0; n0 < N; n0 += 64) {
      const int mr = m0 + 4 * ty, nc = n0 + 2 * tx;
      const bool am = mr < M, bn = nc < N;
      float acc[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = 0.f;
      const float4* ap = reinterpret_cast<const float4*>(At + mr);
      const float2* bp = reinterpret_cast<const float2*>(Bk + nc);
      const int sa = lda >> 2, sb = ldb >> 1;
#pragma unroll 4
      for (int k = 0; k < K; ++k) {
        const float4 a = am ? ap[k * sa] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 b = bn ? bp[k * sb] : make_float2(0.f, 0.f);
        const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          acc[i][0] = fmaf(av[i], b.x, acc[i][0]);
          acc[i][1] = fmaf(av[i], b.y, acc[i][1]);
        }
      }
      if (am && bn) epi.block(mr, nc, M, N, acc);
    }
  }
}

// The epilogues take a thread's whole 4 x 2 block (rows m0.., columns n0..,
// clipped to M x N) and split m and n into their (vector, index) parts once,
// stepping them across the block.
struct V4Epi1 {  // Ts[(j * kA + a) * N2p + v * kB + b] for m = v * kA + a, n = j * kB + b
  float* Ts;
  int kA, kB, N2p;
  __device__ void block(int m0, int n0, int M, int N, const float (&acc)[4][2]) const {
    int v = m0 / kA, a = m0 - v * kA;
    const int j0 = n0 / kB, b0 = n0 - j0 * kB;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (m0 + i < M) {
        int j = j0, b = b0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (n0 + c < N) Ts[(j * kA + a) * N2p + v * kB + b] = acc[i][c];
          if (++b == kB) { b = 0; ++j; }
        }
      }
      if (++a == kA) { a = 0; ++v; }
    }
  }
};

struct V4Epi2 {  // Yold <- alpha (acc + (EA[a] + EB[b]) x) + beta x + gamma z at (v, a, b)
  const float* Ycur;
  float* Yold;
  const float* EA;
  const float* EB;
  int kA, kB, M1p;
  float alpha, beta, gamma;
  __device__ void block(int a0, int n0, int M, int N, const float (&acc)[4][2]) const {
    const int v0 = n0 / kB, b0 = n0 - v0 * kB;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int a = a0 + i;
      if (a >= M) break;
      const float ea = EA[a];
      int v = v0, b = b0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (n0 + c < N) {
          const int idx = b * M1p + v * kA + a;
          const float x = Ycur[idx];
          float y = alpha * (acc[i][c] + (ea + EB[b]) * x) + beta * x;
          if (gamma != 0.f) y += gamma * Yold[idx];
          Yold[idx] = y;
        }
        if (++b == kB) { b = 0; ++v; }
      }
    }
  }
};

// One launch: Out = normalised p(H) X (deg >= 1) or Out = H X (deg == 0), as
// cheb_fused_kernel<float>, with both operators staged in shared memory.
__global__ void __launch_bounds__(kV4Threads)
    cheb_fused_v4_kernel(const float* X, const float* __restrict__ HX, const float* __restrict__ EA,
                         const float* __restrict__ EB, const float* __restrict__ Acat,
                         const float* __restrict__ Bcat, float* Out, FusedArgs p) {
  extern __shared__ __align__(16) unsigned char fused_smem[];
  float* sm = reinterpret_cast<float*>(fused_smem);
  const int kA = p.kA, kB = p.kB, no = p.n_ops;
  const int n = kA * kB;
  const int v0 = blockIdx.x * p.vpc;
  const int nvl = min(p.vpc, p.nv - v0);
  if (nvl <= 0) return;
  const V4Layout L = v4_layout(kA, kB, no, p.vpc);
  float* Yp = sm;
  float* Yc = Yp + L.y;
  float* Ts = Yc + L.y;
  float* As = Ts + L.ts;
  float* Bt = As + L.as;
  float* red = Bt + L.bt;
  const long base = (long)v0 * n;
  const int cnt = nvl * n;
  const float s1e = (float)(p.sigma1 / p.e);
  // zero every buffer once, so the padding a float4 may cover holds finite values
  for (int i = threadIdx.x; i < (int)(2 * L.y + L.ts + L.as + L.bt); i += blockDim.x) sm[i] = 0.f;
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {  // global (v, a, b) -> Y[b][v kA + a]
    const int v = i / n, r = i - v * n, a = r / kB, b = r - a * kB;
    const int idx = b * L.M1p + v * kA + a;
    const float x = X[base + i];
    Yp[idx] = x;
    if (!p.compute_hx && p.deg >= 1) Yc[idx] = s1e * (HX[base + i] - (float)p.c * x);
  }
  for (int i = threadIdx.x; i < kA * no * kA; i += blockDim.x) {  // Acat[a][(j, a')] -> As[(j, a')][a]
    const int a = i / (no * kA), k = i - a * (no * kA);
    As[k * L.kAp + a] = Acat[i];
  }
  for (int i = threadIdx.x; i < no * kB * kB; i += blockDim.x) {  // Bcat[(j, b)][b'] -> Bt[b'][(j, b)]
    const int r = i / kB, k = i - r * kB;
    Bt[k * L.N1p + r] = Bcat[i];
  }
  __syncthreads();
  auto product = [&](const float* Ysrc, const V4Epi2& e2) {
    if (no > 0) {
      cta_gemm_v4(nvl * kA, no * kB, kB, Ysrc, L.M1p, Bt, L.N1p, V4Epi1{Ts, kA, kB, L.N2p});
      __syncthreads();
    }
    cta_gemm_v4(kA, nvl * kB, no * kA, As, L.kAp, Ts, L.N2p, e2);
    __syncthreads();
  };
  if (p.compute_hx || p.deg == 0) {
    const float a1 = p.deg == 0 ? 1.f : s1e;
    const float b1 = p.deg == 0 ? 0.f : (float)(-p.c) * s1e;
    product(Yp, V4Epi2{Yp, Yc, EA, EB, kA, kB, L.M1p, a1, b1, 0.f});
  }
  double sigma = p.sigma1;
  const double tau = 2.0 / p.sigma1;
  for (int d = 2; d <= p.deg; ++d) {
    const double s1 = 1.0 / (tau - sigma);
    product(Yc, V4Epi2{Yc, Yp, EA, EB, kA, kB, L.M1p, (float)(2 * s1 / p.e), (float)(-2 * s1 * p.c / p.e),
                       (float)(-sigma * s1)});
    float* t = Yp;  // the new term was written over the old one
    Yp = Yc;
    Yc = t;
    sigma = s1;
  }
  if (p.deg == 0) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int v = i / n, r = i - v * n, a = r / kB, b = r - a * kB;
      Out[base + i] = Yc[b * L.M1p + v * kA + a];
    }
    return;
  }
  for (int v = 0; v < nvl; ++v) {
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int a = i / kB, b = i - a * kB;
      const float y = Yc[b * L.M1p + v * kA + a];
      s += y * y;
    }
    s = block_sum(s, red);
    const float inv = s > 0.f ? 1.f / sqrtf(s) : 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int a = i / kB, b = i - a * kB;
      Out[base + (long)v * n + i] = Yc[b * L.M1p + v * kA + a] * inv;
    }
  }
}

// ---------------------------------------------------------------------------
// The same fused filter for FP64 data in double-FP32 arithmetic, for the FP64
// refinement of the mixed paths.  This part's FP64 pipe issues ~1.9 DFMA per
// clock per SM against 128 FP32 FMAs, so FP64-accurate products are formed on
// the FP32 pipe instead: every value is an unevaluated sum hi + lo of two
// floats (a "double-float", 48 significant bits), a product's rounding error
// is recovered exactly with an FMA (Dekker's product, here in its FMA form)
// and every addition into an accumulator keeps its error by Knuth's TwoSum, so
// one multiply-add costs 12 FP32 instructions.  The lo*lo cross term is
// dropped (2^-48 relative).  Sums over K <= 192 terms stay within ~1e-13
// relative, against the 1e-8 residual target of the refinement.
// Operators come pre-split (hi, lo) in global memory; the vectors and the
// stage-1 intermediate are held split in shared memory; the recurrence's
// epilogue and the final normalisation are evaluated in FP64 (a few
// operations per element and step, against ~K multiply-adds).
// ---------------------------------------------------------------------------


// cta_gemm in double-float: C(m, n) = sum_k A(m, k) B(k, n), operands float2,
// by kDfThreads = 512 threads in 64 x 64 tiles: a warp owns four rows 16 apart
// (one row a load, so its A operand is a broadcast), its lanes two columns 32
// apart.  Sixteen warps a CTA: the dependent double-float chains need more
// warps in flight than the eight of the FP32 kernels.
constexpr int kDfThreads = 512;

template <class Epi>
__device__ __forceinline__ void cta_gemm_df(int M, int N, int K, const float2* A, int sam, int sak, const float2* B,
                                            int sbk, int sbn, const Epi& epi) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int m0 = 0; m0 < M; m0 += 64) {
    for (int n0 = 0; n0 < N; n0 += 64) {
      int ar[4], bc[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) ar[i] = min(m0 + ty + 16 * i, M - 1) * sam;
#pragma unroll
      for (int j = 0; j < 2; ++j) bc[j] = min(n0 + tx + 32 * j, N - 1) * sbn;
      float s[4][2], t[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) s[i][j] = t[i][j] = 0.f;
#pragma unroll 2
      for (int k = 0; k < K; ++k) {
        float2 a[4], b[2];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = A[ar[i] + k * sak];
#pragma unroll
        for (int j = 0; j < 2; ++j) b[j] = B[k * sbk + bc[j]];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) df_mac(s[i][j], t[i][j], a[i], b[j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int n = n0 + tx + 32 * j;
          if (n < N) epi(m, n, s[i][j], t[i][j]);
        }
      }
    }
  }
}

struct DfEpi1 {  // T[((j*kA + a)*nvl + v)*kB + b] = (s + t) renormalised
  float2* Ts;
  int kA, kB, nvl;
  __device__ void operator()(int m, int n, float s, float t) const {
    const int v = m / kA, a = m - v * kA, j = n / kB, b = n - j * kB;
    const float hi = s + t;
    Ts[((j * kA + a) * nvl + v) * kB + b] = make_float2(hi, t - (hi - s));
  }
};

struct DfEpi2 {  // Yold <- alpha (acc + (EA[a] + EB[b]) x) + beta x + gamma z, in FP64
  const float2* Ycur;
  float2* Yold;
  const double* EA;
  const double* EB;
  int kA, kB;
  double alpha, beta, gamma;
  __device__ void operator()(int a, int n, float s, float t) const {
    const int v = n / kB, b = n - v * kB;
    const int idx = (v * kA + a) * kB + b;
    const double x = df_value(Ycur[idx]);
    double y = alpha * ((double)s + (double)t + (EA[a] + EB[b]) * x) + beta * x;
    if (gamma != 0.0) y += gamma * df_value(Yold[idx]);
    Yold[idx] = df_split(y);
  }
};

// Out = normalised p(H) X (deg >= 1, H X formed in the kernel) or Out = H X
// (deg == 0), FP64 in and out, double-float inside.  Ahl (kA x n_ops kA) and
// Bhl (n_ops kB x kB) are Acat and Bcat split into (hi, lo).  X and Out may
// be the same array.
__global__ void __launch_bounds__(kDfThreads)
    cheb_fused_df_kernel(const double* X, const double* __restrict__ EA, const double* __restrict__ EB,
                         const float2* __restrict__ Ahl, const float2* __restrict__ Bhl, double* Out, FusedArgs p) {
  extern __shared__ __align__(16) unsigned char fused_smem[];
  float2* sm = reinterpret_cast<float2*>(fused_smem);
  const int kA = p.kA, kB = p.kB, no = p.n_ops;
  const int n = kA * kB;
  const int v0 = blockIdx.x * p.vpc;
  const int nvl = min(p.vpc, p.nv - v0);
  if (nvl <= 0) return;
  float2* Yp = sm;
  float2* Yc = Yp + (size_t)p.vpc * n;
  float2* Ts = Yc + (size_t)p.vpc * n;
  double* red = reinterpret_cast<double*>(Ts + (size_t)no * p.vpc * n);
  const long base = (long)v0 * n;
  const int cnt = nvl * n;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) Yp[i] = df_split(X[base + i]);
  __syncthreads();
  auto product = [&](const float2* Ysrc, const DfEpi2& e2) {
    if (no > 0) {
      cta_gemm_df(nvl * kA, no * kB, kB, Ysrc, kB, 1, Bhl, 1, kB, DfEpi1{Ts, kA, kB, nvl});
      __syncthreads();
    }
    cta_gemm_df(kA, nvl * kB, no * kA, Ahl, no * kA, 1, Ts, nvl * kB, 1, e2);
    __syncthreads();
  };
  const double s1e = p.deg == 0 ? 1.0 : p.sigma1 / p.e;
  const double b1 = p.deg == 0 ? 0.0 : -p.c * s1e;
  product(Yp, DfEpi2{Yp, Yc, EA, EB, kA, kB, s1e, b1, 0.0});
  double sigma = p.sigma1;
  const double tau = 2.0 / p.sigma1;
  for (int d = 2; d <= p.deg; ++d) {
    const double s1 = 1.0 / (tau - sigma);
    product(Yc, DfEpi2{Yc, Yp, EA, EB, kA, kB, 2 * s1 / p.e, -2 * s1 * p.c / p.e, -sigma * s1});
    float2* t = Yp;
    Yp = Yc;
    Yc = t;
    sigma = s1;
  }
  if (p.deg == 0) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) Out[base + i] = df_value(Yc[i]);
    return;
  }
  for (int v = 0; v < nvl; ++v) {
    const float2* y = Yc + (size_t)v * n;
    double s = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double yi = df_value(y[i]);
      s += yi * yi;
    }
    s = block_sum(s, red);
    const double inv = s > 0 ? 1.0 / sqrt(s) : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) Out[base + (long)v * n + i] = df_value(y[i]) * inv;
  }
}

// (hi, lo) split of an FP64 array
__global__ void df_split_kernel(const double* __restrict__ in, long count, float2* __restrict__ out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    out[i] = df_split(in[i]);
}

}  // namespace rmc
