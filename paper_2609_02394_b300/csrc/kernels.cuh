// Device kernels of the merge step (Algorithm 1, inner loop) and the leaf
// build (Algorithm 1, first step).  Every kernel here is launched by the host
// driver in rmc.cu; see the comments there for the order.
#pragma once

#include <algorithm>

#include "common.cuh"
#include "gemm.cuh"

namespace rmc {

constexpr int kMaxOps = 32;        // carried operators / coupling terms per merge
constexpr int kMaxSmallDim = 160;  // Jacobi eigensolver: matrix held in shared memory

struct Coefs {
  double c[kMaxOps];
};

// ---------------------------------------------------------------------------
// Kronecker-form product with H_eff (Eq. (7)) in two GEMM stages:
//   stage 1: T[(j, a), (v, b)] = sum_b' X[v][a][b'] * B_j[b][b']
//   stage 2: Y[v][a][b] = alpha * ( (EA[a] + EB[b]) X[v][a][b]
//                                   + sum_{j, a'} coef_j A_j[a][a'] T[(j, a'), (v, b)] )
//                         + beta * X[v][a][b] + gamma * Z[v][a][b]
// Stage 2 contracts over (j, a') at once with Acat[a][(j, a')] = coef_j A_j[a][a'].
// ---------------------------------------------------------------------------

template <typename T>
__global__ void build_acat_kernel(const T* __restrict__ A, Coefs coef, int kA, int n_ops, T* __restrict__ Acat) {
  const long total = (long)kA * n_ops * kA;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int a = (int)(e / (n_ops * kA));
    const int r = (int)(e % (n_ops * kA));
    const int j = r / kA, ap = r % kA;
    Acat[e] = (T)coef.c[j] * A[((long)j * kA + a) * kA + ap];
  }
}

template <typename T>
struct EpiKron1 {  // m = v*kA + a, n = j*kB + b  ->  T[((j*kA + a)*nv + v)*kB + b]
  T* Tbuf;
  int kA, kB, nv;
  __device__ void operator()(int, int, int m, int n, T acc) const {
    const int v = m / kA, a = m % kA, j = n / kB, b = n % kB;
    Tbuf[(((long)j * kA + a) * nv + v) * kB + b] = acc;
  }
};

template <typename T>
struct EpiKron2 {  // m = a, n = v*kB + b
  const T* X;
  const T* Z;
  const T* EA;
  const T* EB;
  T* Y;
  int kA, kB;
  T alpha, beta, gamma;
  __device__ void operator()(int, int, int m, int n, T acc) const {
    const int v = n / kB, b = n % kB;
    const long idx = ((long)v * kA + m) * kB + b;
    const T x = X[idx];
    T y = alpha * (acc + (EA[m] + EB[b]) * x) + beta * x;
    if (gamma != T(0)) y += gamma * Z[idx];
    Y[idx] = y;
  }
};

// Tensor-core variant: the stage-1 output is laid out as stage 2's K-major
// operand, T'[(v, b)][(j, a)], and stage 2 computes Y^T rows (v, b).
template <typename T>
struct EpiKron1T {  // m = v*kA + a, n = j*kB + b  ->  T'[(v*kB + b)*(n_ops*kA) + j*kA + a]
  T* Tbuf;
  int kA, kB, n_ops;
  __device__ void operator()(int, int, int m, int n, T acc) const {
    const int v = m / kA, a = m % kA, j = n / kB, b = n % kB;
    Tbuf[((long)v * kB + b) * ((long)n_ops * kA) + (long)j * kA + a] = acc;
  }
  // The 32 x 32 block of rows row0 .. row0 + 31 (a0 .. a0 + 31 of one vector)
  // and columns n0 .. n0 + 31 (b0 .. b0 + 31 of one operator j) is the block of
  // T' (rows v*kB + b, columns j*kA + a) at x = j*kA + a0, y = v*kB + b0.
  __device__ bool block_xy(int, int row0, int n0, int* x, int* y) const {
    if ((kA & 31) || (kB & 31) || (row0 & 31) || (n0 & 31)) return false;
    const int v = row0 / kA, a0 = row0 % kA, j = n0 / kB, b0 = n0 % kB;
    *x = j * kA + a0;
    *y = v * kB + b0;
    return true;
  }
  __device__ void values(int, int, int, const float (&val)[32], float (&out)[32]) const {
#pragma unroll
    for (int t = 0; t < 32; ++t) out[t] = val[t];
  }
  // cnt (<= 32) consecutive columns n0 .. n0 + cnt - 1 of row m: the index
  // arithmetic once per run, then (j, b) stepped
  __device__ void run(int, int m, int n0, const float (&val)[32], int cnt) const {
    const int v = m / kA, a = m % kA;
    int j = n0 / kB, b = n0 % kB;
    const long ld = (long)n_ops * kA;
    T* base = Tbuf + (long)v * kB * ld + a;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (t < cnt) {
        base[(long)b * ld + (long)j * kA] = (T)val[t];
        if (++b == kB) {
          b = 0;
          ++j;
        }
      }
    }
  }
};

template <typename T>
struct EpiKron2T {  // m = v*kB + b, n = a
  const T* X;
  const T* Z;
  const T* EA;
  const T* EB;
  T* Y;
  int kA, kB;
  T alpha, beta, gamma;
  __device__ void operator()(int, int, int m, int n, T acc) const {
    const int v = m / kB, b = m % kB;
    const long idx = ((long)v * kA + n) * kB + b;
    const T x = X[idx];
    T y = alpha * (acc + (EA[n] + EB[b]) * x) + beta * x;
    if (gamma != T(0)) y += gamma * Z[idx];
    Y[idx] = y;
  }
  // The 32 x 32 block of rows row0 .. row0 + 31 (b0 .. b0 + 31 of one vector)
  // and columns a0 .. a0 + 31 is the block of Y (rows v*kA + a, columns b) at
  // x = b0, y = v*kA + a0.
  __device__ bool block_xy(int, int row0, int n0, int* x, int* y) const {
    if ((kA & 31) || (kB & 31) || (row0 & 31) || (n0 & 31)) return false;
    const int v = row0 / kB, b0 = row0 % kB;
    *x = b0;
    *y = v * kA + n0;
    return true;
  }
  // the final values of the 32 columns a = n0 .. n0 + 31 of row (v, b)
  __device__ void values(int, int m, int n0, const float (&val)[32], float (&out)[32]) const {
    const int v = m / kB, b = m % kB;
    const T eb = __ldg(EB + b);
    const long idx0 = ((long)v * kA + n0) * kB + b;
    T x[32], z[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      x[t] = __ldg(X + idx0 + (long)t * kB);
      z[t] = gamma != T(0) ? __ldg(Z + idx0 + (long)t * kB) : T(0);
    }
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      T y = alpha * ((T)val[t] + (__ldg(EA + n0 + t) + eb) * x[t]) + beta * x[t];
      if (gamma != T(0)) y += gamma * z[t];
      out[t] = (float)y;
    }
  }
  // cnt (<= 32) consecutive columns a = n0 .. n0 + cnt - 1 of row (v, b).
  // Every input of the run is loaded before the first store, so the loads
  // overlap (a store to Y could otherwise alias a later X load and serialise
  // them on the memory latency).
  __device__ void run(int, int m, int n0, const float (&val)[32], int cnt) const {
    const int v = m / kB, b = m % kB;
    const T eb = __ldg(EB + b);
    const long idx0 = ((long)v * kA + n0) * kB + b;
    T x[32], z[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      x[t] = t < cnt ? __ldg(X + idx0 + (long)t * kB) : T(0);
      z[t] = (gamma != T(0) && t < cnt) ? __ldg(Z + idx0 + (long)t * kB) : T(0);
    }
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (t < cnt) {
        T y = alpha * ((T)val[t] + (__ldg(EA + n0 + t) + eb) * x[t]) + beta * x[t];
        if (gamma != T(0)) y += gamma * z[t];
        Y[idx0 + (long)t * kB] = y;
      }
    }
  }
};

// Split-K partial products of the tensor-core Gram form, stored transposed:
// split sp of acc[m][n] to Pt[(sp*N + n)*M + m] (Pt viewed as a (splits*N) x M
// row-major matrix, so a warp's 32 rows m are the inner dimension of its
// 32 x 32 TMA block store, as the staging layout has them).
struct EpiSplitT {
  float* Pt;
  int M, N;
  __device__ bool block_xy(int sp, int row0, int n0, int* x, int* y) const {
    *x = row0;
    *y = sp * N + n0;
    return true;
  }
  __device__ void values(int, int, int, const float (&val)[32], float (&out)[32]) const {
#pragma unroll
    for (int t = 0; t < 32; ++t) out[t] = val[t];
  }
  __device__ void run(int sp, int m, int n0, const float (&val)[32], int cnt) const {
    float* p = Pt + ((long)sp * N + n0) * M + m;
#pragma unroll
    for (int t = 0; t < 32; ++t)
      if (t < cnt) p[(long)t * M] = val[t];
  }
};

// G[m][n] = sum over the splits of Pt[(sp*N + n)*M + m], in split order
// (consecutive threads take consecutive m, so the reads of Pt are coalesced).
__global__ void reduce_splits_t_kernel(const float* __restrict__ Pt, int splits, int M, int N, float* __restrict__ G) {
  const long total = (long)M * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int n = (int)(e / M), m = (int)(e % M);
    float acc = 0.0f;
    for (int sp = 0; sp < splits; ++sp) acc += Pt[sp * total + e];
    G[(long)m * N + n] = acc;
  }
}

// G <- (G + G^T) / 2 for a square m x m matrix (each pair once).
__global__ void symmetrize_kernel(float* __restrict__ G, int m) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)m * m; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    if (j > i) {
      const float v = 0.5f * (G[(long)i * m + j] + G[(long)j * m + i]);
      G[(long)i * m + j] = v;
      G[(long)j * m + i] = v;
    }
  }
}

// Y = alpha * acc + beta * Src (Src may alias nothing written by the GEMM).
template <typename T>
struct EpiAxpby {
  T* C;
  const T* Src;
  long ldc, lds;
  long batch_stride_c, batch_stride_s;
  T alpha, beta;
  __device__ void operator()(int bt, int, int m, int n, T acc) const {
    T v = alpha * acc;
    if (beta != T(0)) v += beta * Src[(long)bt * batch_stride_s + (long)m * lds + n];
    C[(long)bt * batch_stride_c + (long)m * ldc + n] = v;
  }
};

// ---------------------------------------------------------------------------
// Elementwise helpers
// ---------------------------------------------------------------------------

template <typename TO, typename TI>
__global__ void convert_kernel(const TI* __restrict__ in, TO* __restrict__ out, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    out[e] = (TO)in[e];
}

// Diagonal of H_eff (Eq. (7)): D[a*kB + b] = EA[a] + EB[b] + sum_j coef_j A_j[a][a] B_j[b][b].
__global__ void diag_kernel(const double* __restrict__ EA, const double* __restrict__ EB,
                            const double* __restrict__ A, const double* __restrict__ B, Coefs coef,
                            int n_ops, int kA, int kB, double* __restrict__ D) {
  const long n = (long)kA * kB;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int a = (int)(e / kB), b = (int)(e % kB);
    double d = EA[a] + EB[b];
    for (int j = 0; j < n_ops; ++j)
      d += coef.c[j] * A[((long)j * kA + a) * kA + a] * B[((long)j * kB + b) * kB + b];
    D[e] = d;
  }
}

__device__ __forceinline__ unsigned long long order_key(double x) {
  unsigned long long u = __double_as_longlong(x);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// One CTA (1024 threads): the b smallest entries of D (ties broken by index),
// written as idx[0..b-1] in ascending (D, index) order; also min and max of D.
// Radix select on order-preserving 64-bit keys, stable compaction, bitonic
// sort of the selected pairs.  b <= 1024.
__global__ void __launch_bounds__(1024) select_smallest_kernel(const double* __restrict__ D, long n, int b,
                                                               int* __restrict__ idx, double* __restrict__ dminmax) {
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long s_prefix, s_mask;
  __shared__ long s_need;
  __shared__ unsigned long long skey[1024];
  __shared__ int sidx[1024];
  __shared__ int s_take_less, s_take_eq;
  __shared__ double red[32];
  const int tid = threadIdx.x;

  double lo = INFINITY, hi = -INFINITY;
  for (long i = tid; i < n; i += blockDim.x) { lo = fmin(lo, D[i]); hi = fmax(hi, D[i]); }
  hi = block_max(hi, red);
  lo = -block_max(-lo, red);
  if (tid == 0) { dminmax[0] = lo; dminmax[1] = hi; s_prefix = 0; s_mask = 0; s_need = b; }
  __syncthreads();

  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const unsigned long long pre = s_prefix, msk = s_mask;
    for (long i = tid; i < n; i += blockDim.x) {
      const unsigned long long k = order_key(D[i]);
      if ((k & msk) == pre) atomicAdd(&hist[(k >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      long need = s_need, cum = 0;
      int d = 0;
      for (; d < 256; ++d) {
        if (cum + (long)hist[d] >= need) break;
        cum += hist[d];
      }
      s_need = need - cum;
      s_prefix = pre | ((unsigned long long)d << shift);
      s_mask = msk | (0xFFull << shift);
    }
    __syncthreads();
  }
  const unsigned long long kstar = s_prefix;
  const long need_eq = s_need;  // equal keys to take (>= 1)
  // stable compaction in index order
  if (tid == 0) { s_take_less = 0; s_take_eq = 0; }
  __syncthreads();
  __shared__ int wsum_l[32], wsum_e[32];
  for (long base = 0; base < n; base += blockDim.x) {
    const long i = base + tid;
    int isl = 0, ise = 0;
    unsigned long long k = 0;
    if (i < n) {
      k = order_key(D[i]);
      isl = k < kstar;
      ise = k == kstar;
    }
    // block exclusive scans of isl and ise
    const int lane = tid & 31, wid = tid >> 5;
    int xl = isl, xe = ise;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int yl = __shfl_up_sync(0xffffffffu, xl, o), ye = __shfl_up_sync(0xffffffffu, xe, o);
      if (lane >= o) { xl += yl; xe += ye; }
    }
    if (lane == 31) { wsum_l[wid] = xl; wsum_e[wid] = xe; }
    __syncthreads();
    if (wid == 0) {
      int vl = wsum_l[lane], ve = wsum_e[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int yl = __shfl_up_sync(0xffffffffu, vl, o), ye = __shfl_up_sync(0xffffffffu, ve, o);
        if (lane >= o) { vl += yl; ve += ye; }
      }
      wsum_l[lane] = vl;
      wsum_e[lane] = ve;
    }
    __syncthreads();
    const int exl = xl - isl + (wid ? wsum_l[wid - 1] : 0);
    const int exe = xe - ise + (wid ? wsum_e[wid - 1] : 0);
    const int tl = s_take_less, te = s_take_eq;
    __syncthreads();
    // positions: less-than keys are all taken; equal keys only the first need_eq
    if (isl) {
      const int slot = tl + exl;  // provisional among "less"
      skey[slot] = k;            // less keys never exceed b - need_eq slots
      sidx[slot] = (int)i;
    }
    __syncthreads();
    if (ise && (long)(te + exe) < need_eq) {
      const int slot = (b - (int)need_eq) + te + exe;
      skey[slot] = k;
      sidx[slot] = (int)i;
    }
    __syncthreads();
    if (tid == 0) { s_take_less = tl + wsum_l[31]; s_take_eq = te + wsum_e[31]; }
    __syncthreads();
  }
  // bitonic sort of (key, index) over the next power of two >= b
  int P = 1;
  while (P < b) P <<= 1;
  for (int i = b + tid; i < P; i += blockDim.x) { skey[i] = ~0ull; sidx[i] = 0x7fffffff; }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = ((i & size) == 0);
          const bool gt = (skey[i] > skey[j]) || (skey[i] == skey[j] && sidx[i] > sidx[j]);
          if (gt == up) {
            unsigned long long tk = skey[i]; skey[i] = skey[j]; skey[j] = tk;
            int ti = sidx[i]; sidx[i] = sidx[j]; sidx[j] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < b; i += blockDim.x) idx[i] = sidx[i];
}

// Start block of the subspace iteration: X[i] = e_{idx[i]} + amp * r_i, r_i
// uniform in [-1, 1) per element from the splitmix64 mixing function (Steele,
// Lea and Flood, 2014) of the element's flat index.  The unit vectors alone
// each lie in one symmetry sector of H (parity, magnetisation) and the filter
// keeps them there, so a low state whose sector holds too few of the chosen
// unit vectors would never enter the block; the small deterministic
// perturbation gives every vector a component in every sector.  Writes all of
// X (vector-major, b x n).
__device__ __forceinline__ double splitmix_uniform(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

template <typename T>
__global__ void start_vectors_kernel(const int* __restrict__ idx, int b, long n, double amp, T* __restrict__ X) {
  const long total = (long)b * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n);
    const long r = e - (long)i * n;
    X[e] = T((r == idx[i] ? 1.0 : 0.0) + amp * splitmix_uniform((unsigned long long)e));
  }
}

// X[i] = e_{idx[i]}  (vector-major, X zeroed by the caller)
template <typename T>
__global__ void unit_vectors_kernel(const int* __restrict__ idx, int b, long n, T* __restrict__ X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < b) X[(long)i * n + idx[i]] = T(1);
}

// Normalise each vector (one CTA per vector); records the norms.
template <typename T>
__global__ void normalize_kernel(T* __restrict__ X, long n, T* __restrict__ norms) {
  __shared__ T red[32];
  T* x = X + (long)blockIdx.x * n;
  T s = 0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) s += x[i] * x[i];
  s = block_sum(s, red);
  const T nr = sqrt(s);
  const T inv = nr > T(0) ? T(1) / nr : T(0);
  for (long i = threadIdx.x; i < n; i += blockDim.x) x[i] *= inv;
  if (threadIdx.x == 0 && norms) norms[blockIdx.x] = nr;
}

// Residual norms of Ritz pairs, rn[i] = ||HX_i - theta_i X_i|| (one CTA per
// vector, warp-shuffle block reduction), and the count of i < k_conv with
// rn[i] > tol * max(1, |theta_i|) into status[0] (zeroed by the caller).
template <typename T>
__global__ void residual_kernel(const T* __restrict__ X, const T* __restrict__ HX, const T* __restrict__ theta,
                                long n, int k_conv, double tol, double* __restrict__ rn, int* __restrict__ status) {
  __shared__ T red[32];
  const int i = blockIdx.x;
  const T* x = X + (long)i * n;
  const T* hx = HX + (long)i * n;
  const T th = theta[i];
  T s = 0;
  for (long r = threadIdx.x; r < n; r += blockDim.x) {
    const T d = hx[r] - th * x[r];
    s += d * d;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double r = sqrt((double)s);
    rn[i] = r;
    if (i < k_conv && !(r <= tol * fmax(1.0, fabs((double)th)))) atomicAdd(status, 1);
  }
}

// Flip each vector so that its entry of largest magnitude (first one on exact
// ties) is positive (one CTA per vector).
__global__ void gauge_kernel(double* __restrict__ C, long n) {
  __shared__ double sv[32];
  __shared__ long si[32];
  double* c = C + (long)blockIdx.x * n;
  double best = -1.0;
  long bi = 0x7fffffffffffffffL;
  for (long r = threadIdx.x; r < n; r += blockDim.x) {
    const double a = fabs(c[r]);
    if (a > best) { best = a; bi = r; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const long oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (lane == 0) { sv[wid] = best; si[wid] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 1; w < nw; ++w)
      if (sv[w] > sv[0] || (sv[w] == sv[0] && si[w] < si[0])) { sv[0] = sv[w]; si[0] = si[w]; }
  }
  __syncthreads();
  const bool flip = c[si[0]] < 0.0;
  __syncthreads();
  if (flip)
    for (long r = threadIdx.x; r < n; r += blockDim.x) c[r] = -c[r];
}

// ---------------------------------------------------------------------------
// Small dense symmetric eigensolver, one CTA: cyclic parallel Jacobi in FP32
// with round-robin pairing (all m(m-1)/2 pairs once per sweep, m/2 disjoint
// rotations per round; each 2x2 block of A updated as J_k^T A_kl J_l).  Warps
// take block rows k (and rows of V), lanes take block columns l; a lane keeps
// the pair and rotation of its columns in registers for the round, so the
// inner loops do no index arithmetic beyond one multiply-add per access (the
// kernel is bound by instruction issue on its SM).  Stops when the
// off-diagonal norm is below 1e-6 ||A||_F, or when a sweep no longer halves it
// (the FP32 rounding floor).  Eigenvalues ascending into w, eigenvectors as
// columns of the row-major m x m V.  m <= kMaxSmallDim.  status[0] += 1 if the
// sweep cap was hit first.
// ---------------------------------------------------------------------------
constexpr int kJacobiLaneCols = (kMaxSmallDim / 2 + 31) / 32;  // block columns a lane holds

template <typename TI, typename TO>
__global__ void __launch_bounds__(1024) jacobi_kernel(const TI* __restrict__ S, int m, TO* __restrict__ w,
                                                      TO* __restrict__ V, int* __restrict__ status, int max_sweeps) {
  extern __shared__ float smem[];
  const int mm = (m + 1) & ~1;  // even
  const int ld = mm + 1;        // padded row stride of A
  float* A = smem;              // mm x ld
  float* Vs = A + mm * ld;      // m x mm
  float* cs = Vs + m * mm;      // mm/2
  float* sn = cs + mm / 2;
  int* P = (int*)(sn + mm / 2);
  int* Q = P + mm / 2;
  __shared__ float red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int half = mm / 2;

  for (int i = warp; i < mm; i += nw)
    for (int j = lane; j < mm; j += 32) {
      float v = 0.f;
      if (i < m && j < m) v = (float)(0.5 * ((double)S[i * m + j] + (double)S[j * m + i]));
      A[i * ld + j] = v;
    }
  for (int i = warp; i < m; i += nw)
    for (int j = lane; j < mm; j += 32) Vs[i * mm + j] = (i == j) ? 1.f : 0.f;
  __syncthreads();
  float fro = 0.f;
  for (int i = warp; i < m; i += nw)
    for (int j = lane; j < m; j += 32) fro += A[i * ld + j] * A[i * ld + j];
  fro = sqrtf(block_sum(fro, red));
  const float target = 1e-6f * fro;

  float prev = INFINITY;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    float off = 0.f;
    for (int i = warp; i < m; i += nw)
      for (int j = lane; j < m; j += 32)
        if (j != i) off += A[i * ld + j] * A[i * ld + j];
    off = sqrtf(block_sum(off, red));
    if (off <= target || fro == 0.f || (off > 0.5f * prev && off < 1e-4f * fro)) break;
    prev = off;
    for (int r = 0; r < mm - 1; ++r) {
      if (tid < half) {
        const int k = tid;
        int p, q;
        if (k == 0) { p = r; q = mm - 1; }
        else {
          p = r + k; if (p >= mm - 1) p -= mm - 1;
          q = r - k; if (q < 0) q += mm - 1;
        }
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, sv = 0.f;
        if (q < m) {
          const float apq = A[p * ld + q];
          if (apq != 0.f) {
            const float app = A[p * ld + p], aqq = A[q * ld + q];
            const float tau = (aqq - app) / (2.f * apq);
            const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + t * t);
            sv = t * c;
          }
        }
        cs[k] = c; sn[k] = sv; P[k] = p; Q[k] = q;
      }
      __syncthreads();
      // this lane's block columns l = lane + 32 j
      int pl[kJacobiLaneCols], ql[kJacobiLaneCols];
      float cl[kJacobiLaneCols], sl[kJacobiLaneCols];
#pragma unroll
      for (int j = 0; j < kJacobiLaneCols; ++j) {
        const int l = lane + 32 * j;
        const bool on = l < half;
        pl[j] = on ? P[l] : 0;
        ql[j] = on ? Q[l] : 0;
        cl[j] = on ? cs[l] : 1.f;
        sl[j] = on ? sn[l] : 0.f;
      }
      // A <- J^T A J: block row k on a warp, its block columns on the lanes
      for (int k = warp; k < half; k += nw) {
        const int pk = P[k], qk = Q[k];
        const float ck = cs[k], sk = sn[k];
        float* rp = A + pk * ld;
        float* rq = A + qk * ld;
#pragma unroll
        for (int j = 0; j < kJacobiLaneCols; ++j) {
          const int l = lane + 32 * j;
          if (l < half) {
            const float a00 = rp[pl[j]], a01 = rp[ql[j]];
            const float a10 = rq[pl[j]], a11 = rq[ql[j]];
            const float b00 = ck * a00 - sk * a10, b01 = ck * a01 - sk * a11;
            const float b10 = sk * a00 + ck * a10, b11 = sk * a01 + ck * a11;
            float n00 = b00 * cl[j] - b01 * sl[j], n01 = b00 * sl[j] + b01 * cl[j];
            float n10 = b10 * cl[j] - b11 * sl[j], n11 = b10 * sl[j] + b11 * cl[j];
            if (k == l) { n01 = 0.f; n10 = 0.f; }
            rp[pl[j]] = n00; rp[ql[j]] = n01;
            rq[pl[j]] = n10; rq[ql[j]] = n11;
          }
        }
      }
      // V <- V J: a row of V on a warp, its column pairs on the lanes
      for (int row = warp; row < m; row += nw) {
        float* vr = Vs + row * mm;
#pragma unroll
        for (int j = 0; j < kJacobiLaneCols; ++j) {
          if (lane + 32 * j < half) {
            const float vp = vr[pl[j]], vq = vr[ql[j]];
            vr[pl[j]] = cl[j] * vp - sl[j] * vq;
            vr[ql[j]] = sl[j] * vp + cl[j] * vq;
          }
        }
      }
      __syncthreads();
    }
  }
  if (sweep == max_sweeps && tid == 0 && status) atomicAdd(status, 1);
  // sort eigenvalues ascending (rank sort, ties by index)
  for (int i = tid; i < m; i += nt) {
    const float di = A[i * ld + i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const float dj = A[j * ld + j];
      rank += (dj < di) || (dj == di && j < i);
    }
    w[rank] = (TO)di;
    for (int row = 0; row < m; ++row) V[row * m + rank] = (TO)Vs[row * mm + i];
  }
}

// Threads for jacobi_kernel on an m x m matrix: a warp for each of the m/2
// block rows, at least 2 and at most 32 warps.
inline int jacobi_threads(int m) {
  const int half = ((m + 1) & ~1) / 2;
  return 32 * std::min(32, std::max(2, half));
}

inline size_t jacobi_smem_bytes(int m) {
  const int mm = (m + 1) & ~1;
  return sizeof(float) * ((size_t)mm * (mm + 1) + (size_t)m * mm + mm) + sizeof(int) * mm;
}

// Ogita-Aishima refinement (Japan J. Indust. Appl. Math. 35, 2018), the step
// between the three products: given R = I - V^T V and Sp = V^T A V (m x m,
// FP64), form lambda_i = Sp_ii / (1 - R_ii) and the correction E with
// E_ij = (Sp_ij + lambda_j R_ij) / (lambda_j - lambda_i) where
// |lambda_i - lambda_j| > delta and R_ij / 2 otherwise (clustered pairs are
// only re-orthogonalised), delta = 2 (||Sp - diag(lambda)||_F + ||A||_F ||R||_F).
// R is overwritten by E.  Three launches, rows of the m x m matrices dealt to
// the CTAs (an FP64 division per entry: one SM's FP64 rate made a one-CTA
// form the slowest kernel of the refinement): oa_sums_kernel (lambda and
// per-CTA partial sums of the three norms), oa_update_kernel (every CTA
// reduces the partial sums in the same fixed order, then corrects its rows
// and records its max |E|), oa_finish_kernel (the stop test).  Each returns
// at once when *done is set.
__global__ void oa_sums_kernel(const double* __restrict__ R, const double* __restrict__ Sp,
                               const double* __restrict__ A, int m, double* __restrict__ lam,
                               double* __restrict__ part, const int* __restrict__ done) {
  if (*done) return;
  __shared__ double red[32];
  double an = 0.0, off = 0.0, rr = 0.0;
  for (int i = blockIdx.x; i < m; i += gridDim.x) {
    const double* Ai = A + (size_t)i * m;
    const double* Si = Sp + (size_t)i * m;
    const double* Ri = R + (size_t)i * m;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const double r = Ri[j];
      double d = Si[j];
      if (j == i) {
        const double li = Si[j] / (1.0 - r);
        lam[i] = li;
        d -= li;
      }
      an += Ai[j] * Ai[j];
      off += d * d;
      rr += r * r;
    }
  }
  an = block_sum(an, red);
  off = block_sum(off, red);
  rr = block_sum(rr, red);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = an;
    part[3 * blockIdx.x + 1] = off;
    part[3 * blockIdx.x + 2] = rr;
  }
}

__global__ void oa_update_kernel(double* __restrict__ R, const double* __restrict__ Sp,
                                 const double* __restrict__ lam, int m, const double* __restrict__ part, int nparts,
                                 double* __restrict__ emax_part, const int* __restrict__ done) {
  if (*done) return;
  __shared__ double red[32];
  double an = 0.0, off = 0.0, rr = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
    an += part[3 * b];
    off += part[3 * b + 1];
    rr += part[3 * b + 2];
  }
  an = block_sum(an, red);
  off = block_sum(off, red);
  rr = block_sum(rr, red);
  const double delta = 2.0 * (sqrt(off) + sqrt(an) * sqrt(rr));
  double emax = 0.0;
  for (int i = blockIdx.x; i < m; i += gridDim.x) {
    const double li = lam[i];
    double* Ri = R + (size_t)i * m;
    const double* Si = Sp + (size_t)i * m;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const double r = Ri[j];
      const double lj = lam[j];
      double E;
      if (j != i && fabs(li - lj) > delta) E = (Si[j] + lj * r) / (lj - li);
      else E = 0.5 * r;
      Ri[j] = E;
      emax = fmax(emax, fabs(E));
    }
  }
  emax = block_max(emax, red);
  if (threadIdx.x == 0) emax_part[blockIdx.x] = emax;
}

// Stop once the correction is at the FP64 rounding level, or once it no
// longer shrinks quadratically (near-degenerate pairs leave rounding noise of
// order u ||A|| / gap that no further step removes).
__global__ void oa_finish_kernel(const double* __restrict__ emax_part, int nparts, int* __restrict__ done,
                                 double* __restrict__ prev_emax) {
  if (*done) return;
  __shared__ double red[32];
  double emax = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) emax = fmax(emax, emax_part[b]);
  emax = block_max(emax, red);
  if (threadIdx.x == 0) {
    const double pe = *prev_emax;
    if (emax <= 4e-16 || (emax < 1e-8 && emax > 0.01 * pe)) *done = 1;
    *prev_emax = emax;
  }
}

// E = (I - G) / 2 (m x m): one Newton-Schulz orthonormalisation step
// V <- V + V E makes V^T V = I up to O(||I - G||^2).
__global__ void half_identity_minus_kernel(const double* __restrict__ G, int m, double* __restrict__ E) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x)
    E[e] = 0.5 * (((e / m) == (e % m) ? 1.0 : 0.0) - G[e]);
}

// Clean-up for a nearly diagonal symmetric S (m x m, FP64): classical Jacobi
// -- repeatedly the off-diagonal entry of largest magnitude is found and
// annihilated by an exact rotation -- until every |S_pq| <= tol * ||S||_F or
// 4m rotations were made.  Ogita-Aishima steps leave exactly this kind of
// matrix when near-degenerate pairs (gap below their coupling bound) stay
// unrotated; a handful of exact rotations finishes them.  S lives in shared
// memory; the rotations are also applied to the columns of V (row-major,
// global).  lam[i] = S_ii on return.  One CTA.
__global__ void __launch_bounds__(1024) jacobi_cleanup_kernel(const double* __restrict__ Sin, int m,
                                                              double* __restrict__ V, double* __restrict__ lam,
                                                              double tol) {
  extern __shared__ double S[];  // m x m
  __shared__ double red[32];
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_p, s_q;
  __shared__ double s_c, s_s;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  double fro = 0.0;
  for (int e = tid; e < m * m; e += nt) {
    const double v = 0.5 * (Sin[e] + Sin[(e % m) * m + e / m]);
    S[e] = v;
    fro += v * v;
  }
  fro = sqrt(block_sum(fro, red));
  const double thresh = tol * fro;
  for (int rot = 0; rot < 4 * m; ++rot) {
    // argmax |S_pq| over p < q
    double best = -1.0;
    int bi = 0;
    for (int e = tid; e < m * m; e += nt) {
      const int p = e / m, q = e % m;
      if (q > p) {
        const double a = fabs(S[e]);
        if (a > best) { best = a; bi = e; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { sv[wid] = best; si[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      int w = 0;
      for (int j = 1; j < (nt >> 5); ++j)
        if (sv[j] > sv[w] || (sv[j] == sv[w] && si[j] < si[w])) w = j;
      s_p = si[w] / m;
      s_q = si[w] % m;
      sv[0] = sv[w];
      if (sv[w] > thresh) {
        const int p = s_p, q = s_q;
        const double apq = S[p * m + q], app = S[p * m + p], aqq = S[q * m + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        s_c = 1.0 / sqrt(1.0 + t * t);
        s_s = t * s_c;
      }
    }
    __syncthreads();
    if (!(sv[0] > thresh)) break;
    const int p = s_p, q = s_q;
    const double c = s_c, s = s_s;
    // rows p, q then columns p, q of S (J = [[c, s], [-s, c]] in (p, q)), and V <- V J
    for (int j = tid; j < m; j += nt) {
      const double ap = S[p * m + j], aq = S[q * m + j];
      S[p * m + j] = c * ap - s * aq;
      S[q * m + j] = s * ap + c * aq;
    }
    __syncthreads();
    for (int j = tid; j < m; j += nt) {
      const double ap = S[j * m + p], aq = S[j * m + q];
      S[j * m + p] = c * ap - s * aq;
      S[j * m + q] = s * ap + c * aq;
      const double vp = V[j * m + p], vq = V[j * m + q];
      V[j * m + p] = c * vp - s * vq;
      V[j * m + q] = s * vp + c * vq;
    }
    __syncthreads();
    if (tid == 0) { S[p * m + q] = 0.0; S[q * m + p] = 0.0; }
    __syncthreads();
  }
  for (int i = tid; i < m; i += nt) lam[i] = S[i * m + i];
}

// The same clean-up for matrices too large for shared memory (m up to 1024;
// 512 threads, where 1024 made it spill):
// S is a global m x m scratch (this CTA's own), and each row keeps its largest
// off-diagonal |S_ij| and its column in shared memory, so a rotation costs
// O(m) work instead of an O(m^2) search: after rotating (p, q) the rows p and
// q, and every row whose largest entry sat in column p or q, are scanned again;
// every other row only compares its two changed entries with its maximum.
__global__ void __launch_bounds__(512) jacobi_cleanup_global_kernel(const double* __restrict__ Sin, int m,
                                                                     double* __restrict__ S,
                                                                     double* __restrict__ V,
                                                                     double* __restrict__ lam, double tol) {
  __shared__ double rmax[1024];
  __shared__ int rarg[1024];
  __shared__ bool rescan[1024];
  __shared__ double red[32];
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_p, s_q, s_n;
  __shared__ double s_c, s_s;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  double fro = 0.0;
  for (int i = wid; i < m; i += nw)
    for (int j = lane; j < m; j += 32) {
      const double v = 0.5 * (Sin[i * m + j] + Sin[j * m + i]);
      S[i * m + j] = v;
      fro += v * v;
    }
  fro = sqrt(block_sum(fro, red));  // (its barriers also publish S to the CTA)
  const double thresh = tol * fro;
  // largest off-diagonal entry of row i (ties: the lowest column), by one warp
  auto scan_row = [&](int i) {
    double best = -1.0;
    int arg = i == 0 ? 1 : 0;
    for (int j = lane; j < m; j += 32) {
      const double a = j == i ? -1.0 : fabs(S[i * m + j]);
      if (a > best) { best = a; arg = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
      if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
    }
    if (lane == 0) { rmax[i] = best; rarg[i] = arg; }
  };
  for (int i = wid; i < m; i += nw) scan_row(i);
  __syncthreads();
  for (int rot = 0; rot < 4 * m; ++rot) {
    // the row with the largest entry (ties: the lowest row)
    double best = -1.0;
    int bi = 0;
    for (int i = tid; i < m; i += nt)
      if (rmax[i] > best) { best = rmax[i]; bi = i; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { sv[wid] = best; si[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      int w = 0;
      for (int j = 1; j < nw; ++j)
        if (sv[j] > sv[w] || (sv[j] == sv[w] && si[j] < si[w])) w = j;
      const int a = si[w], b = rarg[si[w]];
      s_p = a < b ? a : b;
      s_q = a < b ? b : a;
      sv[0] = sv[w];
      if (sv[w] > thresh) {
        const int p = s_p, q = s_q;
        const double apq = S[p * m + q], app = S[p * m + p], aqq = S[q * m + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        s_c = 1.0 / sqrt(1.0 + t * t);
        s_s = t * s_c;
      }
    }
    __syncthreads();
    if (!(sv[0] > thresh)) break;
    const int p = s_p, q = s_q;
    const double c = s_c, s = s_s;
    for (int j = tid; j < m; j += nt) {
      const double ap = S[p * m + j], aq = S[q * m + j];
      S[p * m + j] = c * ap - s * aq;
      S[q * m + j] = s * ap + c * aq;
    }
    __syncthreads();
    for (int j = tid; j < m; j += nt) {
      const double ap = S[j * m + p], aq = S[j * m + q];
      S[j * m + p] = c * ap - s * aq;
      S[j * m + q] = s * ap + c * aq;
      const double vp = V[j * m + p], vq = V[j * m + q];
      V[j * m + p] = c * vp - s * vq;
      V[j * m + q] = s * vp + c * vq;
    }
    __syncthreads();
    if (tid == 0) { S[p * m + q] = 0.0; S[q * m + p] = 0.0; }
    __syncthreads();
    // row maxima: cheap updates first, then the rows to scan again
    for (int i = tid; i < m; i += nt) {
      rescan[i] = i == p || i == q || rarg[i] == p || rarg[i] == q;
      if (rescan[i]) continue;
      const double ap = fabs(S[i * m + p]), aq = fabs(S[i * m + q]);
      const int lo = p < q ? p : q, hi = p < q ? q : p;
      const double alo = lo == p ? ap : aq, ahi = lo == p ? aq : ap;
      if (alo > rmax[i] || (alo == rmax[i] && lo < rarg[i])) { rmax[i] = alo; rarg[i] = lo; }
      if (ahi > rmax[i] || (ahi == rmax[i] && hi < rarg[i])) { rmax[i] = ahi; rarg[i] = hi; }
    }
    __syncthreads();
    if (tid == 0) {  // the rows to scan again (more than 32: all rows, rare)
      int cnt = 0;
      bool all = false;
      for (int i = 0; i < m; ++i)
        if (rescan[i]) {
          if (cnt < 32) si[cnt++] = i;
          else all = true;
        }
      s_n = all ? -1 : cnt;
    }
    __syncthreads();
    const int nscan = s_n;
    if (nscan >= 0) {
      for (int r = wid; r < nscan; r += nw) scan_row(si[r]);
    } else {
      for (int i = wid; i < m; i += nw) scan_row(i);
    }
    __syncthreads();
  }
  for (int i = tid; i < m; i += nt) lam[i] = S[i * m + i];
}

// V = I (m x m)
__global__ void identity_fill_kernel(double* __restrict__ V, int m) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x)
    V[e] = ((e / m) == (e % m)) ? 1.0 : 0.0;
}

// dst = src (m x m) unless *skip
__global__ void copy_unless_kernel(const double* __restrict__ src, double* __restrict__ dst, int count,
                                   const int* __restrict__ skip) {
  if (*skip) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) dst[e] = src[e];
}

// R = I - G (in place, m x m) unless *skip
__global__ void identity_minus_kernel(double* __restrict__ G, int m, const int* __restrict__ skip) {
  if (*skip) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x)
    G[e] = ((e / m) == (e % m) ? 1.0 : 0.0) - G[e];
}

// Sort eigenpairs ascending by lam (one CTA, rank sort): w[rank]=lam[i],
// Vout[:, rank] = Vin[:, i].
__global__ void sort_pairs_kernel(const double* __restrict__ lam, const double* __restrict__ Vin, int m,
                                  double* __restrict__ w, double* __restrict__ Vout) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double li = lam[i];
    int rank = 0;
    for (int j = 0; j < m; ++j) rank += (lam[j] < li) || (lam[j] == li && j < i);
    w[rank] = li;
    for (int r = 0; r < m; ++r) Vout[r * m + rank] = Vin[r * m + i];
  }
}

// ---------------------------------------------------------------------------
// Cholesky G + shift*max(diag) I = L L^T and L^{-1}, one CTA, computed in TC.
// One m x m array in shared memory: L in the lower triangle (with diagonal),
// the strict lower part of L^{-1} stored transposed in the strict upper
// triangle (its diagonal is 1 / L_ii).  Output Linv (row-major m x m, lower
// triangular) in TO.  status[0] += 1 when a pivot was not positive (the pivot
// is then clamped).
// ---------------------------------------------------------------------------
// With `adaptive` set and G already within 1e-3 of the identity, the kernel
// instead writes the first-order inverse factor I - F^T (F upper triangular,
// F_ij = E_ij for i < j, F_ii = E_ii / 2, E = G - I), whose error is O(|E|^2).
// Threads of a launch: 1024 in FP32; 512 in FP64, where 1024 threads (64
// registers each) made the double-precision factorisation spill.
template <typename TC>
constexpr int cholinv_threads() { return sizeof(TC) == 8 ? 512 : 1024; }

template <typename TC, typename TI, typename TO>
__global__ void __launch_bounds__(cholinv_threads<TC>()) cholinv_kernel(const TI* __restrict__ G, int m, double shift,
                                                       TO* __restrict__ Linv, int* __restrict__ status,
                                                       int adaptive = 0) {
  extern __shared__ unsigned char smem_raw[];
  TC* L = (TC*)smem_raw;  // m x m
  __shared__ TC red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  if (adaptive) {
    TC emax = 0;
    for (int e = tid; e < m * m; e += nt) {
      const int i = e / m, j = e % m;
      emax = fmax(emax, fabs((TC)G[e] - (i == j ? TC(1) : TC(0))));
    }
    emax = block_max(emax, red);
    if (emax < TC(1e-3)) {
      for (int e = tid; e < m * m; e += nt) {
        const int i = e / m, j = e % m;
        TC v = 0;
        if (j < i) v = -TC(0.5) * ((TC)G[j * m + i] + (TC)G[i * m + j]);
        else if (j == i) v = TC(1) - TC(0.5) * ((TC)G[i * m + i] - TC(1));
        Linv[e] = (TO)v;
      }
      return;
    }
  }
  // L uses an odd row stride, so the column accesses of the factorisation and
  // of the solves hit distinct shared-memory banks (an even m put a whole
  // warp's column reads on one bank); dg holds the factor's diagonal, then
  // its reciprocals.
  const int ld = m | 1;
  TC* dg = L + (size_t)m * ld;
  TC dmax = 0;
  for (int i = tid; i < m; i += nt) dmax = fmax(dmax, (TC)G[i * m + i]);
  dmax = block_max(dmax, red);
  const TC sh = (TC)shift * dmax;
  for (int i = warp; i < m; i += nw)
    for (int j = lane; j < m; j += 32)
      L[i * ld + j] = (j <= i) ? (TC)(0.5 * ((double)G[i * m + j] + (double)G[j * m + i])) + (i == j ? sh : TC(0))
                               : TC(0);
  __syncthreads();
  const TC tiny = dmax * (TC)1e-30 + (TC)(sizeof(TC) == 4 ? 1e-37 : 1e-300);
  for (int j = 0; j < m; ++j) {
    // every thread reads the pivot (no thread writes it during this column)
    // and scales its own entries of column j
    TC d = L[j * ld + j];
    bool bad = !(d > tiny);
    if (bad) d = fmax(dmax, tiny) * (TC)1e-12;
    const TC ljj = sqrt(d);
    const TC inv = TC(1) / ljj;
    if (tid == 0) {
      dg[j] = ljj;
      if (bad && status) atomicAdd(status, 1);
    }
    for (int i = j + 1 + tid; i < m; i += nt) L[i * ld + j] *= inv;
    __syncthreads();
    for (int i = j + 1 + warp; i < m; i += nw) {
      const TC lij = L[i * ld + j];
      for (int k = j + 1 + lane; k <= i; k += 32) L[i * ld + k] -= lij * L[k * ld + j];
    }
    __syncthreads();
  }
  for (int i = tid; i < m; i += nt) {
    L[i * ld + i] = dg[i];
    dg[i] = TC(1) / dg[i];
  }
  __syncthreads();
  // L^{-1} by columns, one warp per column c: forward substitution of
  // L y = e_c with y held in registers (lane l owns y_{l + 32 q}); step t
  // finishes y_t on its owner lane, broadcasts it, and every lane removes it
  // from its later rows.  Li[i][c] (i > c) goes to L[c*ld + i], the strict
  // upper triangle, which the factor does not use.
  constexpr int kQ = (kMaxSmallDim + 31) / 32;
  for (int c = warp; c < m; c += nw) {
    TC y[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) y[q] = (lane + 32 * q == c) ? TC(1) : TC(0);
#pragma unroll
    for (int q0 = 0; q0 < kQ; ++q0) {  // y_t lives in y[q0] of lane t % 32
      const int t1 = min(m, 32 * q0 + 32);
      for (int t = max(c, 32 * q0); t < t1; ++t) {
        const TC yt = __shfl_sync(0xffffffffu, y[q0], t & 31) * dg[t];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          if (q < q0) continue;  // rows i > t >= 32 q0 only
          const int i = lane + 32 * q;
          if (i == t) y[q] = yt;
          else if (i > t && i < m) y[q] -= L[i * ld + t] * yt;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int i = lane + 32 * q;
      if (i > c && i < m) L[c * ld + i] = y[q];
    }
  }
  __syncthreads();
  for (int i = warp; i < m; i += nw)
    for (int c = lane; c < m; c += 32) {
      TO v = TO(0);
      if (c == i) v = (TO)dg[i];
      else if (c < i) v = (TO)L[c * ld + i];
      Linv[i * m + c] = v;
    }
}

inline size_t cholinv_smem_bytes(int m, size_t elt) { return ((size_t)m * (m | 1) + m) * elt; }

// out[i][r] = V[r][i] for i < k: the first k columns of a row-major m x m
// eigenvector matrix as k vectors of length m.
template <typename T>
__global__ void columns_to_vectors_kernel(const T* __restrict__ V, int m, int k, T* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * m; e += gridDim.x * blockDim.x) {
    const int i = e / m, r = e % m;
    out[e] = V[r * m + i];
  }
}

// out = a1 * P + a2 * Q (elementwise)
template <typename T>
__global__ void axpby_kernel(const T* __restrict__ P, const T* __restrict__ Q, long tot, T a1, T a2, T* __restrict__ out) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x)
    out[e] = a1 * P[e] + a2 * Q[e];
}

// Refinement in defect form (the mixed paths' FP64 refinement of wide
// blocks).  The per-column kernels below take a grid of (chunks of n, rows):
// blockIdx.y is the vector, so no index is divided per element.
inline dim3 rows_grid(long n, int rows) {
  const long chunks = (n + 1023) / 1024;
  return dim3((unsigned)std::max(1L, std::min(chunks, 64L)), (unsigned)std::max(1, rows));
}

// dst[j] = src[idx[j]] for whole vectors of length n (vector-major blocks)
template <typename T>
__global__ void gather_rows_kernel(const T* __restrict__ src, const int* __restrict__ idx, long n, T* __restrict__ dst) {
  const T* sr = src + (long)idx[blockIdx.y] * n;
  T* dr = dst + (long)blockIdx.y * n;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x) dr[r] = sr[r];
}

// dst[idx[j]] = src[j] for whole vectors of length n
template <typename T>
__global__ void scatter_rows_kernel(const T* __restrict__ src, const int* __restrict__ idx, long n, T* __restrict__ dst) {
  const T* sr = src + (long)blockIdx.y * n;
  T* dr = dst + (long)idx[blockIdx.y] * n;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x) dr[r] = sr[r];
}

// dst[idx[j]] = src[j], j < count
__global__ void scatter_values_kernel(const double* __restrict__ src, const int* __restrict__ idx, int count,
                                      double* __restrict__ dst) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < count) dst[idx[j]] = src[j];
}

// Rf = HC - C diag(w): the Ritz residuals, formed in FP64 and kept in FP32
// (they are small; FP32 keeps them to ~6e-8 of their own size).
__global__ void ritz_residual_kernel(const double* __restrict__ C, const double* __restrict__ HC,
                                     const double* __restrict__ w, long n, float* __restrict__ Rf) {
  const long o = (long)blockIdx.y * n;
  const double wi = w[blockIdx.y];
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x)
    Rf[o + r] = (float)(HC[o + r] - wi * C[o + r]);
}

// D[i][r] += s[i] * Rf[i][r]: the source term of the defect recurrence.
__global__ void add_scaled_columns_kernel(float* __restrict__ D, const float* __restrict__ Rf,
                                          const float* __restrict__ s, long n) {
  const long o = (long)blockIdx.y * n;
  const float si = s[blockIdx.y];
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x)
    D[o + r] += si * Rf[o + r];
}

// Y += F (FP32 addend into FP64).
__global__ void add_f32_kernel(double* __restrict__ Y, const float* __restrict__ F, long tot) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x)
    Y[e] += (double)F[e];
}

// For the basis Q = C + E (C orthonormal, E orthogonal to C up to the FP32
// rounding of E):
//   S  = Q^T Q - I = SCE + SCE^T + SEE,
//   Gm = Q^T H Q   = diag(theta) + CR + (C^T H E) + (E^T H C) + EHE,
// with C^T H E = (H C)^T E = R^T E + diag(theta) C^T E, i.e.
//   (C^T H E)_ij = RE_ij + theta_i SCE_ij, (E^T H C)_ij = RE_ji + theta_j SCE_ji.
// SCE = C^T E is the FP64-accurate Gram product (the FP32 rounding of a large
// guard-column correction has components along C that theta would magnify);
// CR = C^T R, RE = R^T E, SEE = E^T E, EHE = E^T H E are FP32 (each involves
// a small factor, or only guard-guard entries carry a large error).
__global__ void defect_gram_kernel(const double* __restrict__ SCE, const float* __restrict__ SEE,
                                   const float* __restrict__ CR, const float* __restrict__ RE,
                                   const float* __restrict__ EHE, const double* __restrict__ theta, int m,
                                   double* __restrict__ S, double* __restrict__ Gm) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int i = e / m, j = e % m;
    const int t = j * m + i;
    S[e] = SCE[e] + SCE[t] + (double)SEE[e];
    const double g = (double)CR[e] + (double)RE[e] + theta[i] * SCE[e] + (double)RE[t] + theta[j] * SCE[t] +
                     (double)EHE[e];
    const double gt = (double)CR[t] + (double)RE[t] + theta[j] * SCE[t] + (double)RE[e] + theta[i] * SCE[e] +
                      (double)EHE[t];
    Gm[e] = (i == j ? theta[i] : 0.0) + 0.5 * (g + gt);
  }
}

// E[i][r] = (float)(Dperp[i][r] / y[i]): each filtered column's correction
// outside span C, relative to its own amplification (one FP64 reciprocal a
// vector; the per-entry product in FP64).
__global__ void scale_columns_inv_kernel(const float* __restrict__ D, const double* __restrict__ y, long n,
                                         float* __restrict__ E) {
  const long o = (long)blockIdx.y * n;
  const double inv = 1.0 / y[blockIdx.y];
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x)
    E[o + r] = (float)((double)D[o + r] * inv);
}

// out = alpha I + beta A (m x m).
__global__ void shifted_identity_kernel(const double* __restrict__ A, int m, double alpha, double beta,
                                        double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x)
    out[e] = ((e / m) == (e % m) ? alpha : 0.0) + (A ? beta * A[e] : 0.0);
}

// Start of the scaled coupled Newton-Schulz iteration for (I + S)^{-1/2}
// (one CTA): c = 1 + trace(SEE) bounds the largest eigenvalue of I + S
// (S = C^T E + E^T C + E^T E with E orthogonal to C, so I + S >= I up to
// rounding and its excess is at most trace(E^T E)); Y = (I + S) / c has its
// spectrum in [1/c, 1], where the iteration converges.  c goes to *cdev.
__global__ void ns_start_kernel(const double* __restrict__ S, const float* __restrict__ SEE, int m,
                                double* __restrict__ Y, double* __restrict__ cdev) {
  __shared__ double red[32];
  __shared__ double cs;
  double t = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) t += fmax(0.0, (double)SEE[(long)i * m + i]);
  t = block_sum(t, red);
  if (threadIdx.x == 0) {
    cs = 1.0 + t;
    *cdev = cs;
  }
  __syncthreads();
  const double inv = 1.0 / cs;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) Y[e] = (((e / m) == (e % m) ? 1.0 : 0.0) + S[e]) * inv;
}

// W <- W / sqrt(c): undo the scaling of ns_start_kernel.
__global__ void scale_inv_sqrt_kernel(double* __restrict__ W, int m, const double* __restrict__ cdev) {
  const double f = 1.0 / sqrt(*cdev);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) W[e] *= f;
}

// F^T for the first-order second Cholesky-QR pass: G = I + E  =>  R ~ I + F,
// F upper triangular with F_ij = E_ij (i < j), F_ii = E_ii / 2; returns
// W = F^T (lower triangular) so that X_new = X - W X.
__global__ void cholqr_first_order_kernel(const double* __restrict__ G, int m, double* __restrict__ W) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int i = e / m, j = e % m;  // W[i][j] = F[j][i]
    double v = 0.0;
    if (j < i) v = 0.5 * (G[j * m + i] + G[i * m + j]);
    else if (j == i) v = 0.5 * (G[i * m + i] - 1.0);
    W[e] = v;
  }
}

// ---------------------------------------------------------------------------
// Leaf build from Pauli terms (Algorithm 1, first step): one CTA; each thread
// owns columns c of the D x D matrix and adds every term's single nonzero in
// that column.  Site s of an L-site block is bit (L-1-s) of the index (site 0
// is the most significant tensor factor).  Pauli codes: 1 = X, 2 = Y (carried
// as iY = [[0,1],[-1,0]]), 3 = Z.  A term is coef * P_{s0} P_{s1} (s1 < 0 for
// an on-site term).
// ---------------------------------------------------------------------------
struct PauliTerm {
  int s0, s1;
  int p0, p1;
  double coef;
};

__device__ __forceinline__ double pauli_apply(int code, int bit, int* flip) {
  // returns the factor of <r|P|c> for the column bit value `bit`; sets *flip
  if (code == 1) { *flip = 1; return 1.0; }
  if (code == 2) { *flip = 1; return bit ? 1.0 : -1.0; }  // iY|0> = -|1>, iY|1> = |0>
  *flip = 0;
  return bit ? -1.0 : 1.0;                                // Z
}

__global__ void pauli_matrix_kernel(const PauliTerm* __restrict__ terms, int n_terms, int L,
                                    double* __restrict__ M) {
  const int D = 1 << L;
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < D * D; e += blockDim.x * gridDim.x) M[e] = 0.0;
  __syncthreads();
  for (int c = threadIdx.x + blockIdx.x * blockDim.x; c < D; c += blockDim.x * gridDim.x) {
    for (int t = 0; t < n_terms; ++t) {
      const PauliTerm pt = terms[t];
      int r = c;
      double v = pt.coef;
      int flip;
      const int b0 = L - 1 - pt.s0;
      v *= pauli_apply(pt.p0, (c >> b0) & 1, &flip);
      if (flip) r ^= (1 << b0);
      if (pt.s1 >= 0) {
        const int b1 = L - 1 - pt.s1;
        v *= pauli_apply(pt.p1, (c >> b1) & 1, &flip);
        if (flip) r ^= (1 << b1);
      }
      M[(long)r * D + c] += v;
    }
  }
}

}  // namespace rmc
