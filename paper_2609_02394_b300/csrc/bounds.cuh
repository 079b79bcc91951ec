// Kernels of the per-merge truncation diagnostics (Sec. IV and Appendix B):
// the merged block's own Hamiltonian applied on its 2^L computational basis,
// and a seeded start vector for the Krylov solves on that space.
#pragma once

#include "common.cuh"

namespace rmc {

// One Pauli-string term of a block Hamiltonian on L sites (site 0 is the most
// significant bit of the basis index).  In real arithmetic every single-site
// factor maps a basis state to one basis state with a sign:
//   X:  |s> -> |s ^ bit>                 (flip)
//   Z:  |s> -> (-1)^bit |s>              (sign)
//   iY: |s> -> (-1)^bit |s ^ bit> on the output index, i.e. (iY x)[0] = x[1],
//       (iY x)[1] = -x[0]                (flip and sign)
// and factors on distinct sites commute through each other's masks, so
//   (term x)[s] = coef * (-1)^popcount(s & sign) * x[s ^ flip].
// A physical YY bond of coefficient c is the term -c (iY)(iY).
struct FullTerm {
  unsigned long long flip, sign;
  double coef;
};

// y = sum_t term_t x over a vector of dim = 2^L entries (grid-stride; the
// term table is small and read through L1 by every thread alike).
__global__ void full_apply_kernel(const FullTerm* __restrict__ terms, int nt, long dim, const double* __restrict__ x,
                                  double* __restrict__ y) {
  for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < dim; s += (long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int t = 0; t < nt; ++t) {
      const FullTerm ft = terms[t];
      const double v = ft.coef * x[(unsigned long long)s ^ ft.flip];
      acc += (__popcll((unsigned long long)s & ft.sign) & 1) ? -v : v;
    }
    y[s] = acc;
  }
}

// x[i] uniform in [-1, 1) from a splitmix64 sequence keyed by (seed, i):
// a reproducible start vector with a component along every eigenvector.
__global__ void seeded_vector_kernel(double* __restrict__ x, long n, unsigned long long seed) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    unsigned long long z = seed * 0x9E3779B97F4A7C15ull + (unsigned long long)i + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

}  // namespace rmc
