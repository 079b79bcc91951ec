"""Closed-form spectra that pin the oracle independently of its own code.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Transverse-field Ising open chain, H = -J sum Z_i Z_{i+1} - h sum X_i
  (Sec. III, Eq. (17)).  Jordan-Wigner maps it to free fermions (Sec. III,
  Eqs. (18)-(19) give the infinite-chain dispersion).  On the open chain the
  single-particle energies are 2 s_m, where s_m are the singular values of the
  N x N upper-bidiagonal matrix with h on the diagonal and J on the
  superdiagonal; the ground energy is -sum s_m and every eigenvalue is
  -sum s_m + 2 sum_{m in S} s_m over subsets S of modes (all fermion parities
  occur on the open chain).  This is the "exact free-fermion reference energy"
  the paper measures its errors against (Sec. IV, Eq. (22)).
* XX chain (the XXZ chain at Delta = 0), H = sum J_i (X X + Y Y): XX + YY =
  2 (s+ s- + s- s+), so it is a free-fermion hopping chain with amplitude
  2 J_i; the single-particle energies are the eigenvalues of the tridiagonal
  matrix T with T[i, i+1] = T[i+1, i] = 2 J_i (4 J cos(m pi / (N+1)) for a
  uniform chain) and every eigenvalue is a subset sum.
* Two-site textbook cases used to pin the Pauli builder.
"""
from __future__ import annotations

import itertools
import math
from typing import List, Sequence

import numpy as np


def tfim_modes(n: int, J: float, h: float) -> np.ndarray:
    """Single-particle half-energies s_m (ascending) of the open TFIM chain."""
    M = np.zeros((n, n))
    for i in range(n):
        M[i, i] = h
        if i + 1 < n:
            M[i, i + 1] = J
    return np.sort(np.linalg.svd(M, compute_uv=False))


def _lowest_subset_sums(base: float, excitations: Sequence[float], count: int) -> np.ndarray:
    """The ``count`` smallest values of base + sum_{m in S} e_m over subsets S,
    for non-negative e_m (ascending).  Exhaustive over the smallest modes: a
    subset containing a mode larger than the count-th smallest single
    excitation can never be among the lowest ``count`` values, so only
    ``min(len, count)`` modes (at most 20) need to be enumerated."""
    e = np.sort(np.asarray(excitations, dtype=float))
    m = min(len(e), count, 20)
    small = e[:m]
    sums = [0.0]
    for r in range(1, m + 1):
        for comb in itertools.combinations(range(m), r):
            sums.append(float(small[list(comb)].sum()))
    sums = np.sort(np.array(sums))[:count]
    return base + sums


def tfim_lowest(n: int, J: float, h: float, count: int) -> np.ndarray:
    """Lowest ``count`` eigenvalues of the open TFIM chain (free fermions)."""
    s = tfim_modes(n, J, h)
    return _lowest_subset_sums(-float(s.sum()), 2.0 * s, count)


def tfim_ground_energy(n: int, J: float, h: float) -> float:
    return -float(tfim_modes(n, J, h).sum())


def xx_modes(Js: Sequence[float]) -> np.ndarray:
    """Single-particle energies of the open XX chain with bond couplings J_i."""
    n = len(Js) + 1
    T = np.zeros((n, n))
    for i, Ji in enumerate(Js):
        T[i, i + 1] = T[i + 1, i] = 2.0 * Ji
    return np.sort(np.linalg.eigvalsh(T))


def xx_lowest(Js: Sequence[float], count: int) -> np.ndarray:
    """Lowest ``count`` eigenvalues of the open XX chain: fill every negative
    mode for the ground state; an excitation adds |eps| of one mode (emptying
    a negative mode or filling a positive one)."""
    eps = xx_modes(Js)
    base = float(eps[eps < 0].sum())
    return _lowest_subset_sums(base, np.abs(eps), count)


def xx_uniform_modes(n: int, J: float) -> np.ndarray:
    """4 J cos(m pi/(n+1)), m = 1..n: the uniform XX chain's mode energies."""
    return np.sort(np.array([4.0 * J * math.cos(m * math.pi / (n + 1)) for m in range(1, n + 1)]))


def two_site_tfim(J: float, h: float) -> np.ndarray:
    """Spectrum of -J Z Z - h (X I + I X): -sqrt(J^2+4h^2), -J, J, sqrt(J^2+4h^2).
    In the X eigenbasis Z Z flips both spins: the pair {|++>, |-->} forms the
    block [[-2h, -J], [-J, 2h]] (eigenvalues -+sqrt(J^2 + 4h^2)) and the pair
    {|+->, |-+>} the block [[0, -J], [-J, 0]] (eigenvalues -+J)."""
    r = math.sqrt(J * J + 4 * h * h)
    return np.sort(np.array([-r, -J, J, r]))


def two_site_heisenberg(J: float) -> np.ndarray:
    """J (X X + Y Y + Z Z) on two spins: singlet -3J, triplet +J (x3)."""
    return np.sort(np.array([-3.0 * J, J, J, J]))


def heisenberg_multiplet_sizes(n: int) -> List[int]:
    """Dimensions 2S+1 of the total-spin multiplets of n spin-1/2 (with
    multiplicity), a check that an SU(2)-symmetric spectrum clusters right."""
    out = []
    for twoS in range(n % 2, n + 1, 2):
        S2 = twoS
        # multiplicity of total spin S among n spins-1/2
        mult = math.comb(n, (n - S2) // 2) - (math.comb(n, (n - S2) // 2 - 1) if (n - S2) // 2 >= 1 else 0)
        out += [S2 + 1] * mult
    return out
