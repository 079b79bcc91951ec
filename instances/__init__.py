"""Seeded synthetic spin-chain instances shared by the oracle and the CUDA path.

This module only *describes* problems: which Pauli operator acts on which site
with which coefficient, how the chain is cut into leaves, and the truncation
parameters.  It holds none of the solver's arithmetic (no matrices, no
Kronecker products, no eigensolves), so that the oracle under ``oracle/`` and
the product under ``paper_2609_02394_b300/`` can both consume it while sharing
no code with each other.

Conventions (fixed here, read from the paper's problem statement):

* Sites are numbered 0..N-1 from the left; site 0 is the most significant
  tensor factor, module A is the left half and B the right half of a merge, so
  a nearest-neighbour bond couples A's last site to B's first site (Sec. III,
  Eq. (15)).
* A Hamiltonian is a sum of on-site terms ``(site, pauli, coef)`` and two-site
  terms ``(i, j, pauli_i, pauli_j, coef)`` with ``i < j`` and physical Pauli
  labels ``'X'``, ``'Y'``, ``'Z'``: H = sum coef * P_site + sum coef * P_i P_j.
  The inter-module coupling of Eq. (3), V = -sum J'_ij O_A,i (x) O_B,j, is the
  subset of two-site terms whose ends fall in different modules; its minus
  sign is folded into ``coef``.
* Models: transverse-field Ising H = -J sum Z_i Z_{i+1} - h sum X_i
  (Sec. III, Eq. (17)); XXZ H = sum J_i (X X + Y Y + Delta Z Z) with Pauli
  (not spin-1/2) normalisation; random-field Heisenberg = XXZ with Delta = 1,
  J = 1 plus sum h_i Z_i.  The paper defines only the Ising chain; the other
  two follow the same Pauli normalisation.
"""
from __future__ import annotations

import dataclasses
import json
from typing import List, Sequence, Tuple

import numpy as np

PAULIS = ("X", "Y", "Z")

OnSite = Tuple[int, str, float]
Bond = Tuple[int, int, str, str, float]


@dataclasses.dataclass
class Chain:
    """A 1-D spin-1/2 chain Hamiltonian plus the truncation parameters."""

    n_sites: int
    onsite: List[OnSite]
    bonds: List[Bond]
    leaf_sites: int  # L0: maximum sites per leaf module
    k: int           # retained states per intermediate block
    q: int           # lowest states wanted at the top
    name: str = ""

    def validate(self) -> None:
        if self.n_sites < 1:
            raise ValueError("chain needs at least one site")
        for s, p, _ in self.onsite:
            if not 0 <= s < self.n_sites or p not in PAULIS:
                raise ValueError(f"bad on-site term {(s, p)}")
            if p == "Y":
                raise ValueError("an on-site Y field is imaginary; real arithmetic only")
        for i, j, pi, pj, _ in self.bonds:
            if not (0 <= i < j < self.n_sites) or pi not in PAULIS or pj not in PAULIS:
                raise ValueError(f"bad bond {(i, j, pi, pj)}")
            if (pi == "Y") != (pj == "Y"):
                raise ValueError("a bond with a single Y factor is imaginary; real arithmetic only")
        if self.leaf_sites < 1 or self.k < 1 or self.q < 1:
            raise ValueError("leaf_sites, k and q must be positive")

    def to_json(self) -> str:
        return json.dumps(dataclasses.asdict(self))

    @staticmethod
    def from_json(text: str) -> "Chain":
        d = json.loads(text)
        d["onsite"] = [tuple(t) for t in d["onsite"]]
        d["bonds"] = [tuple(t) for t in d["bonds"]]
        return Chain(**d)


def tfim(n: int, J: float, h: float, leaf_sites: int, k: int, q: int) -> Chain:
    """Open transverse-field Ising chain, H = -J sum Z_i Z_{i+1} - h sum X_i."""
    onsite = [(i, "X", -float(h)) for i in range(n)]
    bonds = [(i, i + 1, "Z", "Z", -float(J)) for i in range(n - 1)]
    return Chain(n, onsite, bonds, leaf_sites, k, q, f"tfim_N{n}_J{J}_h{h:.6g}")


def xxz(n: int, Js: Sequence[float], delta: float, leaf_sites: int, k: int, q: int,
        fields: Sequence[float] | None = None, name: str = "") -> Chain:
    """Open XXZ chain, H = sum J_i (X X + Y Y + delta Z Z) [+ sum h_i Z_i]."""
    if len(Js) != n - 1:
        raise ValueError("need n-1 bond couplings")
    bonds: List[Bond] = []
    for i, Ji in enumerate(Js):
        bonds.append((i, i + 1, "X", "X", float(Ji)))
        bonds.append((i, i + 1, "Y", "Y", float(Ji)))
        bonds.append((i, i + 1, "Z", "Z", float(Ji) * float(delta)))
    onsite: List[OnSite] = []
    if fields is not None:
        onsite = [(i, "Z", float(hi)) for i, hi in enumerate(fields)]
    return Chain(n, onsite, bonds, leaf_sites, k, q, name or f"xxz_N{n}_D{delta}")


def two_module_tfim(geometry: str, Jp: float, k: int, q: int = 4, J: float = 1.0, h: float = 0.7,
                    gamma: float = 0.2) -> Chain:
    """Two five-site Ising modules (the block Hamiltonian of Appendix C) joined
    by one inter-module ZZ coupling -Jp at the sites of geometry I (A5-B1),
    II (A5-B2), III (A5-B3) or IV (A3-B3), 1-based within each module, or by
    the next-nearest form 'NNN': -Jp (A5-B1 + gamma A4-B1 + gamma A5-B2)."""
    onsite = [(i, "X", -float(h)) for i in range(10)]
    bonds: List[Bond] = [(i, i + 1, "Z", "Z", -float(J)) for m in (0, 5) for i in range(m, m + 4)]
    pairs = {"I": [(5, 1, 1.0)], "II": [(5, 2, 1.0)], "III": [(5, 3, 1.0)], "IV": [(3, 3, 1.0)],
             "NNN": [(5, 1, 1.0), (4, 1, gamma), (5, 2, gamma)]}[geometry]
    for a, b, w in pairs:
        bonds.append((a - 1, 5 + b - 1, "Z", "Z", -float(Jp) * w))
    return Chain(10, onsite, bonds, 5, k, q, f"tfim2x5_{geometry}_Jp{Jp:.3g}_k{k}")


def tfim_nnn(n: int, J: float, h: float, gamma: float, leaf_sites: int, k: int, q: int) -> Chain:
    """Ising chain with next-nearest ZZ couplings of relative strength gamma,
    H = -J sum (Z_i Z_{i+1} + gamma Z_i Z_{i+2}) - h sum X_i."""
    onsite = [(i, "X", -float(h)) for i in range(n)]
    bonds: List[Bond] = [(i, i + 1, "Z", "Z", -float(J)) for i in range(n - 1)]
    bonds += [(i, i + 2, "Z", "Z", -float(J) * float(gamma)) for i in range(n - 2)]
    return Chain(n, onsite, bonds, leaf_sites, k, q, f"tfim_nnn_N{n}_g{gamma:.3g}_L{leaf_sites}_k{k}")


def seed_for(config_index: int) -> int:
    """Seed of workload ``config_index`` (1-based): 2609*100 + index."""
    return 2609 * 100 + config_index


# --- the five workloads -------------------------------------------------------

def tfim_n8() -> Chain:
    """TFIM N=8, J=1, h=0.8, leaves of 2 spins, keep k=8, 4 lowest states."""
    return tfim(8, 1.0, 0.8, leaf_sites=2, k=8, q=4)


def xxz_n32(seed: int | None = None) -> Chain:
    """XXZ N=32, Delta=1, J_i ~ U[0.5,1.5], leaves of 4 spins, k=64, 8 lowest."""
    rng = np.random.default_rng(seed_for(2) if seed is None else seed)
    Js = rng.uniform(0.5, 1.5, size=31)
    return xxz(32, Js, 1.0, leaf_sites=4, k=64, q=8, name=f"xxz_N32_k64_seed{seed_for(2) if seed is None else seed}")


def sweep_points() -> List[Chain]:
    """256 TFIM points, h on a uniform grid in [0.2, 2.0], J=1, q=4; (N, k)
    assigned round-robin over {16,24,32,48} x {32,64,128}."""
    combos = [(N, k) for N in (16, 24, 32, 48) for k in (32, 64, 128)]
    out = []
    for i in range(256):
        h = 0.2 + 1.8 * i / 255.0
        N, k = combos[i % len(combos)]
        L0 = 3 if N in (24, 48) else 4
        c = tfim(N, 1.0, h, leaf_sites=L0, k=k, q=4)
        c.name = f"sweep{i}_N{N}_k{k}_h{h:.6f}"
        out.append(c)
    return out


def rf_heisenberg_n128(seed: int | None = None, k: int = 256) -> Chain:
    """Random-field Heisenberg N=128, Delta=1, J=1, h_i ~ U[-2,2], L0=4, 16 lowest."""
    s = seed_for(4) if seed is None else seed
    rng = np.random.default_rng(s)
    hs = rng.uniform(-2.0, 2.0, size=128)
    return xxz(128, [1.0] * 127, 1.0, leaf_sites=4, k=k, q=16, fields=hs,
               name=f"rfheis_N128_k{k}_seed{s}")


def rf_heisenberg_pair(seed: int | None = None) -> Chain:
    """Random-field Heisenberg, 24 sites, Delta = 1, J = 1, h_i ~ U[-2,2], two
    leaves of 12 sites, k = 256: its one merge couples two 256-state blocks
    (dimension 65536, three boundary operators), the shape of every merge above
    the first level of the 128-site chain, with inputs small enough to build
    densely (4096-dimensional leaves)."""
    s = seed_for(4) * 10 + 24 if seed is None else seed
    rng = np.random.default_rng(s)
    hs = rng.uniform(-2.0, 2.0, size=24)
    return xxz(24, [1.0] * 23, 1.0, leaf_sites=12, k=256, q=16, fields=hs, name=f"rfheis_N24_L12_k256_seed{s}")


def serving_requests(n_requests: int, seed: int | None = None) -> List[Chain]:
    """Mixed request stream: model uniform over {TFIM, XXZ, random field},
    N ~ U{8..128}, k in {16,32,64,128,256}, q ~ U{1..16} capped at k."""
    rng = np.random.default_rng(seed_for(5) if seed is None else seed)
    out = []
    for r in range(n_requests):
        model = int(rng.integers(0, 3))
        N = int(rng.integers(8, 129))
        k = int(rng.choice([16, 32, 64, 128, 256]))
        q = int(min(k, rng.integers(1, 17)))
        L0 = 4
        if model == 0:
            c = tfim(N, 1.0, float(rng.uniform(0.2, 2.0)), L0, k, q)
        elif model == 1:
            c = xxz(N, rng.uniform(0.5, 1.5, size=N - 1), 1.0, L0, k, q)
        else:
            c = xxz(N, [1.0] * (N - 1), 1.0, L0, k, q, fields=rng.uniform(-2, 2, size=N))
        c.name = f"req{r}_{c.name}"
        out.append(c)
    return out


def random_block_inputs(rng: np.random.Generator, kA: int, kB: int, n_ops: int,
                        spread: float = 4.0, scale: float = 0.5):
    """Random inputs of one merge in the retained bases (for kernel-level tests):
    ascending energies E_A, E_B, symmetric operators o_A[j], o_B[j] and term
    coefficients.  These are only random numbers of the right shape."""
    EA = np.sort(rng.uniform(-spread, spread, size=kA))
    EB = np.sort(rng.uniform(-spread, spread, size=kB))
    oA = rng.standard_normal((n_ops, kA, kA)) * scale
    oB = rng.standard_normal((n_ops, kB, kB)) * scale
    oA = 0.5 * (oA + oA.transpose(0, 2, 1))
    oB = 0.5 * (oB + oB.transpose(0, 2, 1))
    coef = rng.uniform(-1.0, 1.0, size=n_ops)
    return EA, EB, oA, oB, coef
