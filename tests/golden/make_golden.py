"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
Every value here comes from ``oracle/`` (Algorithm 1 with dense eigensolves,
or a closed form); nothing comes from the CUDA path.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import instances as I  # noqa: E402
from oracle import closed_forms as CF  # noqa: E402
from oracle import rmc_oracle as O  # noqa: E402


def dump(name, payload):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(payload, f, indent=1)
        f.write("\n")


def main():
    if "--bench-only" in sys.argv:
        return bench_batch()
    if "--rfheis-k128" in sys.argv:
        return rfheis_k128()
    if "--pair-65536" in sys.argv:
        return pair_65536()
    c1 = I.tfim_n8()
    r1 = O.solve(c1)
    c1f = I.tfim_n8(); c1f.k = 16
    dump("tfim_n8.json", {
        "source": "oracle (Algorithm 1, dense eigh) and exact diagonalisation of the 256-dim chain",
        "chain": c1.to_json(),
        "energies_k8": r1.energies.tolist(),
        "energies_k16": O.solve(c1f).energies.tolist(),
        "exact": O.exact_spectrum(c1, 4).tolist(),
        "merges": [[m.lo, m.mid, m.hi, m.k_ret, m.k_eff] for m in r1.merges],
    })
    c2 = I.xxz_n32()
    r2 = O.solve(c2)
    dump("xxz_n32_k64.json", {
        "source": "oracle (Algorithm 1, dense eigh), XXZ N=32, Delta=1, J_i~U[0.5,1.5] seed 260902",
        "chain": c2.to_json(),
        "energies": r2.energies.tolist(),
        "merges": [[m.lo, m.mid, m.hi, m.k_ret, m.k_eff] for m in r2.merges],
        "theta_low": [m.theta[: m.k_ret + 8].tolist() for m in r2.merges],
    })
    bench_batch()
    ff = {}
    for N in (16, 24, 32, 48, 64, 128):
        for h in (0.2, 0.7, 1.0, 2.0):
            ff[f"{N}_{h}"] = CF.tfim_lowest(N, 1.0, h, 16).tolist()
    dump("tfim_free_fermion.json", {
        "source": "free-fermion closed form (singular values of the bidiagonal h/J matrix)",
        "lowest16": ff,
    })


def bench_batch():
    """The benchmark batch: XXZ N=32 instances with independent bond draws."""
    seeds = [I.seed_for(2) + 7919 * i for i in range(32)]
    batch = []
    for sd in seeds:
        ch = I.xxz_n32(sd)
        batch.append({"seed": sd, "energies": O.solve(ch).energies.tolist()})
    dump("bench_xxz_n32_k64.json", {
        "source": "oracle (Algorithm 1, dense eigh): XXZ N=32, Delta=1, J_i~U[0.5,1.5] per seed, L0=4, k=64, q=8",
        "instances": batch,
    })


def rfheis_k128():
    """The 128-site random-field Heisenberg chain at k = 128: fifteen merges of
    dimension 16384, dense (the lowest k_ret + 1 eigenpairs of each from dsyevr).
    Takes about an hour on 8 host cores."""
    t0 = time.time()
    c = I.rf_heisenberg_n128(k=128)
    r = O.solve(c)
    dump("rfheis_n128_k128.json", {
        "source": "oracle (Algorithm 1, dense H_eff of every merge; lowest k_ret+1 eigenpairs by LAPACK dsyevr "
                  "above 4096 rows): random-field Heisenberg N=128, h_i~U[-2,2] seed 260904, L0=4, k=128, q=16",
        "chain": c.to_json(),
        "energies": r.energies.tolist(),
        "merges": [[m.lo, m.mid, m.hi, m.k_ret, m.k_eff] for m in r.merges],
        "theta_low": [m.theta[: m.k_ret + 1].tolist() for m in r.merges],
        "host_seconds": time.time() - t0,
    })


def pair_65536():
    """One merge of two 256-state blocks (dimension 65536): the 24-site
    random-field chain with 12-site leaves.  The leaves are dense 4096 x 4096
    eigensolves; the merge's dense H_eff (34 GB) gives its lowest 257
    eigenvalues by dsyevr.  Needs ~40 GB of host memory and about an hour on
    8 cores."""
    t0 = time.time()
    c = I.rf_heisenberg_pair()
    A = O.leaf_block(c, 0, 12, c.k)
    B = O.leaf_block(c, 12, 24, c.k)
    blk, rec = O.merge_blocks(c, A, B, c.k, False)
    dump("rfheis_pair_n65536.json", {
        "source": "oracle (leaves: dense eigh of 4096 x 4096; merge: dense 65536 x 65536 H_eff of Eq. (7), lowest "
                  "257 eigenpairs by LAPACK dsyevr): random-field Heisenberg N=24, L0=12, k=256, seed 2609064",
        "chain": c.to_json(),
        "leaf_k": [len(A.E), len(B.E)],
        "leaf_E0": [float(A.E[0]), float(B.E[0])],
        "k_ret": rec.k_ret, "k_eff": rec.k_eff,
        "theta": rec.theta.tolist(),
        "host_seconds": time.time() - t0,
    })


if __name__ == "__main__":
    main()
