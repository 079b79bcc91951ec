"""Plain FP64 CPU oracle of the recursive module-coupling eigensolver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference arm use it.  It shares no code with the CUDA path:
both sides read problem *descriptions* from ``instances`` and nothing else.
"""
from .rmc_oracle import (  # noqa: F401
    Block,
    MergeRecord,
    OracleResult,
    block_hamiltonian,
    boundary_ops,
    carried_matrix,
    cut_rule,
    effective_hamiltonian,
    exact_spectrum,
    full_chain_hamiltonian,
    gauge_fix,
    leaf_block,
    merge_blocks,
    merge_terms,
    lift_states,
    pauli_matrix,
    rotate_operator,
    solve,
    sparse_exact_lowest,
    split_tree,
)
from . import closed_forms  # noqa: F401
