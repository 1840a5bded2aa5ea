"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package draws random numbers and evaluates the Slater-Koster model
that stands in for the paper's DFT Hamiltonian and overlap (Sec. 2.2,
Eq. 2).  It contains none of the method's own arithmetic: no range
masks, no truncated products, no LNV energy, gradient or line search.
Both the oracle and the GPU path call it with their own pair lists.
"""
from .silicon import (  # noqa: F401
    A_SI, SEED_BASE, diamond_si_positions, sk_blocks, SK_H, SK_S, config_seed,
    batch_system_seed, batch_workload, md_trajectory,
)
