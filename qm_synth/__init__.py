"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds NO arithmetic of the method (no G-sphere, no FFT grid rule, no
Hamiltonian, no eigensolver).  It only describes the synthetic Si-like cells
(lattice, atom sites, k-points, cutoffs, band counts), evaluates the synthetic
potential V_loc(r) and the Gaussian projector functions beta(q) at points the
caller supplies, and draws seeded random numbers.  Both sides of every parity
test consume exactly the arrays produced here.
"""
from .cells import (Cell, config1, config2, config3_cells, config4, config5, small_cells, fcc_si2, cubic_si8,
                    fcc_supercell, KPTS_MP222_SHIFTED_FULL)
from .fields import vloc_on_grid, beta_of_q, dvals, psi_random, psi_random_real

__all__ = [
    "Cell", "config1", "config2", "config3_cells", "fcc_supercell", "KPTS_MP222_SHIFTED_FULL", "config4", "config5", "small_cells", "fcc_si2",
    "cubic_si8", "vloc_on_grid", "beta_of_q", "dvals", "psi_random", "psi_random_real",
]
