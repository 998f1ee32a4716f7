"""FP64 CPU oracle of the RT-TDDFT auxiliary-subspace step (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this package.  The CUDA library never imports, links or calls it.
"""
from .rttddft_oracle import (Oracle, explicit_operators, explicit_dv, hamiltonian,
                             interstitial_potential, embedding, ritz_basis, fix_phases,
                             propagate_exact, propagate_cn, critical_timestep,
                             overall_speedup, full_basis_propagator, polarizability, F_CRIT,
                             interstitial_density, hartree_table, mt_density)

__all__ = ["Oracle", "explicit_operators", "explicit_dv", "hamiltonian",
           "interstitial_potential", "embedding", "ritz_basis", "fix_phases",
           "propagate_exact", "propagate_cn", "critical_timestep", "overall_speedup",
           "full_basis_propagator", "polarizability", "F_CRIT",
           "interstitial_density", "hartree_table", "mt_density"]
