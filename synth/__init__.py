"""Seeded synthetic LAPW+LO systems for the RT-TDDFT step.

This package only draws random numbers and lays out shapes (G-vector sets,
augmentation blocks, local-orbital counts, pulse samples).  It contains none
of the method's arithmetic: no Hamiltonian or overlap is applied or formed
here.  Both the CPU oracle and the CUDA path consume its output.
"""
from .system import (CONFIGS, make_system, pulse_samples, make_dv,
                     dv_scale_samples, basis_sizes, tiny_config)

__all__ = ["CONFIGS", "make_system", "pulse_samples", "make_dv",
           "dv_scale_samples", "basis_sizes", "tiny_config"]
