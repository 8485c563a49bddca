"""Seeded synthetic inputs shared by the oracle and the GPU path.

This package holds only input generation: the SplitMix64 counter generator,
the synthetic one- and two-body integrals, exact operator-string (finite-state)
matrix-product-operator construction for the Heisenberg chain and the
second-quantised electronic Hamiltonian, and the raw random TT cores used as
initial guesses.  It contains none of the A2DMRG arithmetic (no
orthogonalisation, no eigensolver, no truncation, no coarse step); both the
oracle and the CUDA path take these arrays as their inputs.
"""
from .rng import SplitMix64, uniform_pm1, standard_normal
from .hamiltonians import (heisenberg_mpo, chemistry_integrals, chemistry_mpo,
                           hubbard_integrals)
from .tt_init import random_tt_cores, tt_bond_dims
from .configs import CONFIGS, get_config

__all__ = ["SplitMix64", "uniform_pm1", "standard_normal", "heisenberg_mpo",
           "chemistry_integrals", "chemistry_mpo", "hubbard_integrals",
           "random_tt_cores", "tt_bond_dims", "CONFIGS", "get_config"]
