"""GB300-native (sm_103a) two-site A2DMRG: C-ABI library + thin Python binding."""
from .a2dmrg import (A2Error, Context, MPO, TT, additive_sweep, classical_sweep, coarse_solve,
                     energy, env_update, heff_apply, lib, svd_split, gemm_bf16,
                     device_error, profile, PROFILE_KINDS, PRECISION, fold_split,
                     HeffOp, energy_gradient, energy_autograd, set_autotune, lq,
                     selftest_timeout, last_error)

__all__ = ["A2Error", "Context", "MPO", "TT", "additive_sweep", "classical_sweep",
           "coarse_solve", "energy", "env_update", "heff_apply", "lib", "svd_split", "PRECISION",
           "gemm_bf16", "device_error", "profile", "PROFILE_KINDS", "fold_split", "HeffOp",
           "energy_gradient", "energy_autograd", "set_autotune", "lq", "selftest_timeout",
           "last_error"]
