"""Raw random TT cores for the seeded initial guess.

Bond dimensions are min(r0, exact maximal rank) with the exact maximal rank of
bond k equal to min(prod n_0..n_k, prod n_{k+1}..n_{L-1}).  Entries are
SplitMix64 uniforms on [-1, 1), filled site by site in row-major
[D_left][n][D_right] order from one stream.  No orthogonalisation is done here.
"""
import numpy as np

from .rng import SplitMix64


def tt_bond_dims(phys, r0):
    L = len(phys)
    dims = [1]
    for k in range(L - 1):
        left = int(np.prod(phys[:k + 1], dtype=object))
        right = int(np.prod(phys[k + 1:], dtype=object))
        dims.append(int(min(r0, left, right)))
    dims.append(1)
    return dims


def random_tt_cores(phys, r0, seed):
    dims = tt_bond_dims(phys, r0)
    g = SplitMix64(seed)
    cores = []
    for k, n in enumerate(phys):
        shape = (dims[k], n, dims[k + 1])
        cores.append(g.uniform_pm1(int(np.prod(shape))).reshape(shape))
    return cores
