"""Reduced density matrices of a full state vector and the gradient of the energy with
respect to the Hamiltonian's coefficients (oracle; test only).

For H(h, eri) = sum h_ij a+_{is} a_{js} + 1/2 sum eri_ijkl a+_{is} a+_{kt} a_{lt} a_{js}
(Jordan-Wigner matrices of oracle.ed) the energy of a fixed normalised state is linear
in the coefficients, so its gradient is the reduced density matrices:
    dE/dh[i, j]         = sum_s   <a+_{is} a_{js}>                (one-particle RDM)
    dE/deri[i, j, k, l] = 1/2 sum_{s,t} <a+_{is} a+_{kt} a_{lt} a_{js}>   (two-particle)
(Hellmann-Feynman; at an eigenstate the same numbers are the total derivative of the
eigenvalue).  Pinned in tests/test_gradient_oracle.py by the identity
<psi|H|psi> = sum h * dE/dh + sum eri * dE/deri against oracle.ed.fermion_sparse.
"""
import itertools

import numpy as np

from oracle.ed import _annihilators


def hamiltonian_gradient(psi, L):
    psi = np.asarray(psi, dtype=np.float64).ravel()
    psi = psi / np.linalg.norm(psi)
    a = _annihilators(L)
    ad = [x.T.tocsr() for x in a]
    a_psi = [x @ psi for x in a]                      # a_p |psi>
    gh = np.zeros((L, L))
    for i, j in itertools.product(range(L), repeat=2):
        gh[i, j] = sum(float(a_psi[2 * i + s] @ a_psi[2 * j + s]) for s in (0, 1))
    geri = np.zeros((L, L, L, L))
    # <a+_i a+_k a_l a_j> = <(a_k a_i) psi, (a_l a_j) psi>
    pair = {}
    for p, q in itertools.product(range(2 * L), repeat=2):
        pair[(p, q)] = a[p] @ a_psi[q]                # a_p a_q |psi>
    for i, j, k, l in itertools.product(range(L), repeat=4):
        v = 0.0
        for s, t in itertools.product((0, 1), repeat=2):
            v += float(pair[(2 * k + t, 2 * i + s)] @ pair[(2 * l + t, 2 * j + s)])
        geri[i, j, k, l] = 0.5 * v
    return gh, geri
