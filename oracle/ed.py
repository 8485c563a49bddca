"""Exact diagonalisation references built without any MPO (oracle; test only).

* Heisenberg chain: sparse Kronecker sums of S+S-, S-S+, SzSz.
* Electronic Hamiltonian of Sec. 3.2 in the full Fock space (R^{4^L} over
  spatial sites, local basis index n_up + 2 n_dn), from Jordan-Wigner matrices
  a_p = Z x ... x Z x c x I x ... (mode order 1up, 1dn, 2up, ...), with
  H = sum h_ij a+_{is} a_{js} + 1/2 sum (ij|kl) a+_{is} a+_{kt} a_{lt} a_{js}.
Both are used as independent pins of the MPOs and of the DMRG energies.
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def heisenberg_sparse(L, J=1.0):
    sp_ = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))
    sm_ = sp_.T.tocsr()
    sz = sp.csr_matrix(np.diag([0.5, -0.5]))

    def site_op(op, i):
        return sp.kron(sp.kron(sp.identity(2 ** i), op), sp.identity(2 ** (L - i - 1)),
                       format="csr")

    H = sp.csr_matrix((2 ** L, 2 ** L))
    for i in range(L - 1):
        H = H + J * (0.5 * site_op(sp_, i) @ site_op(sm_, i + 1)
                     + 0.5 * site_op(sm_, i) @ site_op(sp_, i + 1)
                     + site_op(sz, i) @ site_op(sz, i + 1))
    return H.tocsr()


def _annihilators(L):
    """a_p for p = 2i + s as sparse 4^L matrices in the TT index order."""
    Z = sp.csr_matrix(np.diag([1.0, -1.0]))
    c = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))
    I = sp.identity(2, format="csr")
    # Kronecker position order: (site0,dn), (site0,up), (site1,dn), ...
    positions = []
    for i in range(L):
        positions += [(i, 1), (i, 0)]
    ops = []
    for p in range(2 * L):
        mats = []
        for (i, s) in positions:
            q = 2 * i + s
            mats.append(Z if q < p else (c if q == p else I))
        m = mats[0]
        for x in mats[1:]:
            m = sp.kron(m, x, format="csr")
        ops.append(m.tocsr())
    return ops


def fermion_sparse(h, eri):
    L = h.shape[0]
    a = _annihilators(L)
    ad = [x.T.tocsr() for x in a]
    dim = 4 ** L
    H = sp.csr_matrix((dim, dim))
    for i, j in itertools.product(range(L), repeat=2):
        if h[i, j] != 0.0:
            for s in (0, 1):
                H = H + h[i, j] * (ad[2 * i + s] @ a[2 * j + s])
    for i, j, k, l in itertools.product(range(L), repeat=4):
        v = eri[i, j, k, l]
        if v == 0.0:
            continue
        for s, t in itertools.product((0, 1), repeat=2):
            H = H + 0.5 * v * (ad[2 * i + s] @ ad[2 * k + t] @ a[2 * l + t] @ a[2 * j + s])
    return H.tocsr()


def number_operator(L):
    a = _annihilators(L)
    N = sp.csr_matrix((4 ** L, 4 ** L))
    for x in a:
        N = N + x.T @ x
    return N.tocsr()


def ground_energy(H):
    if H.shape[0] <= 2048:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    return float(spla.eigsh(H, k=1, which="SA", tol=1e-14)[0][0])
