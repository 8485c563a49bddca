"""MPO helpers (oracle; test infrastructure only).

MPO cores are W[w_l, s, t, w_r] (s = bra/output, t = ket/input), eq. MPO.
mpo_dense is pinned against exact diagonalisation Hamiltonians built
independently from Jordan-Wigner matrices (tests/test_oracle_ed.py).
"""
import numpy as np

from .tt import tt_round


def mpo_dense(cores):
    """Full operator matrix (prod n) x (prod n) of the MPO, C-ordered sites."""
    M = cores[0][0]                                     # (n, n, R1)
    dim = M.shape[0]
    for c in cores[1:]:
        Rl, n, _, Rr = c.shape
        # M[(S),(T),w] x c[w,s,t,w'] -> [(S s),(T t),w']
        M = np.einsum("STw,wstv->SsTtv", M, c, optimize=True)
        dim *= n
        M = M.reshape(dim, dim, Rr)
    return M[:, :, 0]


def mpo_apply_full(cores, x):
    return mpo_dense(cores) @ x


def mpo_compress(cores, tol):
    """Compress an MPO by TT rounding of its cores viewed with merged (s,t)."""
    L = len(cores)
    tt = [c.reshape(c.shape[0], c.shape[1] * c.shape[2], c.shape[3]) for c in cores]
    out, _ = tt_round(tt, 1 << 30, tol)
    res = []
    for c, o in zip(cores, out):
        n = c.shape[1]
        res.append(np.ascontiguousarray(o.reshape(o.shape[0], n, n, o.shape[2])))
    return res
