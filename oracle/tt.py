"""Tensor-train utilities (oracle; test infrastructure only).

Cores are float64 arrays [D_left][n][D_right] (Def. TT parameter space, Sec. 2.1).
Pinned by tests/test_oracle_tt.py: tt_full against brute-force products of
slices, orthogonality invariants, inner products against full vectors, and
tt_round against the SVD of the full tensor on tiny cases.
"""
import numpy as np


def tt_full(cores):
    """tau(U) of Def. (TT contraction mapping), as a C-ordered full vector."""
    v = cores[0].reshape(-1, cores[0].shape[2])           # (n0, r1)
    for c in cores[1:]:
        r, n, rr = c.shape
        v = (v @ c.reshape(r, n * rr)).reshape(-1, rr)
    return v.reshape(-1)


def qr_pos(M):
    """Reduced Householder QR, M = Q R, with diag(R) >= 0."""
    Q, R = np.linalg.qr(M, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s, (R.T * s).T


def lq_pos(M):
    """Reduced LQ, M = L Q, Q with orthonormal rows, diag(L) >= 0."""
    Q, R = qr_pos(M.T)
    return R.T, Q.T


def left_orthogonalize(cores):
    """QR sweep left to right: cores 0..L-2 left-orthogonal, last core holds the rest."""
    out = [c.copy() for c in cores]
    for j in range(len(out) - 1):
        Dl, n, Dr = out[j].shape
        Q, R = qr_pos(out[j].reshape(Dl * n, Dr))
        out[j] = Q.reshape(Dl, n, Q.shape[1])
        out[j + 1] = np.tensordot(R, out[j + 1], axes=(1, 0))
    return out


def right_orthogonalize(cores):
    """LQ sweep right to left: cores 1..L-1 right-orthogonal."""
    out = [c.copy() for c in cores]
    for j in range(len(out) - 1, 0, -1):
        Dl, n, Dr = out[j].shape
        Lf, Q = lq_pos(out[j].reshape(Dl, n * Dr))
        out[j] = Q.reshape(Q.shape[0], n, Dr)
        out[j - 1] = np.tensordot(out[j - 1], Lf, axes=(2, 0))
    return out


def tt_inner(a, b):
    """<tau(a), tau(b)> by left-to-right transfer matrices."""
    E = np.ones((1, 1))
    for ca, cb in zip(a, b):
        E = np.einsum("ab,asc,bsd->cd", E, ca, cb, optimize=True)
    return float(E[0, 0])


def tt_norm(a):
    return np.sqrt(max(tt_inner(a, a), 0.0))


def tt_scale(cores, alpha):
    out = [c.copy() for c in cores]
    out[-1] = out[-1] * alpha
    return out


def tt_add(terms, coeffs):
    """Plain TT sum sum_j c_j tau(terms[j]) with block-diagonal cores."""
    L = len(terms[0])
    out = []
    for k in range(L):
        blocks = [t[k] for t in terms]
        n = blocks[0].shape[1]
        if k == 0:
            core = np.concatenate([c * b for c, b in zip(coeffs, blocks)], axis=2)
        elif k == L - 1:
            core = np.concatenate(blocks, axis=0)
        else:
            Dl = sum(b.shape[0] for b in blocks)
            Dr = sum(b.shape[2] for b in blocks)
            core = np.zeros((Dl, n, Dr))
            i = j = 0
            for b in blocks:
                core[i:i + b.shape[0], :, j:j + b.shape[2]] = b
                i += b.shape[0]
                j += b.shape[2]
        if L == 1:
            core = sum(c * b for c, b in zip(coeffs, blocks))
        out.append(core)
    return out


def truncation_rank(s, D_max, tol):
    """Smallest r <= D_max with sqrt(sum_{k>=r} s_k^2) <= tol * ||s||_2, r >= 1.

    s must be sorted descending.  Returns (r, discarded 2-norm)."""
    s2 = s * s
    total = s2.sum()
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])   # tail[r] = sum_{k>=r}
    thr = (tol * tol) * total
    r = len(s)
    for cand in range(1, len(s) + 1):
        if tail[cand] <= thr:
            r = cand
            break
    r = max(1, min(r, D_max))
    return r, float(np.sqrt(tail[r]))


def svd_split(M, D_max, tol):
    """Truncated SVD M ~ P diag(s) Q (Alg. 1 step 2); returns P, s, Q, discarded."""
    P, s, Q = np.linalg.svd(M, full_matrices=False)
    r, disc = truncation_rank(s, D_max, tol)
    return P[:, :r], s[:r], Q[:r], disc


def tt_round(cores, D_max, tol):
    """Oseledets TT rounding: right-orthogonalise, then a left-to-right
    truncated-SVD sweep.  Output cores 0..L-2 are left-orthogonal."""
    out = right_orthogonalize(cores)
    disc_max = 0.0
    for j in range(len(out) - 1):
        Dl, n, Dr = out[j].shape
        P, s, Q, disc = svd_split(out[j].reshape(Dl * n, Dr), D_max, tol)
        disc_max = max(disc_max, disc / max(np.linalg.norm(s), 1e-300))
        out[j] = P.reshape(Dl, n, P.shape[1])
        out[j + 1] = np.tensordot(s[:, None] * Q, out[j + 1], axes=(1, 0))
    return out, disc_max
