"""Particle-number preserving tensor trains with U(1) x U(1) charges (oracle; test
infrastructure only: nothing on the GPU path imports it).

Sec. 3.2 (particle-number constraint): a TT that is an eigenfunction of the number
operators has block-sparse cores.  Every bond index carries the charge q = (N_up, N_dn) of
the modes to its left; a core entry U[a, s, b] can be nonzero only where
q_right[b] = q_left[a] + q(s), q(s) the occupation of local state s (index n_up + 2 n_dn,
the basis of synthetic.hamiltonians and oracle.ed).  The two-site DMRG micro-iteration
preserves the structure (the projected operator commutes with the number operators), and
so do linear combinations of such TTs; what must be adapted is every factorisation: the
truncated SVD and the orthogonalising LQ act on the nonzero blocks one charge at a time,
the truncation choosing the kept singular values over all blocks together (Sec. 3.2, the
block-wise SVD of the particle-preserving TT rounding).

Representation: dense cores plus a charge label per bond index ("masked dense"); every
operation keeps the entries outside the allowed pattern exactly zero.  The charged
versions of the classical two-site sweep (Alg. 1) and of the A2DMRG global iteration
(Alg. 2) reuse the dense environment, H_eff, Lanczos, coarse-solve and TT-sum code of this
package and replace only the factorisations.  Pinned by tests/test_oracle_blocksparse.py:
block-wise truncated SVD against the dense one of the same block-diagonal matrix, support
of every TT on its sector, exact particle numbers in the truncating regime, the U = 0
free-fermion closed form and exact diagonalisation in the sector (Hubbard, L <= 6).
"""
import numpy as np

from .coarse import coarse_solve
from .env import env_left_update, heff_apply, left_envs, right_envs, sandwich
from .lanczos import lanczos_lowest
from .tt import lq_pos, truncation_rank, tt_add, tt_full, tt_inner, tt_scale


# ----------------------------------------------------------------------- charges
def local_charges(n=4):
    """q(s) for the local basis s = n_up + 2 n_dn (n = 4) of a spatial orbital."""
    assert n == 4, "charged TTs are defined for spatial orbitals (n = 4)"
    return np.array([[s & 1, s >> 1] for s in range(n)], dtype=np.int64)


def core_mask(ql, qr, qs):
    """Allowed entries of a core: mask[a, s, b] = (ql[a] + qs[s] == qr[b])."""
    tot = ql[:, None, None, :] + qs[None, :, None, :]
    return np.all(tot == qr[None, None, :, :], axis=3)


def two_site_mask(ql, qr, qs):
    tot = ql[:, None, None, None, :] + qs[None, :, None, None, :] + qs[None, None, :, None, :]
    return np.all(tot == qr[None, None, None, :, :], axis=4)


def _count(m, k):
    """Number of ways to place k particles of one spin on m orbitals."""
    if k < 0 or k > m:
        return 0
    from math import comb
    return comb(m, k)


def reachable(L, j, Nu, Nd):
    """Charges (n_up, n_dn) a bond after j of L orbitals can carry in the sector (Nu, Nd),
    with the dimensions of the left and right spaces that carry them."""
    out = []
    for nu in range(max(0, Nu - (L - j)), min(j, Nu) + 1):
        for nd in range(max(0, Nd - (L - j)), min(j, Nd) + 1):
            left = _count(j, nu) * _count(j, nd)
            right = _count(L - j, Nu - nu) * _count(L - j, Nd - nd)
            out.append(((nu, nd), left, right))
    return out


def random_charged_tt(L, Nu, Nd, D, seed):
    """A TT in the sector (Nu, Nd): bond charges spread over the reachable charges (at most
    min(left, right) indices per charge, at most D per bond), seeded normal entries on the
    allowed positions.  Returns (cores, q) with q[j] the (D_j x 2) charges of bond j."""
    rng = np.random.default_rng(seed)
    qs = local_charges()
    q = [np.zeros((1, 2), dtype=np.int64)]
    for j in range(1, L):
        opts = reachable(L, j, Nu, Nd)
        caps = [min(l, r) for _, l, r in opts]
        mult = [0] * len(opts)
        total = 0
        while total < D and any(m < c for m, c in zip(mult, caps)):
            for i in range(len(opts)):      # round robin over the charges
                if total < D and mult[i] < caps[i]:
                    mult[i] += 1
                    total += 1
        lab = [opts[i][0] for i in range(len(opts)) for _ in range(mult[i])]
        q.append(np.array(lab, dtype=np.int64).reshape(-1, 2))
    q.append(np.array([[Nu, Nd]], dtype=np.int64))
    cores = []
    for j in range(L):
        m = core_mask(q[j], q[j + 1], qs)
        cores.append(rng.standard_normal(m.shape) * m)
    nrm = np.sqrt(tt_inner(cores, cores))
    return tt_scale(cores, 1.0 / nrm), q


def particle_numbers(cores):
    """(<N_up>, <N_dn>, <N_up^2> - <N_up>^2 + <N_dn^2> - <N_dn>^2) of tau(cores) / norm,
    from the full vector (small L)."""
    v = tt_full(cores)
    L = len(cores)
    idx = np.arange(v.size)
    nu = np.zeros(v.size)
    nd = np.zeros(v.size)
    for j in range(L):
        s = (idx // 4 ** (L - 1 - j)) % 4
        nu += s & 1
        nd += s >> 1
    p = v * v / (v @ v)
    mu, md = p @ nu, p @ nd
    var = p @ (nu - mu) ** 2 + p @ (nd - md) ** 2
    return float(mu), float(md), float(var)


def sector_support(cores, Nu, Nd):
    """Largest |entry| of the full vector outside the sector (Nu, Nd)."""
    v = tt_full(cores)
    L = len(cores)
    idx = np.arange(v.size)
    nu = np.zeros(v.size, dtype=np.int64)
    nd = np.zeros(v.size, dtype=np.int64)
    for j in range(L):
        s = (idx // 4 ** (L - 1 - j)) % 4
        nu += s & 1
        nd += s >> 1
    out = (nu != Nu) | (nd != Nd)
    return float(np.abs(v[out]).max()) if out.any() else 0.0


# ------------------------------------------------------------- block factorisations
def _groups(qrow, qcol):
    """Common charges of a block-diagonal matrix and their row / column index sets."""
    keys = sorted(set(map(tuple, qrow)) & set(map(tuple, qcol)))
    out = []
    for c in keys:
        r = np.nonzero(np.all(qrow == c, axis=1))[0]
        k = np.nonzero(np.all(qcol == c, axis=1))[0]
        out.append((np.array(c, dtype=np.int64), r, k))
    return out


def block_svd_split(M, qrow, qcol, D_max, tol):
    """Truncated SVD M ~ P diag(s) Q of a matrix that is block diagonal in the charges
    (M[r, c] = 0 unless qrow[r] == qcol[c]), block by block: the singular values of all
    blocks are ranked together and the smallest r <= D_max with discarded 2-norm
    <= tol * ||s|| is kept (the rule of the dense split).  Returns P (rows x r),
    s (descending), Q (r x cols), the discarded 2-norm and the charges of the r kept
    indices."""
    parts = []
    for c, ri, ci in _groups(qrow, qcol):
        if len(ri) == 0 or len(ci) == 0:
            continue
        U, s, Vt = np.linalg.svd(M[np.ix_(ri, ci)], full_matrices=False)
        for k in range(len(s)):
            parts.append((s[k], c, ri, ci, U[:, k], Vt[k]))
    if not parts:   # a zero matrix: keep one (zero) direction of the first row's charge
        P = np.zeros((M.shape[0], 1))
        P[0, 0] = 1.0
        return P, np.zeros(1), np.zeros((1, M.shape[1])), 0.0, qrow[:1].copy()
    order = sorted(range(len(parts)), key=lambda t: -parts[t][0])
    s_all = np.array([parts[t][0] for t in order])
    r, disc = truncation_rank(s_all, D_max, tol)
    P = np.zeros((M.shape[0], r))
    Q = np.zeros((r, M.shape[1]))
    qnew = np.zeros((r, 2), dtype=np.int64)
    for k, t in enumerate(order[:r]):
        s, c, ri, ci, u, vt = parts[t]
        P[ri, k] = u
        Q[k, ci] = vt
        qnew[k] = c
    return P, s_all[:r], Q, disc, qnew


def block_lq(M, qrow, qcol):
    """M = L Q block by block (Q with orthonormal rows, diag(L) >= 0 in every block).
    Returns L (rows x k), Q (k x cols) and the charges of the k new indices."""
    Ls, Qs, qs_ = [], [], []
    blocks = []
    for c, ri, ci in _groups(qrow, qcol):
        if len(ri) == 0 or len(ci) == 0:
            continue
        Lb, Qb = lq_pos(M[np.ix_(ri, ci)])
        blocks.append((c, ri, ci, Lb, Qb))
    k = sum(b[3].shape[1] for b in blocks)
    Lm = np.zeros((M.shape[0], max(k, 1)))
    Qm = np.zeros((max(k, 1), M.shape[1]))
    qn = np.zeros((max(k, 1), 2), dtype=np.int64)
    off = 0
    for c, ri, ci, Lb, Qb in blocks:
        kb = Lb.shape[1]
        Lm[np.ix_(ri, np.arange(off, off + kb))] = Lb
        Qm[np.ix_(np.arange(off, off + kb), ci)] = Qb
        qn[off:off + kb] = c
        off += kb
    if k == 0:
        qn[0] = qrow[0]
    return Lm, Qm, qn


def _row_charges(ql, qs):
    """Charges of the rows (a, s) of a core reshaped to (Dl n) x Dr."""
    return (ql[:, None, :] + qs[None, :, :]).reshape(-1, 2)


def _col_charges(qr, qs):
    """Charges of the columns (s, b) of a core reshaped to Dl x (n Dr): what the left
    bond must carry, q_right[b] - q(s)."""
    return (qr[None, :, :] - qs[:, None, :]).reshape(-1, 2)


def charged_orthogonal_copies(U, q):
    """Alg. 2 step 1 with charges: right-orthogonal cores V[i] (i >= 1), centres C[i] and the
    charges qV[i] of the bonds of V (qV[i] for the bond left of core i)."""
    qs = local_charges()
    L = len(U)
    V, C = [None] * L, [None] * L
    qV = list(q)
    C[L - 1] = U[L - 1].copy()
    for i in range(L - 1, 0, -1):
        Dl, n, Dr = C[i].shape
        Lf, Qm, qn = block_lq(C[i].reshape(Dl, n * Dr), q[i], _col_charges(qV[i + 1], qs))
        V[i] = Qm.reshape(-1, n, Dr)
        qV[i] = qn
        C[i - 1] = np.tensordot(U[i - 1], Lf, axes=(2, 0))
    return V, C, qV


def charged_round(cores, q, D_max, tol):
    """Particle-preserving TT rounding: block-wise right-orthogonalisation, then a
    left-to-right block-wise truncated SVD.  Returns (cores, charges, max relative
    discarded)."""
    qs = local_charges()
    out = [c.copy() for c in cores]
    qq = list(q)
    for j in range(len(out) - 1, 0, -1):
        Dl, n, Dr = out[j].shape
        Lf, Qm, qn = block_lq(out[j].reshape(Dl, n * Dr), qq[j], _col_charges(qq[j + 1], qs))
        out[j] = Qm.reshape(-1, n, Dr)
        qq[j] = qn
        out[j - 1] = np.tensordot(out[j - 1], Lf, axes=(2, 0))
    disc_max = 0.0
    for j in range(len(out) - 1):
        Dl, n, Dr = out[j].shape
        P, s, Q, disc, qn = block_svd_split(out[j].reshape(Dl * n, Dr),
                                            _row_charges(qq[j], qs), qq[j + 1], D_max, tol)
        disc_max = max(disc_max, disc / max(np.linalg.norm(s), 1e-300))
        out[j] = P.reshape(Dl, n, -1)
        qq[j + 1] = qn
        out[j + 1] = np.tensordot(s[:, None] * Q, out[j + 1], axes=(1, 0))
    return out, qq, disc_max


def charged_two_site_split(x, ql, qr, D_max, tol):
    """Alg. 1 step 2 on a charged two-site tensor x [Dl, n, n, Dr]: (left core, right core
    Sigma Q, discarded, charges of the new bond)."""
    qs = local_charges()
    Dl, n1, n2, Dr = x.shape
    P, s, Q, disc, qn = block_svd_split(x.reshape(Dl * n1, n2 * Dr), _row_charges(ql, qs),
                                        _col_charges(qr, qs), D_max, tol)
    return P.reshape(Dl, n1, -1), (s[:, None] * Q).reshape(-1, n2, Dr), disc, qn


def _masked_lowest(HL, W1, W2, HR, x0, mask, eig_tol, max_krylov):
    """Lowest eigenpair of the two-site projected operator restricted to the allowed
    block pattern (the operator conserves the charges; the projection removes rounding
    outside the pattern)."""
    mv = lambda v: heff_apply(HL, W1, W2, HR, v * mask) * mask
    th, x, nmv, _ = lanczos_lowest(mv, x0 * mask, tol=eig_tol, max_krylov=max_krylov)
    return th, x * mask, nmv


# ------------------------------------------------------------------ Alg. 1 / Alg. 2
def charged_half_sweep_lr(cores, q, mpo, D_max, svd_tol, eig_tol, max_krylov=40):
    """Alg. 1, left to right, on a right-orthogonal charged TT (cores 1..L-1)."""
    qs = local_charges()
    L = len(cores)
    U = [c.copy() for c in cores]
    qq = list(q)
    HR = right_envs(U, mpo, downto=2)
    HL = np.ones((1, 1, 1))
    energies, disc_max = [], 0.0
    for i in range(L - 1):
        x0 = np.tensordot(U[i], U[i + 1], axes=(2, 0))
        mask = two_site_mask(qq[i], qq[i + 2], qs)
        th, x, _ = _masked_lowest(HL, mpo[i], mpo[i + 1], HR[i + 2], x0, mask, eig_tol,
                                  max_krylov)
        U[i], U[i + 1], disc, qq[i + 1] = charged_two_site_split(x, qq[i], qq[i + 2],
                                                                 D_max, svd_tol)
        disc_max = max(disc_max, disc)
        HL = env_left_update(HL, U[i], mpo[i], U[i])
        energies.append(th)
    return U, qq, energies, disc_max


def charged_right_orthogonalize(cores, q):
    qs = local_charges()
    out = [c.copy() for c in cores]
    qq = list(q)
    for j in range(len(out) - 1, 0, -1):
        Dl, n, Dr = out[j].shape
        Lf, Qm, qn = block_lq(out[j].reshape(Dl, n * Dr), qq[j], _col_charges(qq[j + 1], qs))
        out[j] = Qm.reshape(-1, n, Dr)
        qq[j] = qn
        out[j - 1] = np.tensordot(out[j - 1], Lf, axes=(2, 0))
    return out, qq


def charged_dmrg(cores, q, mpo, D_max, svd_tol, eig_tol, n_sweeps, max_krylov=40):
    """Left-to-right half-sweeps of Alg. 1 (each from the right-orthogonalised iterate);
    returns (cores, charges, energies of every half-sweep's last micro-step)."""
    U, qq = cores, q
    hist = []
    for _ in range(n_sweeps):
        U, qq = charged_right_orthogonalize(U, qq)
        U, qq, e, _ = charged_half_sweep_lr(U, qq, mpo, D_max, svd_tol, eig_tol, max_krylov)
        hist.append(e[-1])
    return U, qq, hist


def charged_global_iteration(U, q, mpo, sizes, D_max, svd_tol=1e-10, eig_tol=1e-10,
                             coarse_eps=1e-10, max_krylov=40):
    """One A2DMRG global iteration (Alg. 2, two-site, groups of `sizes` bonds) on a
    charged left-orthogonal TT: the particle-preserving version of
    oracle.a2dmrg.global_iteration (block-wise LQ, masked local solves, block-wise
    truncated SVD, TT sum with concatenated charges, block-wise rounding)."""
    qs = local_charges()
    L = len(U)
    assert sum(sizes) == L - 1
    groups, k = [], 0
    for s_ in sizes:
        groups.append((k, k + s_ - 1))
        k += s_
    V, C, qV = charged_orthogonal_copies(U, q)
    HL = left_envs(U, mpo)
    HR = right_envs(V, mpo, downto=2)
    basis, qbasis, local_e = [list(U)], [list(q)], []
    for kg, mg in groups:
        Hl = HL[kg]
        centre = C[kg]
        qloc = list(q[:kg + 1]) + list(qV[kg + 1:])   # charges of (U.., C_kg, V..)
        new = {}
        th = None
        for kk in range(kg, mg + 1):
            x0 = np.tensordot(centre, V[kk + 1], axes=(2, 0))
            mask = two_site_mask(qloc[kk], qloc[kk + 2], qs)
            th, x, _ = _masked_lowest(Hl, mpo[kk], mpo[kk + 1], HR[kk + 2], x0, mask, eig_tol,
                                      max_krylov)
            new[kk], centre, _, qloc[kk + 1] = charged_two_site_split(x, qloc[kk], qloc[kk + 2],
                                                                     D_max, svd_tol)
            Hl = env_left_update(Hl, new[kk], mpo[kk], new[kk])
        new[mg + 1] = centre
        basis.append(list(U[:kg]) + [new[kk] for kk in range(kg, mg + 2)] + list(V[mg + 2:]))
        qbasis.append(qloc)
        local_e.append(th)
    m = len(basis)
    S = np.zeros((m, m))
    A = np.zeros((m, m))
    for i in range(m):
        for j in range(i, m):
            S[i, j] = S[j, i] = tt_inner(basis[i], basis[j])
            A[i, j] = A[j, i] = sandwich(basis[i], mpo, basis[j])
    c, lam, p = coarse_solve(A, S, coarse_eps)
    X = tt_add(basis, c)
    qX = [np.concatenate([qb[j] for qb in qbasis], axis=0) for j in range(L + 1)]
    qX[0] = q[0].copy()
    qX[L] = q[L].copy()
    Unew, qnew, disc_c = charged_round(X, qX, D_max, svd_tol)
    Unew = tt_scale(Unew, 1.0 / np.sqrt(tt_inner(Unew, Unew)))
    E = sandwich(Unew, mpo, Unew) / tt_inner(Unew, Unew)
    return Unew, qnew, dict(energy=E, lambda_coarse=lam, coarse_rank=p, local_energies=local_e,
                            compression_discarded=disc_c)


def charge_violation(cores, q):
    """Largest |entry| of any core outside its allowed pattern (0 for a charged TT)."""
    qs = local_charges()
    worst = 0.0
    for j, c in enumerate(cores):
        m = core_mask(q[j], q[j + 1], qs)
        if (~m).any():
            worst = max(worst, float(np.abs(c[~m]).max()))
    return worst
