"""Two-site A2DMRG global iteration (Alg. 2) with P groups of bonds, FP64.

Reading of 'P subdomains' (Extension Two of the paper's extension remark):
the bonds 0..L-2 are split into P contiguous groups; inside a group the
two-site micro-steps run left to right as in Alg. 1 (each starting from the
k_g-orthogonal copy of the iterate), the groups are independent.  P = L-1 is
exactly Alg. 2; P = 1 is one classical left-to-right half-sweep.

Steps (Alg. 2):
 1. right-to-left LQ sweep W_i = L_i Q_i, V_i = Q_i, W_{i-1} = U_{i-1} L_i, giving
    every i-orthogonal copy (U_0..U_{i-1}, C_i, V_{i+1}..V_{L-1});
 2. per group: Lanczos on H_eff, truncated SVD, group-local left environment;
    the updated TT of group g differs from the iterate on its cores only;
 3. coarse problem over span{tau(U~^0), ..., tau(U~^P)} with U~^0 the iterate,
    S_hat and A_hat by their definitions (eq. A_reduced), solved by
    oracle.coarse.coarse_solve;
 4. compression of sum_j c_j tau(U~^j) by TT rounding to ranks <= D_max
    (TT-rounding named in the text after Alg. 2), normalised, left-orthogonal.
The energy of the new iterate is its Rayleigh quotient (eq. energy_eig).
"""
import numpy as np

from .coarse import coarse_solve
from .env import env_left_update, heff1_apply, heff_apply, left_envs, right_envs, sandwich
from .lanczos import lanczos_lowest
from .tt import lq_pos, qr_pos, svd_split, tt_add, tt_inner, tt_round, tt_scale


def lowest_eigvecs(matvec, x0, K):
    """The K lowest eigenpairs of the symmetric local operator `matvec` (Extension One
    of the extension remark after Alg. 2: keep the K lowest eigenvectors of the local
    problem instead of one).  Plain definition: the dense matrix of the operator (column
    i = the operator applied to the i-th unit tensor) and its full eigendecomposition,
    ascending.  Sign: <x_k, x0> >= 0, as for the Lanczos solution.  K is capped at the
    local dimension."""
    shape = x0.shape
    N = x0.size
    K = min(K, N)
    H = np.empty((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        H[:, i] = matvec(e.reshape(shape)).ravel()
    w, X = np.linalg.eigh(0.5 * (H + H.T))
    xs = []
    for k in range(K):
        x = X[:, k]
        if x @ x0.ravel() < 0:
            x = -x
        xs.append(x.reshape(shape))
    return list(w[:K]), xs


def bond_groups(L, sizes):
    assert sum(sizes) == L - 1, (sizes, L)
    out, k = [], 0
    for s in sizes:
        out.append((k, k + s - 1))
        k += s
    return out


def orthogonal_copies(U):
    """Step 1: LQ sweep.  Returns (V, C): right-orthogonal cores V[i] (i >= 1)
    and centres C[i] so that (U_0..U_{i-1}, C_i, V_{i+1}..) is i-orthogonal."""
    L = len(U)
    V = [None] * L
    C = [None] * L
    C[L - 1] = U[L - 1].copy()
    for i in range(L - 1, 0, -1):
        Dl, n, Dr = C[i].shape
        Lf, Q = lq_pos(C[i].reshape(Dl, n * Dr))
        V[i] = Q.reshape(Q.shape[0], n, Dr)
        C[i - 1] = np.tensordot(U[i - 1], Lf, axes=(2, 0))
    return V, C


def energy(U, mpo):
    return sandwich(U, mpo, U) / tt_inner(U, U)


def global_iteration(U, mpo, sizes, D_max, svd_tol=1e-10, eig_tol=1e-10,
                     coarse_eps=1e-10, max_krylov=40, n_eig=1):
    """n_eig = K > 1: Extension One.  The last micro-step of every group keeps its K
    lowest eigenvectors; each gives one updated TT (its own truncated SVD), so the coarse
    space has K*P + 1 vectors, ordered [iterate, group 0 (lowest first), group 1, ...];
    local_energies then lists the K eigenvalues of every group in the same order."""
    L = len(U)
    groups = bond_groups(L, sizes)
    V, C = orthogonal_copies(U)
    HL = left_envs(U, mpo)
    HR = right_envs(V, mpo, downto=2)
    updated, local_e, kry, disc_max = [], [], [0] * (L - 1), 0.0
    for kg, mg in groups:
        Hl = HL[kg]
        centre = C[kg]
        new = {}
        th = None
        extra = []
        for k in range(kg, mg + 1):
            x0 = np.tensordot(centre, V[k + 1], axes=(2, 0))
            mv = lambda v, Hl=Hl, k=k: heff_apply(Hl, mpo[k], mpo[k + 1], HR[k + 2], v)
            if n_eig > 1 and k == mg:
                ths, xs = lowest_eigvecs(mv, x0, n_eig)
                th, x, nmv = ths[0], xs[0], x0.size
                for th_e, x_e in zip(ths[1:], xs[1:]):
                    Dl, n1, n2, Dr = x_e.shape
                    P, s, Q, disc = svd_split(x_e.reshape(Dl * n1, n2 * Dr), D_max, svd_tol)
                    disc_max = max(disc_max, disc)
                    extra.append((th_e, [P.reshape(Dl, n1, -1),
                                         (s[:, None] * Q).reshape(-1, n2, Dr)]))
            else:
                th, x, nmv, _ = lanczos_lowest(mv, x0, tol=eig_tol, max_krylov=max_krylov)
            kry[k] = nmv
            Dl, n1, n2, Dr = x.shape
            P, s, Q, disc = svd_split(x.reshape(Dl * n1, n2 * Dr), D_max, svd_tol)
            disc_max = max(disc_max, disc)
            new[k] = P.reshape(Dl, n1, -1)
            Hl = env_left_update(Hl, new[k], mpo[k], new[k])
            centre = (s[:, None] * Q).reshape(-1, n2, Dr)
        new[mg + 1] = centre
        Ug = list(U[:kg]) + [new[k] for k in range(kg, mg + 2)] + list(V[mg + 2:])
        updated.append(Ug)
        local_e.append(th)
        for th_e, tail in extra:
            updated.append(list(U[:kg]) + [new[k] for k in range(kg, mg)] + tail
                           + list(V[mg + 2:]))
            local_e.append(th_e)
    basis = [list(U)] + updated
    m = len(basis)
    S = np.zeros((m, m))
    A = np.zeros((m, m))
    for i in range(m):
        for j in range(i, m):
            S[i, j] = S[j, i] = tt_inner(basis[i], basis[j])
            A[i, j] = A[j, i] = sandwich(basis[i], mpo, basis[j])
    c, lam, p = coarse_solve(A, S, coarse_eps)
    X = tt_add(basis, c)
    Unew, disc_c = tt_round(X, D_max, svd_tol)
    Unew = tt_scale(Unew, 1.0 / np.sqrt(tt_inner(Unew, Unew)))
    E_new = energy(Unew, mpo)
    report = dict(energy=E_new, lambda_coarse=lam, coeffs=c, coarse_rank=p,
                  S_hat=S, A_hat=A, local_energies=local_e, krylov=kry,
                  max_discarded=disc_max, compression_discarded=disc_c,
                  local_rayleigh=[A[g, g] / S[g, g] for g in range(1, m)],
                  basis=basis)
    return Unew, report


def core_groups(L, sizes):
    assert sum(sizes) == L, (sizes, L)
    out, k = [], 0
    for s in sizes:
        out.append((k, k + s - 1))
        k += s
    return out


def global_iteration_onesite(U, mpo, sizes, D_max, svd_tol=1e-10, eig_tol=1e-10,
                             coarse_eps=1e-10, max_krylov=40, n_eig=1):
    """One-site A2DMRG global iteration (Alg. 2, one-site case) with P groups of cores.

    The cores 0..L-1 are split into P contiguous groups; inside a group the one-site
    micro-steps run left to right as in Alg. 1 (one-site): the j-th step takes the
    lowest eigenvector of the one-site H_eff of the current j-orthogonal TT, and unless
    it is the group's last core it is orthogonalised (QR, diag R >= 0) and R is moved
    into the next core (Alg. 1, step 2, one-site).  Ranks do not change.  P = L is
    exactly Alg. 2 in the one-site case (coarse dimension L + 1), P = 1 a classical
    one-site half-sweep.  Coarse problem and compression as in the two-site case.
    n_eig = K > 1: Extension One, the K lowest eigenvectors of every group's last core
    each replace that core (coarse dimension K*P + 1, ordered as in global_iteration).
    """
    L = len(U)
    groups = core_groups(L, sizes)
    V, C = orthogonal_copies(U)
    HL = left_envs(U, mpo)
    HR = right_envs(V, mpo, downto=1)
    updated, local_e, kry = [], [], [0] * L
    for kg, mg in groups:
        Hl = HL[kg]
        centre = C[kg]
        new = {}
        th = None
        extra = []
        for j in range(kg, mg + 1):
            mv = lambda v, Hl=Hl, j=j: heff1_apply(Hl, mpo[j], HR[j + 1], v)
            if n_eig > 1 and j == mg:
                ths, xs = lowest_eigvecs(mv, centre, n_eig)
                th, x, nmv = ths[0], xs[0], centre.size
                extra = list(zip(ths[1:], xs[1:]))
            else:
                th, x, nmv, _ = lanczos_lowest(mv, centre, tol=eig_tol, max_krylov=max_krylov)
            kry[j] = nmv
            if j < mg:
                Dl, n, Dr = x.shape
                Q, R = qr_pos(x.reshape(Dl * n, Dr))
                new[j] = Q.reshape(Dl, n, -1)
                Hl = env_left_update(Hl, new[j], mpo[j], new[j])
                centre = np.tensordot(R, V[j + 1], axes=(1, 0))
            else:
                new[j] = x
        Ug = list(U[:kg]) + [new[j] for j in range(kg, mg + 1)] + list(V[mg + 1:])
        updated.append(Ug)
        local_e.append(th)
        for th_e, x_e in extra:
            updated.append(list(U[:kg]) + [new[j] for j in range(kg, mg)] + [x_e]
                           + list(V[mg + 1:]))
            local_e.append(th_e)
    basis = [list(U)] + updated
    m = len(basis)
    S = np.zeros((m, m))
    A = np.zeros((m, m))
    for i in range(m):
        for j in range(i, m):
            S[i, j] = S[j, i] = tt_inner(basis[i], basis[j])
            A[i, j] = A[j, i] = sandwich(basis[i], mpo, basis[j])
    c, lam, p = coarse_solve(A, S, coarse_eps)
    X = tt_add(basis, c)
    Unew, disc_c = tt_round(X, D_max, svd_tol)
    Unew = tt_scale(Unew, 1.0 / np.sqrt(tt_inner(Unew, Unew)))
    E_new = energy(Unew, mpo)
    report = dict(energy=E_new, lambda_coarse=lam, coeffs=c, coarse_rank=p,
                  S_hat=S, A_hat=A, local_energies=local_e, krylov=kry,
                  compression_discarded=disc_c,
                  local_rayleigh=[A[g, g] / S[g, g] for g in range(1, m)],
                  basis=basis)
    return Unew, report


def run(U0, mpo, sizes, D_max, n_iter, tol_rel=1e-6, **kw):
    U = U0
    E_prev = energy(U, mpo)
    hist = []
    for it in range(n_iter):
        U, rep = global_iteration(U, mpo, sizes, D_max, **kw)
        rep["energy_prev"] = E_prev
        hist.append(rep)
        if abs(rep["energy"] - E_prev) < tol_rel * abs(rep["energy"]):
            break
        E_prev = rep["energy"]
    return U, hist
