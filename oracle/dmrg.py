"""Classical two-site DMRG (Alg. 1) in plain FP64 (oracle; test only).

Input: a right-orthogonal TT (Alg. 1 'Require').  One call of `half_sweep_lr`
performs micro-steps i = 0..L-2 left to right: the two-site micro-iteration
(lowest eigenpair of the projected operator, Lemma DMRG micro-iterations),
then the truncated SVD step W = P Sigma Q with U_i = P and Sigma Q carried to
site i+1 (Alg. 1 step 2).  `half_sweep_rl` repeats the steps right to left.
Energies after every micro-step are returned (monotonicity pin).
"""
import numpy as np

from .env import env_left_update, env_right_update, heff_apply, right_envs, left_envs
from .lanczos import lanczos_lowest
from .tt import svd_split


def two_site_solve(HL, W1, W2, HR, x0, eig_tol, max_krylov):
    mv = lambda v: heff_apply(HL, W1, W2, HR, v)
    return lanczos_lowest(mv, x0, tol=eig_tol, max_krylov=max_krylov)


def half_sweep_lr(cores, mpo, D_max, svd_tol, eig_tol, max_krylov=40, HR=None):
    """cores: right-orthogonal (cores 1..L-1).  Returns left-orthogonal cores
    (0..L-2) with the centre at L-1, energies per micro-step, stats."""
    L = len(cores)
    U = [c.copy() for c in cores]
    HR = right_envs(U, mpo, downto=2) if HR is None else HR
    HL = np.ones((1, 1, 1))
    energies, kry, disc_max = [], [], 0.0
    for i in range(L - 1):
        x0 = np.tensordot(U[i], U[i + 1], axes=(2, 0))
        th, x, nmv, _ = two_site_solve(HL, mpo[i], mpo[i + 1], HR[i + 2], x0,
                                        eig_tol, max_krylov)
        Dl, n1, n2, Dr = x.shape
        P, s, Q, disc = svd_split(x.reshape(Dl * n1, n2 * Dr), D_max, svd_tol)
        disc_max = max(disc_max, disc)
        U[i] = P.reshape(Dl, n1, -1)
        U[i + 1] = (s[:, None] * Q).reshape(-1, n2, Dr)
        HL = env_left_update(HL, U[i], mpo[i], U[i])
        energies.append(th)
        kry.append(nmv)
    return U, energies, dict(krylov=kry, max_discarded=disc_max)


def half_sweep_rl(cores, mpo, D_max, svd_tol, eig_tol, max_krylov=40):
    """cores: left-orthogonal (0..L-2).  Returns right-orthogonal cores."""
    L = len(cores)
    U = [c.copy() for c in cores]
    HLs = left_envs(U, mpo, upto=L - 2)
    HR = np.ones((1, 1, 1))
    energies, kry, disc_max = [], [], 0.0
    for i in range(L - 2, -1, -1):
        x0 = np.tensordot(U[i], U[i + 1], axes=(2, 0))
        th, x, nmv, _ = two_site_solve(HLs[i], mpo[i], mpo[i + 1], HR, x0,
                                        eig_tol, max_krylov)
        Dl, n1, n2, Dr = x.shape
        P, s, Q, disc = svd_split(x.reshape(Dl * n1, n2 * Dr), D_max, svd_tol)
        disc_max = max(disc_max, disc)
        U[i + 1] = Q.reshape(-1, n2, Dr)
        U[i] = (P * s).reshape(Dl, n1, -1)
        HR = env_right_update(HR, U[i + 1], mpo[i + 1], U[i + 1])
        energies.append(th)
        kry.append(nmv)
    return U, energies, dict(krylov=kry, max_discarded=disc_max)


def classical_dmrg(cores_right_orth, mpo, D_max, svd_tol, eig_tol, n_half_sweeps,
                   max_krylov=40):
    U = cores_right_orth
    hist = []
    for h in range(n_half_sweeps):
        if h % 2 == 0:
            U, e, st = half_sweep_lr(U, mpo, D_max, svd_tol, eig_tol, max_krylov)
        else:
            U, e, st = half_sweep_rl(U, mpo, D_max, svd_tol, eig_tol, max_krylov)
        hist.append(dict(energies=e, **st))
    return U, hist
