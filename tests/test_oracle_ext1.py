"""Pins of the oracle's Extension One (the K lowest eigenvectors of each group's last
local problem enrich the coarse space, extension remark after Alg. 2), two-site and
one-site: with every eigenvector kept (K = local dimension, no truncation) the coarse
eigenvalue is the Rayleigh-Ritz value of the Hamiltonian on the sum of the local
subspaces, computed here by brute force from full tensors; the local eigenvalues
interlace with the exact spectrum; enlarging K never raises the coarse eigenvalue; the
K = 1 part of the enriched basis is the plain iteration's basis."""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse.linalg

from oracle import a2dmrg
from oracle.ed import fermion_sparse, heisenberg_sparse
from oracle.mpo import mpo_dense
from oracle.tt import left_orthogonalize, right_orthogonalize, tt_full, tt_inner
from synthetic import chemistry_integrals, chemistry_mpo, heisenberg_mpo, random_tt_cores


def _normalised_left(cores):
    U = left_orthogonalize(cores)
    U[-1] = U[-1] / np.sqrt(tt_inner(U, U))
    return U


def _sites_basis(U, j, width):
    """Columns: full tensors of the j-orthogonal form of U with sites j..j+width-1
    replaced by every unit tensor (orthonormal columns: the local subspace)."""
    Y = U[:j] + right_orthogonalize(U[j:])
    Dl, Dr = Y[j].shape[0], Y[j + width - 1].shape[2]
    ns = [Y[j + q].shape[1] for q in range(width)]
    N = Dl * int(np.prod(ns)) * Dr
    cols = []
    for idx in range(N):
        e = np.zeros(N)
        e[idx] = 1.0
        if width == 1:
            blk = [e.reshape(Dl, ns[0], Dr)]
        else:   # the two-site tensor as (identity core) x (reshaped tensor)
            blk = [np.eye(Dl * ns[0]).reshape(Dl, ns[0], Dl * ns[0]),
                   e.reshape(Dl * ns[0], ns[1], Dr)]
        cols.append(tt_full(Y[:j] + blk + Y[j + width:]))
    return np.array(cols).T


def _ritz_on_span(H, vecs, rel=1e-8):
    B = np.concatenate(vecs, axis=1)
    Uu, s, _ = np.linalg.svd(B, full_matrices=False)
    Q = Uu[:, s > rel * s[0]]
    return np.linalg.eigvalsh(Q.T @ H @ Q)[0]


def test_two_site_all_eigenvectors_equals_brute_force_span():
    L = 7
    mpo = heisenberg_mpo(L)
    H = mpo_dense(mpo)
    U = _normalised_left(random_tt_cores([2] * L, 2, 41))
    sizes = [1] * (L - 1)
    K = max(U[k].shape[0] * 4 * U[k + 1].shape[2] for k in range(L - 1))
    # every group keeps all its eigenvectors (K is capped at each local dimension)
    _, rep = a2dmrg.global_iteration(U, mpo, sizes, D_max=64, svd_tol=0.0, n_eig=K)
    vecs = [tt_full(U)[:, None]] + [_sites_basis(U, k, 2) for k in range(L - 1)]
    lam = _ritz_on_span(H, vecs)
    assert abs(rep["lambda_coarse"] - lam) < 1e-9 * abs(lam)


def test_one_site_all_eigenvectors_equals_brute_force_span():
    L = 7
    mpo = heisenberg_mpo(L)
    H = mpo_dense(mpo)
    U = _normalised_left(random_tt_cores([2] * L, 2, 43))
    K = max(U[j].shape[0] * 2 * U[j].shape[2] for j in range(L))
    _, rep = a2dmrg.global_iteration_onesite(U, mpo, [1] * L, D_max=64, svd_tol=0.0, n_eig=K)
    vecs = [tt_full(U)[:, None]] + [_sites_basis(U, j, 1) for j in range(L)]
    lam = _ritz_on_span(H, vecs)
    assert abs(rep["lambda_coarse"] - lam) < 1e-9 * abs(lam)


@pytest.mark.parametrize("one_site", [False, True])
def test_interlacing_and_monotone_in_K(one_site):
    """theta_k of a local problem >= the k-th exact eigenvalue (Cauchy interlacing for
    P* A P); lambda_coarse(K=3) <= lambda_coarse(K=1); the basis of K = 1 is the
    lowest-eigenvector part of the K = 3 basis."""
    L = 6
    h, eri = chemistry_integrals(L, 2505)
    mpo = chemistry_mpo(h, eri)
    U = _normalised_left(random_tt_cores([4] * L, 4, 12))
    K = 3
    sizes = [2, 2, 2] if one_site else [2, 2, 1]
    it = a2dmrg.global_iteration_onesite if one_site else a2dmrg.global_iteration
    _, r1 = it(U, mpo, sizes, D_max=4)
    _, rK = it(U, mpo, sizes, D_max=4, n_eig=K)
    ex = np.sort(scipy.sparse.linalg.eigsh(fermion_sparse(h, eri), k=K, which="SA")[0])
    P = len(sizes)
    th = np.array(rK["local_energies"]).reshape(P, K)
    for g in range(P):
        assert np.all(np.diff(th[g]) >= -1e-12)
        assert np.all(th[g] >= ex - 1e-9)
        assert abs(th[g, 0] - r1["local_energies"][g]) < 1e-9 * abs(th[g, 0])
    assert rK["lambda_coarse"] <= r1["lambda_coarse"] + 1e-9
    sel = [0] + [1 + g * K for g in range(P)]
    assert np.allclose(rK["S_hat"][np.ix_(sel, sel)], r1["S_hat"], atol=1e-8)
    assert np.allclose(rK["A_hat"][np.ix_(sel, sel)], r1["A_hat"], atol=1e-8)
    # one-site: the eigenvectors of one local problem stay orthonormal in the full space
    # (no truncation; two-site eigenvectors are truncated separately)
    S = rK["S_hat"]
    for g in range(P if one_site else 0):
        blk = S[1 + g * K:1 + (g + 1) * K, 1 + g * K:1 + (g + 1) * K]
        assert np.allclose(blk, np.eye(K), atol=1e-9)


def test_heisenberg_interlacing_against_dense_spectrum():
    L = 6
    mpo = heisenberg_mpo(L)
    U = _normalised_left(random_tt_cores([2] * L, 3, 5))
    K = 4
    _, rep = a2dmrg.global_iteration(U, mpo, [5], D_max=3, n_eig=K)
    ex = scipy.linalg.eigvalsh(heisenberg_sparse(L).toarray())[:K]
    assert np.all(np.array(rep["local_energies"]) >= ex - 1e-9)
