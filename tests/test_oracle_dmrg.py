"""Pins of the oracle's local problem, classical DMRG and A2DMRG against ED,
brute-force projections, closed forms and the variational invariants."""
import numpy as np
import pytest
import scipy.linalg

from oracle import a2dmrg
from oracle.coarse import coarse_solve
from oracle.dmrg import classical_dmrg
from oracle.ed import fermion_sparse, ground_energy, heisenberg_sparse
from oracle.env import heff_apply, heff_dense, left_envs, right_envs
from oracle.lanczos import lanczos_lowest
from oracle.mpo import mpo_dense
from oracle.tt import left_orthogonalize, right_orthogonalize, tt_full, tt_inner
from synthetic import chemistry_integrals, chemistry_mpo, heisenberg_mpo, random_tt_cores


def _normalised_left(cores):
    U = left_orthogonalize(cores)
    U[-1] = U[-1] / np.sqrt(tt_inner(U, U))
    return U


@pytest.mark.parametrize("k", [0, 2, 4])
def test_heff_equals_projected_operator(k):
    """H_eff from environments equals P* A P with P the two-site retraction
    (Def. retraction) of a k-orthogonal decomposition (Lemma micro-iterations)."""
    L = 6
    mpo = heisenberg_mpo(L)
    Lk = left_orthogonalize(random_tt_cores([2] * L, 4, 3))
    Y = Lk[:k] + right_orthogonalize(Lk[k:])          # k-orthogonal decomposition
    Dl, n, Dr = Y[k].shape[0], 2, Y[k + 1].shape[2]
    cols = []
    for idx in range(Dl * n * n * Dr):
        E = np.zeros(Dl * n * n * Dr)
        E[idx] = 1.0
        Q, Rm = np.linalg.qr(E.reshape(Dl * n, n * Dr))
        c = Y[:k] + [Q.reshape(Dl, n, -1), Rm.reshape(-1, n, Dr)] + Y[k + 2:]
        cols.append(tt_full(c))
    P = np.array(cols).T
    assert np.allclose(P.T @ P, np.eye(P.shape[1]), atol=1e-12)    # Lemma (retraction)
    HL = left_envs(Y, mpo)[k]
    HR = right_envs(Y, mpo, downto=k + 2)[k + 2]
    Heff = heff_dense(HL, mpo[k], mpo[k + 1], HR)
    assert np.allclose(Heff, P.T @ mpo_dense(mpo) @ P, atol=1e-12)
    assert np.abs(Heff - Heff.T).max() < 1e-13 * np.abs(Heff).max()


def test_lanczos_matches_eigh():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((300, 300))
    A = A + A.T
    ev = np.linalg.eigvalsh(A)[0]
    th, x, nmv, cyc = lanczos_lowest(lambda v: A @ v, rng.standard_normal(300), tol=1e-12)
    assert abs(th - ev) < 1e-9 * abs(ev)
    assert np.linalg.norm(A @ x - th * x) < 1e-8 * np.abs(ev)


def test_classical_dmrg_heisenberg_ed_and_monotone():
    L = 10
    mpo = heisenberg_mpo(L)
    E_ed = ground_energy(heisenberg_sparse(L))
    R = right_orthogonalize(random_tt_cores([2] * L, 4, 7))
    U, hist = classical_dmrg(R, mpo, 32, 1e-14, 1e-12, 4)
    e = np.concatenate([h["energies"] for h in hist])
    assert abs(e[-1] - E_ed) < 1e-10 * abs(E_ed)
    assert np.all(np.diff(e) <= 1e-10)                   # no truncation: monotone
    assert np.all(e >= E_ed - 1e-10)


def test_classical_dmrg_chemistry_ed():
    h, eri = chemistry_integrals(5, 21)
    mpo = chemistry_mpo(h, eri)
    E_ed = ground_energy(fermion_sparse(h, eri))
    R = right_orthogonalize(random_tt_cores([4] * 5, 4, 1))
    U, hist = classical_dmrg(R, mpo, 64, 1e-14, 1e-12, 4)
    assert abs(hist[-1]["energies"][-1] - E_ed) < 1e-10 * abs(E_ed)


def test_free_fermion_dmrg_closed_form():
    h, _ = chemistry_integrals(4, 11)
    eri = np.zeros((4,) * 4)
    e = np.linalg.eigvalsh(h)
    mpo = chemistry_mpo(h, eri)
    U0 = _normalised_left(random_tt_cores([4] * 4, 4, 2))
    U, hist = a2dmrg.run(U0, mpo, [1, 1, 1], 16, 20, tol_rel=1e-14)
    assert abs(hist[-1]["energy"] - 2 * e[e < 0].sum()) < 1e-10


@pytest.fixture(scope="module")
def heis12():
    L = 12
    return L, heisenberg_mpo(L), ground_energy(heisenberg_sparse(L))


def test_a2dmrg_c1_exact_rank_reaches_ed(heis12):
    L, mpo, E_ed = heis12
    U0 = _normalised_left(random_tt_cores([2] * L, 4, 23429))
    U, hist = a2dmrg.run(U0, mpo, [6, 5], 64, 20, tol_rel=1e-14)
    assert abs(hist[-1]["energy"] - E_ed) < 1e-10 * abs(E_ed)


def test_a2dmrg_c1_truncated_variational(heis12):
    L, mpo, E_ed = heis12
    U0 = _normalised_left(random_tt_cores([2] * L, 4, 23429))
    U, hist = a2dmrg.run(U0, mpo, [6, 5], 32, 20, tol_rel=1e-12)
    E = hist[-1]["energy"]
    assert E >= E_ed - 1e-12 and E - E_ed < 1e-6
    for rep in hist:
        lam = rep["lambda_coarse"]
        # the coarse minimiser beats every element of the span (eq. d_opt_lin_3)
        assert lam <= rep["energy_prev"] + 1e-10
        assert all(lam <= e + 1e-10 for e in rep["local_rayleigh"])
        assert lam >= E_ed - 1e-10


def test_a2dmrg_single_iteration_once_full_rank(heis12):
    """Fig. 7 behaviour: with no truncation and ranks at the separation ranks
    the iteration reaches the minimiser in one global iteration."""
    L, mpo, E_ed = heis12
    U0 = _normalised_left(random_tt_cores([2] * L, 64, 5))   # full exact ranks
    U, rep = a2dmrg.global_iteration(U0, mpo, [1] * (L - 1), 64)
    assert abs(rep["energy"] - E_ed) < 1e-10 * abs(E_ed)


def test_coarse_matrices_brute_force(heis12):
    L, mpo, E_ed = heis12
    U0 = _normalised_left(random_tt_cores([2] * L, 4, 23429))
    U1, rep = a2dmrg.global_iteration(U0, mpo, [6, 5], 32)
    Y = np.array([tt_full(b) for b in rep["basis"]]).T
    H = heisenberg_sparse(L)
    assert np.allclose(rep["S_hat"], Y.T @ Y, atol=1e-12)
    assert np.allclose(rep["A_hat"], Y.T @ (H @ Y), atol=1e-12)
    # the compressed iterate approximates sum_j c_j tau(U~^j) within the truncation
    x = Y @ rep["coeffs"]
    xu = tt_full(U1)
    assert abs(abs(x @ xu) / np.linalg.norm(x) - 1.0) < 1e-8


def test_p1_reduces_to_a_classical_half_sweep(heis12):
    L, mpo, E_ed = heis12
    U0 = _normalised_left(random_tt_cores([2] * L, 4, 8))
    U1, rep = a2dmrg.global_iteration(U0, mpo, [L - 1], 32)
    R = right_orthogonalize(U0)
    _, hist = classical_dmrg(R, mpo, 32, 1e-10, 1e-10, 1)
    assert rep["lambda_coarse"] <= hist[0]["energies"][-1] + 1e-9


def test_coarse_solve_generalized_eigh():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((6, 6))
    S = B @ B.T + 6 * np.eye(6)
    A = rng.standard_normal((6, 6))
    A = A + A.T
    c, lam, p = coarse_solve(A, S, 1e-10)
    w = scipy.linalg.eigh(A, S, eigvals_only=True)
    assert p == 6 and abs(lam - w[0]) < 1e-12 * max(1, abs(w[0]))
    assert abs(c @ S @ c - 1.0) < 1e-12 and c[0] >= 0


def test_coarse_solve_rank_deficient():
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((50, 4))
    Y = np.concatenate([Y, Y[:, :1]], axis=1)              # duplicated vector
    H = rng.standard_normal((50, 50))
    H = H + H.T
    c, lam, p = coarse_solve(Y.T @ H @ Y, Y.T @ Y, 1e-10)
    Q, _ = np.linalg.qr(Y[:, :4])
    assert p == 4
    assert abs(lam - np.linalg.eigvalsh(Q.T @ H @ Q)[0]) < 1e-10
