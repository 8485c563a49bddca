"""Pins of the particle-number preserving (U(1) x U(1)) oracle (oracle/blocksparse.py):
the block-wise truncated SVD equals the dense one of the same block-diagonal matrix, the
block-wise LQ reproduces its matrix with orthonormal rows, every charged TT lives in its
sector, the particle numbers stay exact in the truncating regime, and the charged DMRG
(Alg. 1) and A2DMRG (Alg. 2) reach the sector's exact ground energy: exact
diagonalisation restricted to the sector (Hubbard L = 6, U = 4, half filling) and the
U = 0 free-fermion closed form E = sum over spins and k <= N_s of -2t cos(k pi / (L+1))
(open chain); and, loosely, the half-filled chain's bulk energy against the Lieb-Wu
integral."""
import numpy as np
import pytest

from oracle.blocksparse import (block_lq, block_svd_split, charge_violation, charged_dmrg,
                                charged_global_iteration, charged_half_sweep_lr,
                                charged_right_orthogonalize, charged_round, particle_numbers,
                                random_charged_tt, reachable, sector_support)
from oracle.ed import fermion_sparse
from oracle.tt import svd_split, tt_full, tt_inner
from synthetic import chemistry_mpo, hubbard_integrals


def _block_diagonal(rng, rows, cols, charges):
    qr = np.array([charges[i] for i in rng.integers(0, len(charges), rows)])
    qc = np.array([charges[i] for i in rng.integers(0, len(charges), cols)])
    M = rng.standard_normal((rows, cols)) * np.all(qr[:, None, :] == qc[None, :, :], axis=2)
    return M, qr, qc


@pytest.mark.parametrize("D_max,tol", [(100, 1e-12), (7, 0.0), (100, 0.3)])
def test_block_svd_equals_dense_svd(D_max, tol):
    rng = np.random.default_rng(11)
    M, qr, qc = _block_diagonal(rng, 40, 30, [(0, 0), (1, 0), (0, 1), (1, 1), (2, 1)])
    P, s, Q, disc, qn = block_svd_split(M, qr, qc, D_max, tol)
    P0, s0, Q0, d0 = svd_split(M, D_max, tol)
    assert len(s) == len(s0)
    assert np.allclose(s, s0, rtol=1e-12, atol=1e-13)
    assert abs(disc - d0) < 1e-12
    assert np.abs(P.T @ P - np.eye(len(s))).max() < 1e-13
    assert np.abs((P * s) @ Q - (P0 * s0) @ Q0).max() < 1e-12
    # every kept direction lives on the rows and columns of one charge
    for k in range(len(s)):
        assert np.all(np.all(qr[np.abs(P[:, k]) > 0] == qn[k], axis=1))
        assert np.all(np.all(qc[np.abs(Q[k]) > 0] == qn[k], axis=1))


def test_block_lq():
    rng = np.random.default_rng(5)
    M, qr, qc = _block_diagonal(rng, 12, 40, [(0, 0), (1, 0), (1, 1)])
    L, Q, qn = block_lq(M, qr, qc)
    assert np.abs(L @ Q - M).max() < 1e-13
    assert np.abs(Q @ Q.T - np.eye(Q.shape[0])).max() < 1e-13
    for k in range(Q.shape[0]):
        assert np.all(np.all(qc[np.abs(Q[k]) > 0] == qn[k], axis=1))
        assert np.all(np.all(qr[np.abs(L[:, k]) > 0] == qn[k], axis=1))


def test_reachable_charges_and_sector_support():
    # bond after 2 of 4 orbitals in the sector (2, 1): n_up in 0..2, n_dn in 0..1
    got = {c for c, _, _ in reachable(4, 2, 2, 1)}
    assert got == {(nu, nd) for nu in range(3) for nd in range(2)}
    U, q = random_charged_tt(5, 2, 3, 12, 2)
    assert charge_violation(U, q) == 0.0
    assert sector_support(U, 2, 3) == 0.0
    nu, nd, var = particle_numbers(U)
    assert abs(nu - 2) < 1e-12 and abs(nd - 3) < 1e-12 and var < 1e-20


def test_charged_rounding_keeps_sector_and_is_exact_without_truncation():
    U, q = random_charged_tt(6, 2, 3, 10, 7)
    V, qv, disc = charged_round(U, q, 1000, 0.0)
    assert charge_violation(V, qv) == 0.0
    assert np.abs(tt_full(V) - tt_full(U)).max() < 1e-13
    W, qw, _ = charged_round(U, q, 3, 0.0)            # truncating
    assert charge_violation(W, qw) == 0.0 and sector_support(W, 2, 3) == 0.0


def _hubbard(L, U):
    h, eri = hubbard_integrals(L, 1.0, U)
    return h, eri, chemistry_mpo(h, eri)


def _sector_ground_energy(h, eri, L, Nu, Nd):
    H = fermion_sparse(h, eri)
    idx = np.arange(4 ** L)
    nu = np.zeros(4 ** L, dtype=np.int64)
    nd = np.zeros(4 ** L, dtype=np.int64)
    for j in range(L):
        s = (idx // 4 ** (L - 1 - j)) % 4
        nu += s & 1
        nd += s >> 1
    sel = np.nonzero((nu == Nu) & (nd == Nd))[0]
    return float(np.linalg.eigvalsh(H[sel][:, sel].toarray())[0])


def test_charged_dmrg_hubbard_ed_sector():
    L, Nu, Nd = 6, 3, 3
    h, eri, mpo = _hubbard(L, 4.0)
    E_ed = _sector_ground_energy(h, eri, L, Nu, Nd)
    U, q = random_charged_tt(L, Nu, Nd, 8, 3)
    U2, q2, hist = charged_dmrg(U, q, mpo, 400, 1e-13, 1e-12, 3)
    assert abs(hist[-1] - E_ed) < 1e-9
    assert charge_violation(U2, q2) == 0.0
    nu, nd, var = particle_numbers(U2)
    assert abs(nu - Nu) < 1e-12 and abs(nd - Nd) < 1e-12 and var < 1e-20


def test_free_fermion_closed_form():
    L, Nu, Nd = 8, 4, 3
    _, _, mpo = _hubbard(L, 0.0)
    E_exact = sum(-2.0 * np.cos(k * np.pi / (L + 1)) for N in (Nu, Nd) for k in range(1, N + 1))
    U, q = random_charged_tt(L, Nu, Nd, 8, 4)
    _, _, hist = charged_dmrg(U, q, mpo, 256, 1e-13, 1e-12, 4)
    assert abs(hist[-1] - E_exact) < 1e-8


def test_truncating_dmrg_preserves_particle_number():
    L, Nu, Nd = 6, 3, 2
    _, _, mpo = _hubbard(L, 4.0)
    U, q = random_charged_tt(L, Nu, Nd, 8, 9)
    U2, q2, _ = charged_dmrg(U, q, mpo, 5, 1e-12, 1e-10, 2)
    assert max(c.shape[2] for c in U2) <= 5
    assert charge_violation(U2, q2) == 0.0 and sector_support(U2, Nu, Nd) == 0.0
    nu, nd, var = particle_numbers(U2)
    assert abs(nu - Nu) < 1e-12 and abs(nd - Nd) < 1e-12 and var < 1e-20


def test_charged_a2dmrg_converges_in_sector():
    """Alg. 2 with the particle-preserving factorisations: every iterate stays in the
    sector (also while truncating), the energies do not increase, and the iteration
    reaches the sector's exact ground energy when the bond cap holds the ground state."""
    L, Nu, Nd = 6, 3, 3
    h, eri, mpo = _hubbard(L, 4.0)
    E_ed = _sector_ground_energy(h, eri, L, Nu, Nd)
    U, q = random_charged_tt(L, Nu, Nd, 8, 3)
    U, q = charged_right_orthogonalize(U, q)
    U, q, _, _ = charged_half_sweep_lr(U, q, mpo, 16, 1e-12, 1e-10)   # left-orthogonal start
    prev = np.inf
    for _ in range(6):
        U, q, rep = charged_global_iteration(U, q, mpo, [2, 2, 1], 400, 1e-13, 1e-12, 1e-10)
        assert charge_violation(U, q) == 0.0 and sector_support(U, Nu, Nd) == 0.0
        assert rep["energy"] <= prev + 1e-10
        prev = rep["energy"]
    assert abs(prev - E_ed) < 1e-8
    nu, nd, _ = particle_numbers(U)
    assert abs(nu - Nu) < 1e-12 and abs(nd - Nd) < 1e-12
    # truncating: the sector is kept exactly
    U, q = random_charged_tt(L, Nu, Nd, 8, 5)
    U, q = charged_right_orthogonalize(U, q)
    U, q, _, _ = charged_half_sweep_lr(U, q, mpo, 6, 1e-12, 1e-10)
    U, q, rep = charged_global_iteration(U, q, mpo, [2, 2, 1], 6, 1e-12, 1e-10, 1e-10)
    assert max(c.shape[2] for c in U) <= 6
    assert charge_violation(U, q) == 0.0 and sector_support(U, Nu, Nd) == 0.0
    assert abs(tt_inner(U, U) - 1.0) < 1e-12


def test_half_filled_hubbard_bulk_energy_lieb_wu():
    """Loose bulk check: the energy per site of the half-filled chain at U = 4 from two open
    chains, (E(12) - E(8)) / 4 (the boundary terms cancel), against the Lieb-Wu integral
    e = -4 int_0^inf J0(w) J1(w) / (w (1 + exp(w U / 2))) dw (t = 1), within 1 %."""
    from scipy import integrate, special
    Uint = 4.0

    def f(w):
        return special.j0(w) * special.j1(w) / (w * (1.0 + np.exp(min(w * Uint / 2.0, 700.0))))

    e_bulk = -4.0 * integrate.quad(f, 0.0, np.inf, limit=400)[0]
    E = {}
    for L in (8, 12):
        _, _, mpo = _hubbard(L, Uint)
        U, q = random_charged_tt(L, L // 2, L // 2, 16, 1)
        _, _, hist = charged_dmrg(U, q, mpo, 64, 1e-10, 1e-9, 8)
        assert abs(hist[-1] - hist[-2]) < 1e-8        # converged
        E[L] = hist[-1]
    e_fin = (E[12] - E[8]) / 4.0
    assert abs(e_fin - e_bulk) < 0.01 * abs(e_bulk), (e_fin, e_bulk)
