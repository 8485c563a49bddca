"""Pins of the MPOs (synthetic) and the ED references (oracle.ed) against
closed forms and each other.  The ED Hamiltonians are built from explicit
Kronecker / Jordan-Wigner matrices and share no code with the MPO automaton."""
import numpy as np
import pytest

from oracle.ed import fermion_sparse, ground_energy, heisenberg_sparse, number_operator
from oracle.mpo import mpo_dense, mpo_compress
from synthetic import chemistry_integrals, chemistry_mpo, heisenberg_mpo, hubbard_integrals


def test_heisenberg_closed_forms():
    assert np.isclose(ground_energy(heisenberg_sparse(2)), -0.75, atol=1e-14)
    assert np.isclose(ground_energy(heisenberg_sparse(4)), -(3 + 2 * np.sqrt(3)) / 4,
                      atol=1e-13)


@pytest.mark.parametrize("L", [2, 5, 8])
def test_heisenberg_mpo_equals_ed(L):
    H = heisenberg_sparse(L).toarray()
    assert np.abs(mpo_dense(heisenberg_mpo(L)) - H).max() < 1e-14


@pytest.mark.parametrize("L,seed", [(2, 1), (3, 2), (4, 3)])
def test_chemistry_mpo_equals_fock_hamiltonian(L, seed):
    h, eri = chemistry_integrals(L, seed)
    H = fermion_sparse(h, eri).toarray()
    M = mpo_dense(chemistry_mpo(h, eri))
    assert np.abs(M - H).max() < 1e-13 * max(1.0, np.abs(H).max())
    assert np.abs(H - H.T).max() < 1e-13


def test_hubbard_two_site_closed_form():
    # two-site Hubbard, two electrons: E = U/2 - sqrt(U^2/4 + 4 t^2) in that sector
    h, eri = hubbard_integrals(2, 1.0, 4.0)
    H = fermion_sparse(h, eri).toarray()
    N = number_operator(2).toarray()
    idx = np.where(np.isclose(np.diag(N), 2.0))[0]
    e = np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0]
    assert np.isclose(e, 2.0 - np.sqrt(4.0 + 4.0), atol=1e-13)
    assert np.abs(mpo_dense(chemistry_mpo(h, eri)) - H).max() < 1e-14


def test_free_fermion_closed_form_in_fock_space():
    # one-body only: E0 = 2 * sum of negative orbital energies (whole Fock space)
    h, _ = chemistry_integrals(4, 11)
    eri = np.zeros((4,) * 4)
    e = np.linalg.eigvalsh(h)
    assert np.isclose(ground_energy(fermion_sparse(h, eri)), 2 * e[e < 0].sum(), atol=1e-12)


def test_mpo_compression_preserves_operator():
    h, eri = chemistry_integrals(3, 5)
    m = chemistry_mpo(h, eri)
    mc = mpo_compress(m, 1e-13)
    assert np.abs(mpo_dense(mc) - mpo_dense(m)).max() < 1e-12
