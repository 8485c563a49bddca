"""CPU: pins of the gradient configuration's references.
* the builder's coefficient map is exactly the linear part of the MPO cores;
* oracle.rdm's gradient satisfies <psi|H|psi> = sum h dE/dh + sum eri dE/deri for the
  independent Fock-space Hamiltonian of oracle.ed (so both RDMs carry the right
  operator order, spin sum and factor 1/2);
* the one-term-operator sandwich used for sampled checks at full size equals the RDM
  entries."""
import numpy as np
import pytest

from oracle.ed import fermion_sparse
from oracle.env import sandwich
from oracle.rdm import hamiltonian_gradient
from oracle.tt import left_orthogonalize, tt_full
from synthetic import chemistry_integrals, chemistry_mpo, random_tt_cores


@pytest.mark.parametrize("L", [4, 5])
def test_coeff_map_is_the_linear_part(L):
    h, eri = chemistry_integrals(L, 2505)
    W1, cm = chemistry_mpo(h, eri, coeff_map=True)
    W2 = chemistry_mpo(2.0 * h, 2.0 * eri)
    theta = np.concatenate([h.ravel(), eri.ravel()])
    assert cm["nparam"] == theta.size
    for j in range(L):
        sel = cm["site"] == j
        lin = np.zeros(W1[j].size)
        np.add.at(lin, cm["index"][sel], theta[cm["param"][sel]] * cm["factor"][sel])
        assert W2[j].shape == W1[j].shape
        d = (W2[j] - W1[j]).ravel()
        assert np.allclose(lin, d, rtol=1e-13, atol=1e-13)


def test_rdm_gradient_reproduces_the_energy():
    L = 4
    h, eri = chemistry_integrals(L, 7)
    H = fermion_sparse(h, eri)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(4 ** L)
    psi /= np.linalg.norm(psi)
    gh, geri = hamiltonian_gradient(psi, L)
    E = float(psi @ (H @ psi))
    assert abs(np.sum(h * gh) + np.sum(eri * geri) - E) < 1e-12 * max(1.0, abs(E))
    assert np.allclose(gh, gh.T, atol=1e-14)
    # two-particle symmetry of the spin-summed RDM: (ij|kl) <-> (kl|ij)
    assert np.allclose(geri, geri.transpose(2, 3, 0, 1), atol=1e-14)


def test_one_term_sandwich_equals_rdm():
    L = 4
    cores = left_orthogonalize(random_tt_cores([4] * L, 16, 11))
    psi = tt_full(cores).ravel()
    nrm2 = float(psi @ psi)
    gh, geri = hamiltonian_gradient(psi, L)
    for (i, j) in [(0, 0), (1, 3), (3, 2)]:
        h1 = np.zeros((L, L))
        h1[i, j] = 1.0
        m = chemistry_mpo(h1, np.zeros((L, L, L, L)))
        assert abs(sandwich(cores, m, cores) / nrm2 - gh[i, j]) < 1e-12
    for (i, j, k, l) in [(0, 1, 2, 3), (2, 2, 1, 1), (3, 0, 0, 3)]:
        e1 = np.zeros((L, L, L, L))
        e1[i, j, k, l] = 1.0
        m = chemistry_mpo(np.zeros((L, L)), e1)
        assert abs(sandwich(cores, m, cores) / nrm2 - geri[i, j, k, l]) < 1e-12
