"""Pins of the oracle's one-site A2DMRG (Alg. 2, one-site case; groups of cores):
the one-site H_eff equals P* A P for the one-site retraction, at full rank one global
iteration reaches the exact ground energy (the coarse space contains the local
solutions, which span the whole space), and the variational chain holds (no
truncation inside the one-site local steps)."""
import numpy as np
import pytest

from oracle import a2dmrg
from oracle.ed import ground_energy, heisenberg_sparse, fermion_sparse
from oracle.env import heff1_apply, left_envs, right_envs
from oracle.mpo import mpo_dense
from oracle.tt import left_orthogonalize, right_orthogonalize, tt_full, tt_inner
from synthetic import chemistry_integrals, chemistry_mpo, heisenberg_mpo, random_tt_cores


def _normalised_left(cores):
    U = left_orthogonalize(cores)
    U[-1] = U[-1] / np.sqrt(tt_inner(U, U))
    return U


@pytest.mark.parametrize("j", [0, 2, 5])
def test_one_site_heff_equals_projected_operator(j):
    L = 6
    mpo = heisenberg_mpo(L)
    Lk = left_orthogonalize(random_tt_cores([2] * L, 4, 9))
    Y = Lk[:j] + right_orthogonalize(Lk[j:])          # j-orthogonal decomposition
    Dl, n, Dr = Y[j].shape
    cols = []
    for idx in range(Dl * n * Dr):
        E = np.zeros(Dl * n * Dr)
        E[idx] = 1.0
        cols.append(tt_full(Y[:j] + [E.reshape(Dl, n, Dr)] + Y[j + 1:]))
    P = np.array(cols).T
    assert np.allclose(P.T @ P, np.eye(P.shape[1]), atol=1e-12)
    HL = left_envs(Y, mpo)[j]
    HR = right_envs(Y, mpo, downto=j + 1)[j + 1]
    H = np.array([heff1_apply(HL, mpo[j], HR, c.reshape(Dl, n, Dr)).ravel()
                  for c in np.eye(Dl * n * Dr)]).T
    assert np.allclose(H, P.T @ mpo_dense(mpo) @ P, atol=1e-12)


@pytest.mark.parametrize("sizes", [[1] * 8, [3, 3, 2], [8]])
def test_full_rank_one_iteration_reaches_ed(sizes):
    L = 8
    mpo = heisenberg_mpo(L)
    E0 = ground_energy(heisenberg_sparse(L))
    U = _normalised_left(random_tt_cores([2] * L, 16, 4))   # exact ranks 2,4,8,16,8,4,2
    U1, rep = a2dmrg.global_iteration_onesite(U, mpo, sizes, D_max=16)
    assert abs(rep["energy"] - E0) < 1e-10 * abs(E0)
    assert abs(rep["lambda_coarse"] - E0) < 1e-10 * abs(E0)


@pytest.mark.parametrize("sizes", [[2, 2, 2], [1] * 6, [4, 2]])
def test_variational_chain_chemistry(sizes):
    """Truncated ranks: lambda_coarse <= every local energy and <= the input energy, and
    the energies stay above the exact ground energy."""
    L = 6
    h, eri = chemistry_integrals(L, 2505)
    mpo = chemistry_mpo(h, eri)
    E0 = ground_energy(fermion_sparse(h, eri))
    U = _normalised_left(random_tt_cores([4] * L, 6, 12))
    E_in = a2dmrg.energy(U, mpo)
    U1, rep = a2dmrg.global_iteration_onesite(U, mpo, sizes, D_max=6)
    lam = rep["lambda_coarse"]
    assert lam <= E_in + 1e-10
    for th, rq in zip(rep["local_energies"], rep["local_rayleigh"]):
        assert abs(th - rq) < 1e-9 * max(1.0, abs(th))          # no truncation locally
        assert lam <= th + 1e-10
    assert E0 - 1e-10 <= lam
    assert E0 - 1e-10 <= rep["energy"]
