"""CPU-only: the identity-on-physical split W = delta_st G + W_rest that the library
uses to fold the dense block of the operator automaton's hand-over core into the
environments (host logic of a2_mpo_fold_split; no device call)."""
import numpy as np
import pytest

from synthetic import chemistry_integrals, chemistry_mpo, heisenberg_mpo


@pytest.fixture(scope="module")
def chem16():
    h, eri = chemistry_integrals(16, 2505)
    return chemistry_mpo(h, eri)


def _a2():
    import paper_2505_23429_gb300 as a2
    return a2


def _check_split(W, G):
    Rl, n, _, Rr = W.shape
    rest = W.copy()
    for s in range(n):
        rest[:, s, s, :] -= G
    # exact: G entries are copies of W entries
    recon = rest.copy()
    for s in range(n):
        recon[:, s, s, :] += G
    assert np.array_equal(recon, W)
    # G is taken only where all diagonal entries agree and are nonzero ...
    diag = np.stack([W[:, s, s, :] for s in range(n)])
    same = np.all(diag == diag[0], axis=0) & (diag[0] != 0)
    assert np.array_equal(G != 0, same)
    assert np.array_equal(G[same], diag[0][same])
    # ... so the remainder has no such entry left
    rd = np.stack([rest[:, s, s, :] for s in range(n)])
    assert not np.any(np.all(rd == rd[0], axis=0) & (rd[0] != 0))


def test_fold_split_hand_over_core(chem16):
    a2 = _a2()
    flags = []
    for j, W in enumerate(chem16):
        G, nnz, foldable = a2.fold_split(W)
        _check_split(W, G)
        assert nnz == np.count_nonzero(G)
        flags.append(foldable)
    # the complementary-operator hand-over core (the one with by far the most nonzeros)
    # is the only one with a large identity block
    nz = [np.count_nonzero(W) for W in chem16]
    assert flags == [j == int(np.argmax(nz)) for j in range(len(chem16))]
    G, nnz, _ = a2.fold_split(chem16[int(np.argmax(nz))])
    assert nnz > 0.7 * np.count_nonzero(chem16[int(np.argmax(nz))]) / 4


def test_fold_split_small_cases():
    a2 = _a2()
    # Heisenberg: identity passes only, never folded
    for W in heisenberg_mpo(6):
        G, nnz, foldable = a2.fold_split(W)
        _check_split(W, G)
        assert not foldable and nnz <= 2
    # constructed core: W = I (x) G0 + sparse off-diagonal part, with one diagonal
    # entry broken so that its position must stay in W_rest
    rng = np.random.default_rng(5)
    Rl, n, Rr = 40, 3, 50
    G0 = rng.standard_normal((Rl, Rr)) * (rng.random((Rl, Rr)) < 0.8)
    W = np.zeros((Rl, n, n, Rr))
    for s in range(n):
        W[:, s, s, :] = G0
    W[:, 0, 1, :] = rng.standard_normal((Rl, Rr)) * (rng.random((Rl, Rr)) < 0.1)
    i, j = np.argwhere(G0 != 0)[0]
    W[i, 2, 2, j] += 1.0
    G, nnz, foldable = a2.fold_split(W)
    _check_split(W, G)
    assert G[i, j] == 0.0 and nnz == np.count_nonzero(G0) - 1
    assert foldable == (nnz >= 1024 and nnz * 64 >= Rl * Rr)


def test_fold_split_rejects_bad_arguments():
    a2 = _a2()
    with pytest.raises(Exception):
        a2.fold_split(np.zeros((0, 2, 2, 3)))
