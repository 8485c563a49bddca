"""GPU parity of Extension One (the K lowest eigenvectors of every group's last local
problem enrich the coarse space; extension remark after Alg. 2) against the oracle,
two-site and one-site, through the C ABI."""
import numpy as np
import pytest

from oracle import a2dmrg as oa2
from oracle.tt import left_orthogonalize, tt_inner
from synthetic import chemistry_integrals, chemistry_mpo, heisenberg_mpo, random_tt_cores

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_23429_gb300 as a2  # noqa: E402

KW = dict(svd_tol=1e-10, eig_tol=1e-11, coarse_eps=1e-10)


@pytest.fixture(scope="module")
def ctx():
    c = a2.Context(0)
    yield c
    c.close()


def _start(phys, r0, seed):
    raw = random_tt_cores(phys, r0, seed)
    U = left_orthogonalize(raw)
    U[-1] = U[-1] / np.sqrt(tt_inner(U, U))
    return raw, U


def _gpu_tt(ctx, raw):
    t = a2.TT.from_cores(ctx, raw)
    t.left_orthogonalize()
    return t


def _check(rep, rep0, vec_tol):
    m = len(rep0["coeffs"])
    assert rep["coarse_dim"] == m
    scale = abs(rep0["lambda_coarse"])
    assert abs(rep["lambda_coarse"] - rep0["lambda_coarse"]) < 1e-9 * scale
    assert np.allclose(rep["energy_local"], rep0["local_energies"], atol=1e-9 * scale)
    # eigenvectors agree to ~ residual / gap: first-order quantities get vec_tol.  The
    # sign of an eigenvector is fixed by its overlap with the start vector, which can be
    # close to zero for the further eigenvectors: compare sign-invariant magnitudes
    for key, sc in (("S_hat", 1.0), ("A_hat", np.abs(rep0["A_hat"]).max())):
        d = np.abs(np.abs(rep[key]) - np.abs(rep0[key]))
        i, j = np.unravel_index(np.argmax(d), d.shape)
        assert d.max() < vec_tol * sc, (key, i, j, rep[key][i, j], rep0[key][i, j])


@pytest.mark.parametrize("sizes,K", [([2, 2, 1], 3), ([1] * 5, 4)])
def test_two_site_chemistry(ctx, sizes, K):
    L = 6
    h, eri = chemistry_integrals(L, 2505)
    m = chemistry_mpo(h, eri)
    raw, U = _start([4] * L, 4, 12)
    U1, rep0 = oa2.global_iteration(U, m, sizes, D_max=4, n_eig=K, **KW)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    rep = a2.additive_sweep(ctx, t, mpo, len(sizes), partition=sizes, D_max=4, prec="fp64",
                            n_eig=K, **KW)
    _check(rep, rep0, 1e-6)
    E, nrm = a2.energy(ctx, t, mpo)
    assert abs(nrm - 1.0) < 1e-12
    assert abs(E - rep0["energy"]) < 1e-7 * abs(E)


@pytest.mark.parametrize("sizes,K", [([2, 2, 2, 2], 4), ([3, 5], 6)])
def test_one_site_heisenberg(ctx, sizes, K):
    L = 8
    m = heisenberg_mpo(L)
    raw, U = _start([2] * L, 4, 7)
    _, rep0 = oa2.global_iteration_onesite(U, m, sizes, D_max=4, n_eig=K, **KW)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    rep = a2.additive_sweep(ctx, t, mpo, len(sizes), partition=sizes, D_max=4, prec="fp64",
                            one_site=True, n_eig=K, **KW)
    _check(rep, rep0, 1e-6)
    E, _ = a2.energy(ctx, t, mpo)
    assert abs(E - rep0["energy"]) < 1e-7 * abs(E)


def test_one_site_all_eigenvectors(ctx):
    """K above every local dimension: each group keeps all its eigenvectors (capped per
    group), 33 coarse vectors; the coarse eigenvalue equals the oracle's, which equals
    the Ritz value on the sum of the one-site subspaces."""
    L = 5
    m = heisenberg_mpo(L)
    raw, U = _start([2] * L, 2, 43)
    _, rep0 = oa2.global_iteration_onesite(U, m, [1] * L, D_max=64, n_eig=8, svd_tol=0.0,
                                           eig_tol=1e-11, coarse_eps=1e-10)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    rep = a2.additive_sweep(ctx, t, mpo, L, partition=[1] * L, D_max=64, prec="fp64",
                            one_site=True, n_eig=8, svd_tol=0.0, eig_tol=1e-11,
                            coarse_eps=1e-10)
    assert rep["coarse_dim"] == len(rep0["coeffs"]) == 33
    assert abs(rep["lambda_coarse"] - rep0["lambda_coarse"]) < 1e-9 * abs(rep0["lambda_coarse"])
    assert np.allclose(np.sort(rep["energy_local"]), np.sort(rep0["local_energies"]),
                       atol=1e-9)


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_mixed_precision_two_site(ctx, prec):
    L = 6
    h, eri = chemistry_integrals(L, 2505)
    m = chemistry_mpo(h, eri)
    raw, U = _start([4] * L, 4, 12)
    _, rep0 = oa2.global_iteration(U, m, [2, 2, 1], D_max=4, n_eig=3, **KW)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    rep = a2.additive_sweep(ctx, t, mpo, 3, partition=[2, 2, 1], D_max=4, prec=prec, n_eig=3,
                            svd_tol=1e-10, eig_tol=1e-7, coarse_eps=1e-10)
    assert rep["coarse_dim"] == 10
    assert abs(rep["lambda_coarse"] - rep0["lambda_coarse"]) < 1e-5 * abs(rep0["lambda_coarse"])


def test_classical_rejects_n_eig(ctx):
    L = 6
    m = heisenberg_mpo(L)
    raw, _ = _start([2] * L, 4, 3)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    with pytest.raises(Exception):
        a2.classical_sweep(ctx, t, mpo, D_max=8, n_eig=2, **KW)
