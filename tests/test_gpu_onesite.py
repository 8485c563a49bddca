"""GPU parity of the one-site case of Alg. 2 (P groups of cores, one-site micro-steps
with QR between the cores of a group, ranks unchanged locally) against the oracle's
one-site global iteration, through the C ABI."""
import numpy as np
import pytest

from oracle import a2dmrg as oa2
from oracle.ed import ground_energy, heisenberg_sparse
from oracle.tt import left_orthogonalize, tt_full, tt_inner
from synthetic import chemistry_integrals, chemistry_mpo, heisenberg_mpo, random_tt_cores

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_23429_gb300 as a2  # noqa: E402

KW = dict(svd_tol=1e-10, eig_tol=1e-10, coarse_eps=1e-10)


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


def _compare(rep, rep0, tol):
    scale = np.abs(rep0["A_hat"]).max()
    assert np.allclose(rep["S_hat"], rep0["S_hat"], atol=tol)
    assert np.allclose(rep["A_hat"], rep0["A_hat"], atol=tol * scale)
    assert abs(rep["lambda_coarse"] - rep0["lambda_coarse"]) < tol * abs(rep0["lambda_coarse"])
    assert np.allclose(rep["energy_local"], rep0["local_energies"], atol=tol * scale)
    assert rep["coarse_rank"] == rep0["coarse_rank"]


@pytest.mark.parametrize("sizes", [[1] * 8, [3, 3, 2], [2, 1, 1, 3, 1]])
def test_full_rank_heisenberg_reaches_ed(ctx, sizes):
    """At full TT rank one iteration reaches the exact ground energy (the local
    solutions span the whole space); the coarse problem matches the oracle."""
    L = 8
    m = heisenberg_mpo(L)
    raw, U = _start([2] * L, 16, 4)
    U1, rep0 = oa2.global_iteration_onesite(U, m, sizes, D_max=16, **KW)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    rep = a2.additive_sweep(ctx, t, mpo, len(sizes), partition=sizes, D_max=16, prec="fp64",
                            one_site=True, **KW)
    _compare(rep, rep0, 1e-9)
    assert len(rep["krylov"]) == L
    E, nrm = a2.energy(ctx, t, mpo)
    assert abs(nrm - 1.0) < 1e-12
    E_ed = ground_energy(heisenberg_sparse(L))
    assert abs(E - rep0["energy"]) < 1e-10 * abs(E)
    assert abs(E - E_ed) < 1e-9 * abs(E_ed)


@pytest.mark.parametrize("sizes", [[2, 2, 2], [1] * 6, [4, 2], [1, 4, 1]])
def test_chemistry_truncated_matches_oracle(ctx, sizes):
    """Truncated ranks (r = 6): every coarse entry, the coarse eigenpair and the
    compressed iterate agree with the oracle's one-site global iteration."""
    L = 6
    h, eri = chemistry_integrals(L, 2505)
    m = chemistry_mpo(h, eri)
    raw, U = _start([4] * L, 6, 12)
    U1, rep0 = oa2.global_iteration_onesite(U, m, sizes, D_max=6, **KW)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    rep = a2.additive_sweep(ctx, t, mpo, len(sizes), partition=sizes, D_max=6, prec="fp64",
                            one_site=True, **KW)
    _compare(rep, rep0, 1e-9)
    assert np.allclose(rep["coeffs"], rep0["coeffs"], atol=1e-7)
    E, _ = a2.energy(ctx, t, mpo)
    assert abs(E - rep0["energy"]) < 1e-9 * abs(E)
    x, x0 = tt_full(t.cores()), tt_full(U1)
    assert abs(abs(x @ x0) - 1.0) < 1e-8


def test_classical_one_site_half_sweep(ctx):
    """P = 1: a classical one-site half-sweep (Alg. 1, one-site case)."""
    L = 6
    h, eri = chemistry_integrals(L, 2505)
    m = chemistry_mpo(h, eri)
    raw, U = _start([4] * L, 6, 12)
    U1, rep0 = oa2.global_iteration_onesite(U, m, [L], D_max=6, **KW)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    rep = a2.classical_sweep(ctx, t, mpo, D_max=6, prec="fp64", one_site=True, **KW)
    assert abs(rep["energy_local"][0] - rep0["local_energies"][0]) < 1e-9 * abs(rep0["energy"])
    E, _ = a2.energy(ctx, t, mpo)
    # a half-sweep's result is its last local solution (no coarse mixing)
    assert abs(E - rep0["local_energies"][0]) < 1e-9 * abs(E)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_precision_one_site(ctx, prec):
    """FP32 local contractions: the energy after one iteration within 1e-5 (relative) of
    the FP64 oracle."""
    L = 6
    h, eri = chemistry_integrals(L, 2505)
    m = chemistry_mpo(h, eri)
    raw, U = _start([4] * L, 6, 12)
    _, rep0 = oa2.global_iteration_onesite(U, m, [2, 2, 2], D_max=6, **KW)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    a2.additive_sweep(ctx, t, mpo, 3, partition=[2, 2, 2], D_max=6, prec=prec, one_site=True,
                      svd_tol=1e-10, eig_tol=1e-7, coarse_eps=1e-10)
    E, _ = a2.energy(ctx, t, mpo)
    assert abs(E - rep0["energy"]) < 1e-5 * abs(rep0["energy"])


def test_invalid_core_partition_raises(ctx):
    L = 6
    m = heisenberg_mpo(L)
    raw, _ = _start([2] * L, 4, 3)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    before = tt_full(t.cores())
    with pytest.raises(Exception):
        a2.additive_sweep(ctx, t, mpo, 2, partition=[3, 2], D_max=8, one_site=True, **KW)
    assert np.array_equal(tt_full(t.cores()), before)
