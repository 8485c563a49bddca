"""The mixed-precision path at the settings it is run with (eig_tol = svd_tol = 1e-6, the
coarse cut eps = 1e-10 of the FP64 path): tensor-core BF16 / split-product Lanczos, FP64
environments computed to FP64-class accuracy, FP64 coarse matrices and the FP64
refinement of every local Ritz pair.  Checked against the FP64 oracle: the coarse
matrices S_hat and A_hat element by element after one global iteration, and converged
energies at truncating bond dimensions within 1e-6 absolute.  C-ABI calls."""
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

PROD = dict(svd_tol=1e-6, eig_tol=1e-6, coarse_eps=1e-10)


@pytest.fixture(scope="module")
def ctx():
    c = a2.Context(0)
    yield c
    assert a2.device_error(c) == 0
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


@pytest.mark.parametrize("prec", ["bf16", "f32emu"])
def test_one_iteration_coarse_matrices_elementwise(ctx, prec):
    """One iteration of the L = 12 Heisenberg workload (D = 32, P = 2) with local solves
    taken to 1e-10: the tensor-core phases stop at their own accuracy and the FP64
    refinement finishes each solve, so S_hat and A_hat (from FP64-class environments)
    match the oracle's full-vector inner products entry by entry."""
    L = 12
    m = heisenberg_mpo(L)
    raw, U = _start([2] * L, 4, 23429)
    kw = dict(svd_tol=1e-10, eig_tol=1e-10, coarse_eps=1e-10)
    _, rep0 = oa2.global_iteration(U, m, [6, 5], 32, **kw)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    rep = a2.additive_sweep(ctx, t, mpo, 2, partition=[6, 5], D_max=32, prec=prec, **kw)
    S0, A0 = rep0["S_hat"], rep0["A_hat"]
    assert np.max(np.abs(rep["S_hat"] - S0)) < 1e-9
    assert np.max(np.abs(rep["A_hat"] - A0)) < 1e-9 * np.abs(A0).max()
    assert abs(rep["lambda_coarse"] - rep0["lambda_coarse"]) < 1e-10 * abs(rep0["lambda_coarse"])
    assert rep["coarse_rank"] == rep0["coarse_rank"]
    assert np.allclose(rep["energy_local"], rep0["local_energies"], rtol=0, atol=1e-9)
    assert rep["matvecs_f64"] > 0
    E, _ = a2.energy(ctx, t, mpo)
    assert abs(E - rep0["energy"]) < 1e-10 * abs(E)


def test_refinement_off_uses_no_fp64_operator(ctx):
    L = 8
    m = heisenberg_mpo(L)
    raw, _ = _start([2] * L, 4, 5)
    mpo = a2.MPO(ctx, m)
    t = _gpu_tt(ctx, raw)
    rep = a2.additive_sweep(ctx, t, mpo, 2, partition=[4, 3], D_max=8, prec="bf16", refine=0,
                            **PROD)
    assert rep["matvecs_f64"] == 0
    t = _gpu_tt(ctx, raw)
    rep = a2.additive_sweep(ctx, t, mpo, 2, partition=[4, 3], D_max=8, prec="bf16", refine=1,
                            **PROD)
    assert rep["matvecs_f64"] >= L - 1          # at least one FP64 application per bond


def _converge_gpu(ctx, mpo, raw, P, sizes, D, n_iter, prec):
    t = _gpu_tt(ctx, raw)
    E_prev = None
    for _ in range(n_iter):
        rep = a2.additive_sweep(ctx, t, mpo, P, partition=sizes, D_max=D, prec=prec, **PROD)
        E = rep["energy_in"]
        if E_prev is not None and abs(E - E_prev) < 1e-12 * abs(E):
            break
        E_prev = E
    return a2.energy(ctx, t, mpo, "fp64")[0]


def test_bf16_converged_heisenberg_truncated_matches_oracle(ctx):
    """L = 12 Heisenberg at D = 32 (truncated: the exact middle rank is 64), production
    tolerances: the BF16 default path converges to the FP64 oracle's energy within 1e-6."""
    L = 12
    m = heisenberg_mpo(L)
    raw, U = _start([2] * L, 4, 23429)
    _, hist = oa2.run(U, m, [6, 5], 32, 12, tol_rel=1e-12, **PROD)
    E_or = hist[-1]["energy"]
    mpo = a2.MPO(ctx, m)
    E = _converge_gpu(ctx, mpo, raw, 2, [6, 5], 32, 12, "bf16")
    assert abs(E - E_or) < 1e-6


def test_bf16_converged_chemistry_truncated_matches_oracle(ctx):
    """Random chemistry Hamiltonian, L = 6 orbitals, D = 48 (the exact middle rank is 64,
    so the middle bond is truncated), P = 3 groups [2, 2, 1], production tolerances: the
    energies the BF16 default path and the FP64 oracle settle at agree within 1e-6.  (At
    stronger truncation both runs keep moving by ~1e-6 from one iteration to the next,
    the compression of the coarse combination discarding a few percent of weight.)"""
    L = 6
    h, eri = chemistry_integrals(L, 2505)
    m = chemistry_mpo(h, eri)
    raw, U = _start([4] * L, 4, 23429)
    _, hist = oa2.run(U, m, [2, 2, 1], 48, 12, tol_rel=1e-11, **PROD)
    E_or = hist[-1]["energy"]
    mpo = a2.MPO(ctx, m)
    E = _converge_gpu(ctx, mpo, raw, 3, [2, 2, 1], 48, 12, "bf16")
    assert abs(E - E_or) < 1e-6
