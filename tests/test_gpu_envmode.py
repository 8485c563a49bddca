"""The memory-limited environment mode (environments rebuilt on demand from the chain
ends, none kept) gives the same global iteration as the stored mode: the same kernels
run on the same data, so the coarse matrices, the coarse eigenpair and the new iterate
agree to the rounding of the precision."""
import numpy as np
import pytest

from oracle import a2dmrg as oa2
from oracle.tt import left_orthogonalize, tt_full, tt_inner
from synthetic import chemistry_integrals, chemistry_mpo, random_tt_cores

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


@pytest.mark.parametrize("prec,one_site,sizes", [("fp64", False, [3, 2, 2]),
                                                  ("bf16", False, [3, 2, 2]),
                                                  ("fp32", True, [3, 3, 2])])
def test_low_memory_matches_stored(ctx, prec, one_site, sizes):
    L = 8
    h, eri = chemistry_integrals(L, 2505)
    m = chemistry_mpo(h, eri)
    raw = random_tt_cores([4] * L, 8, 77)
    mpo = a2.MPO(ctx, m)
    out = {}
    for low in (False, True):
        t = a2.TT.from_cores(ctx, raw)
        t.left_orthogonalize()
        reps = [a2.additive_sweep(ctx, t, mpo, len(sizes), partition=sizes, D_max=8, prec=prec,
                                  one_site=one_site, low_memory=low, sequential=True, **KW)
                for _ in range(2)]
        out[low] = (reps, tt_full(t.cores()))
    # FP64: the same to rounding; FP32 / mixed modes: the split-K reductions add their
    # partial tiles with atomics, so two runs agree to the FP32 rounding level only
    tol = 1e-12 if prec == "fp64" else 2e-6
    for r0, r1 in zip(out[False][0], out[True][0]):
        assert np.allclose(r0["S_hat"], r1["S_hat"], atol=tol)
        assert np.allclose(r0["A_hat"], r1["A_hat"], atol=10 * tol)
        assert abs(r0["lambda_coarse"] - r1["lambda_coarse"]) < tol * abs(r0["lambda_coarse"])
    x0, x1 = out[False][1], out[True][1]
    assert abs(abs(x0 @ x1) - 1.0) < (1e-11 if prec == "fp64" else 1e-5)


def test_low_memory_against_oracle(ctx):
    L = 8
    h, eri = chemistry_integrals(L, 2505)
    m = chemistry_mpo(h, eri)
    raw = random_tt_cores([4] * L, 8, 77)
    U = left_orthogonalize(raw)
    U[-1] = U[-1] / np.sqrt(tt_inner(U, U))
    _, rep0 = oa2.global_iteration(U, m, [3, 2, 2], D_max=8, **KW)
    mpo = a2.MPO(ctx, m)
    t = a2.TT.from_cores(ctx, raw)
    t.left_orthogonalize()
    rep = a2.additive_sweep(ctx, t, mpo, 3, partition=[3, 2, 2], D_max=8, prec="fp64",
                            low_memory=True, **KW)
    assert abs(rep["lambda_coarse"] - rep0["lambda_coarse"]) < 1e-10 * abs(rep0["lambda_coarse"])
    E, _ = a2.energy(ctx, t, mpo)
    assert abs(E - rep0["energy"]) < 1e-10 * abs(E)


@pytest.mark.parametrize("prec,one_site", [("fp64", False), ("bf16", False), ("fp32", True),
                                           ("f64emu", False)])
def test_cuda_graph_matvecs_match_eager(ctx, prec, one_site):
    """H_eff applications replayed from CUDA graphs give the eager path's iteration (to the
    rounding of the precision; split-K tiles are added with atomics)."""
    L = 8
    h, eri = chemistry_integrals(L, 2505)
    m = chemistry_mpo(h, eri)
    raw = random_tt_cores([4] * L, 8, 77)
    sizes = [3, 3, 2] if one_site else [3, 2, 2]
    mpo = a2.MPO(ctx, m)
    out = {}
    for graphs in (False, True):
        t = a2.TT.from_cores(ctx, raw)
        t.left_orthogonalize()
        reps = [a2.additive_sweep(ctx, t, mpo, len(sizes), partition=sizes, D_max=8, prec=prec,
                                  one_site=one_site, graphs=graphs, sequential=True, **KW)
                for _ in range(2)]
        out[graphs] = (reps, a2.energy(ctx, t, mpo)[0])
    tol = 1e-11 if prec in ("fp64", "f64emu") else 2e-6
    for r0, r1 in zip(out[False][0], out[True][0]):
        assert abs(r0["lambda_coarse"] - r1["lambda_coarse"]) < tol * abs(r0["lambda_coarse"])
        assert r0["matvecs"] == r1["matvecs"] or prec not in ("fp64", "f64emu")
    assert abs(out[False][1] - out[True][1]) < tol * abs(out[False][1])
