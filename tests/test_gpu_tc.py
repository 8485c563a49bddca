"""tcgen05 tensor-core path: the BF16 GEMM stages against their plain definition
(FP64 products of the same BF16 inputs) and the BF16 H_eff chain / sweep against
the oracle.  C-ABI calls."""
import numpy as np
import pytest

from oracle.env import heff_apply as oracle_heff
from synthetic import chemistry_integrals, chemistry_mpo, random_tt_cores

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_23429_gb300 as a2  # noqa: E402
from gpu_common import dev, host, rel  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = a2.Context(0)
    yield c
    assert a2.device_error(c) == 0
    c.close()


def _bf16(rows, k, ld, seed):
    g = torch.Generator().manual_seed(seed)
    full = torch.zeros(rows, ld, dtype=torch.bfloat16)
    full[:, :k] = torch.randn(rows, k, generator=g).to(torch.bfloat16)
    return full


@pytest.mark.parametrize("M,N,K,splitk", [
    (128, 128, 64, 1), (256, 256, 256, 1), (200, 300, 72, 1), (1000, 130, 520, 1),
    (129, 257, 8, 1), (64, 40, 16, 1), (4096, 256, 8192, 8), (333, 96, 1000, 3),
    (512, 2048, 256, 1),
    # many tiles per persistent CTA with a ragged last row tile (TMA-store epilogue)
    (58438, 512, 64, 1), (20070, 136, 200, 3), (19999, 300, 40, 1)])
def test_gemm_bf16_matches_definition(ctx, M, N, K, splitk):
    ld = (K + 7) // 8 * 8
    A = _bf16(M, K, ld, 1)
    B = _bf16(N, K, ld, 2)
    C = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    Ad, Bd = A.cuda(), B.cuda()
    torch.cuda.synchronize()
    a2.gemm_bf16(ctx, Ad, Bd, C, K=K, splitk=splitk)
    ref = A[:, :K].double().numpy() @ B[:, :K].double().numpy().T
    got = C.cpu().double().numpy()
    err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-30)
    assert err < 2e-5, err


@pytest.mark.parametrize("k,Dl,Dr", [(0, 1, 16), (2, 16, 64), (3, 64, 16), (1, 4, 64)])
def test_heff_bf16_chemistry(ctx, k, Dl, Dr):
    h, eri = chemistry_integrals(6, 2505)
    m = chemistry_mpo(h, eri)
    mpo = a2.MPO(ctx, m)
    rng = np.random.default_rng(k)
    Lh = rng.standard_normal((Dl, m[k].shape[0], Dl))
    Rh = rng.standard_normal((Dr, m[k + 1].shape[3], Dr))
    x = rng.standard_normal((Dl, 4, 4, Dr))
    ref = oracle_heff(Lh, m[k], m[k + 1], Rh, x)
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    a2.heff_apply(ctx, mpo, k, dev(Lh), dev(Rh), dev(x), y, prec="bf16")
    assert rel(host(y, ctx), ref) < 2e-2


@pytest.mark.parametrize("k,Dl,Dr", [(0, 1, 16), (2, 16, 64), (3, 64, 16), (1, 4, 64), (2, 33, 9)])
def test_heff_f32emu_chemistry(ctx, k, Dl, Dr):
    """Three-slice BF16 products (six pairs) reach FP32 accuracy on tcgen05."""
    h, eri = chemistry_integrals(6, 2505)
    m = chemistry_mpo(h, eri)
    mpo = a2.MPO(ctx, m)
    rng = np.random.default_rng(10 + k)
    Lh = rng.standard_normal((Dl, m[k].shape[0], Dl))
    Rh = rng.standard_normal((Dr, m[k + 1].shape[3], Dr))
    x = rng.standard_normal((Dl, 4, 4, Dr))
    ref = oracle_heff(Lh, m[k], m[k + 1], Rh, x)
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    a2.heff_apply(ctx, mpo, k, dev(Lh), dev(Rh), dev(x), y, prec="f32emu")
    assert rel(host(y, ctx), ref) < 5e-6


def test_f32emu_sweep_energy_within_1e6_of_fp64(ctx):
    h, eri = chemistry_integrals(6, 2505)
    m = chemistry_mpo(h, eri)
    mpo = a2.MPO(ctx, m)
    raw = random_tt_cores([4] * 6, 4, 23429)
    res = {}
    for prec in ("fp64", "f32emu"):
        t = a2.TT.from_cores(ctx, raw)
        t.left_orthogonalize()
        for _ in range(4):
            a2.additive_sweep(ctx, t, mpo, 3, partition=[2, 2, 1], D_max=64, prec=prec,
                              svd_tol=1e-10, eig_tol=1e-8, coarse_eps=1e-10)
        res[prec] = a2.energy(ctx, t, mpo, "fp64")[0]
    assert abs(res["f32emu"] - res["fp64"]) < 1e-6


def test_bf16_sweep_energy_within_1e6_of_fp64(ctx):
    h, eri = chemistry_integrals(6, 2505)
    m = chemistry_mpo(h, eri)
    mpo = a2.MPO(ctx, m)
    raw = random_tt_cores([4] * 6, 4, 23429)
    res = {}
    for prec in ("fp64", "bf16"):
        t = a2.TT.from_cores(ctx, raw)
        t.left_orthogonalize()
        for _ in range(4):
            a2.additive_sweep(ctx, t, mpo, 3, partition=[2, 2, 1], D_max=64, prec=prec,
                              svd_tol=1e-10, eig_tol=1e-8, coarse_eps=1e-10)
        res[prec] = a2.energy(ctx, t, mpo, "fp64")[0]
    assert abs(res["bf16"] - res["fp64"]) < 1e-6


# ---- identity-on-physical fold of the hand-over core (W = I (x) G + W_rest)

@pytest.fixture(scope="module")
def chem16(ctx):
    h, eri = chemistry_integrals(16, 2505)
    m = chemistry_mpo(h, eri)
    return m, a2.MPO(ctx, m)


@pytest.mark.parametrize("prec,tol", [("bf16", 2e-2), ("f32emu", 5e-6)])
@pytest.mark.parametrize("k,Dl,Dr", [(7, 32, 32), (8, 32, 32), (7, 24, 40), (8, 40, 24),
                                     (7, 16, 36), (8, 8, 12)])
def test_heff_hand_over_fold(ctx, chem16, prec, tol, k, Dl, Dr):
    """Bonds 7 / 8 of the L=16 chemistry MPO touch its hand-over core (site 8), whose
    identity block is folded into the right (bond 7) or left (bond 8) environment;
    Dr % 8 != 0 keeps the right fold off.  Folded and unfolded chains both match the
    oracle."""
    m, mpo = chem16
    assert mpo.fold_info(8)[0] and not mpo.fold_info(7)[0]
    rng = np.random.default_rng(100 + k + Dl)
    Lh = rng.standard_normal((Dl, m[k].shape[0], Dl))
    Rh = rng.standard_normal((Dr, m[k + 1].shape[3], Dr))
    x = rng.standard_normal((Dl, 4, 4, Dr))
    ref = oracle_heff(Lh, m[k], m[k + 1], Rh, x)
    out = {}
    for fold in (True, False):
        mpo.set_fold(fold)
        y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
        a2.heff_apply(ctx, mpo, k, dev(Lh), dev(Rh), dev(x), y, prec=prec)
        out[fold] = host(y, ctx)
    mpo.set_fold(True)
    assert rel(out[True], ref) < tol
    assert rel(out[False], ref) < tol


def _fold_mpo(seed, n=2, R=(64, 72, 80)):
    """Four-site operator whose two middle cores both carry a large identity block."""
    rng = np.random.default_rng(seed)
    Ra, Rb, Rc = R
    cores = [rng.standard_normal((1, n, n, Ra)) * 0.5]
    for Rl, Rr in ((Ra, Rb), (Rb, Rc)):
        W = np.zeros((Rl, n, n, Rr))
        G = rng.standard_normal((Rl, Rr)) * (rng.random((Rl, Rr)) < 0.7)
        for s in range(n):
            W[:, s, s, :] = G
        W[:, 0, n - 1, :] = rng.standard_normal((Rl, Rr)) * (rng.random((Rl, Rr)) < 0.05)
        W[:, n - 1, n - 1, :] += rng.standard_normal((Rl, Rr)) * (rng.random((Rl, Rr)) < 0.05)
        cores.append(W)
    cores.append(rng.standard_normal((Rc, n, n, 1)) * 0.5)
    return cores


@pytest.mark.parametrize("prec,tol", [("bf16", 2e-2), ("f32emu", 5e-6)])
@pytest.mark.parametrize("n,Dl,Dr", [(2, 48, 64), (4, 16, 24), (2, 33, 8)])
def test_heff_both_cores_folded(ctx, prec, tol, n, Dl, Dr):
    m = _fold_mpo(7 + n, n=n)
    mpo = a2.MPO(ctx, m)
    assert mpo.fold_info(1)[0] and mpo.fold_info(2)[0]
    rng = np.random.default_rng(Dl)
    Lh = rng.standard_normal((Dl, m[1].shape[0], Dl))
    Rh = rng.standard_normal((Dr, m[2].shape[3], Dr))
    x = rng.standard_normal((Dl, n, n, Dr))
    ref = oracle_heff(Lh, m[1], m[2], Rh, x)
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    a2.heff_apply(ctx, mpo, 1, dev(Lh), dev(Rh), dev(x), y, prec=prec)
    assert rel(host(y, ctx), ref) < tol
    mpo.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "f32emu"])
def test_heff_operator_handle(ctx, chem16, prec):
    """a2_heff_create / a2_heff_apply_op (environments converted once) give the same
    result as a2_heff_apply, call after call (up to the summation order of the split-K
    atomic accumulation)."""
    tol = {"fp64": 1e-13, "fp32": 1e-6, "bf16": 1e-5, "f32emu": 1e-6}[prec]
    m, mpo = chem16
    k, Dl, Dr = 7, 16, 24
    rng = np.random.default_rng(3)
    Lh = dev(rng.standard_normal((Dl, m[k].shape[0], Dl)))
    Rh = dev(rng.standard_normal((Dr, m[k + 1].shape[3], Dr)))
    x = dev(rng.standard_normal((Dl, 4, 4, Dr)))
    y0 = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    a2.heff_apply(ctx, mpo, k, Lh, Rh, x, y0, prec=prec)
    ref = host(y0, ctx)
    op = a2.HeffOp(ctx, mpo, k, Lh, Rh, prec=prec)
    del Lh, Rh
    for _ in range(2):
        y = torch.full(x.shape, float("nan"), dtype=torch.float64, device="cuda")
        op.apply(x, y)
        got = host(y, ctx)
        assert np.all(np.isfinite(got)) and rel(got, ref) < tol
    op.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("f32emu", 1e-6), ("f64emu", 1e-13)])
def test_autotuners_do_not_change_results(ctx, prec, tol):
    """The GEMM and sparse-stage autotuners only pick launch shapes: H_eff with them on
    (after their timing trials) and off agree to the rounding of the precision (split-K
    tiles are added with atomics, so not bitwise)."""
    h, eri = chemistry_integrals(6, 2505)
    m = chemistry_mpo(h, eri)
    mpo = a2.MPO(ctx, m)
    k, Dl, Dr = 2, 48, 40
    rng = np.random.default_rng(77)
    Lh = rng.standard_normal((Dl, m[k].shape[0], Dl))
    Rh = rng.standard_normal((Dr, m[k + 1].shape[3], Dr))
    x = rng.standard_normal((Dl, 4, 4, Dr))
    out = []
    try:
        for on in (True, True, False):
            a2.set_autotune(on, sparse=on)
            y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
            a2.heff_apply(ctx, mpo, k, dev(Lh), dev(Rh), dev(x), y, prec=prec)
            out.append(host(y, ctx))
    finally:
        a2.set_autotune(True)
    assert rel(out[1], out[2]) < tol
    assert rel(out[0], out[1]) < tol
