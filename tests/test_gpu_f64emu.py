"""FP64 emulation of the H_eff tensor-core stages (Ozaki scheme with BF16 slices,
exact per-level FP32 accumulation): the contraction agrees with the oracle's FP64
H_eff and with the FP64 SIMT path to FP64 rounding, including ragged bond dimensions,
long reductions split over many K chunks and rows of zeros; a global iteration in this
precision reproduces the FP64 one.  C-ABI calls."""
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


@pytest.fixture(scope="module")
def chem6():
    h, eri = chemistry_integrals(6, 2505)
    return chemistry_mpo(h, eri)


@pytest.fixture(scope="module")
def chem16():
    h, eri = chemistry_integrals(16, 2505)
    return chemistry_mpo(h, eri)


def _case(m, k, Dl, Dr, seed):
    rng = np.random.default_rng(seed)
    Lh = rng.standard_normal((Dl, m[k].shape[0], Dl))
    Rh = rng.standard_normal((Dr, m[k + 1].shape[3], Dr))
    x = rng.standard_normal((Dl, m[k].shape[1], m[k + 1].shape[1], Dr))
    return Lh, Rh, x


@pytest.mark.parametrize("k,Dl,Dr", [(0, 1, 16), (2, 16, 64), (3, 64, 16), (1, 4, 64),
                                     (2, 33, 9), (2, 200, 24)])
def test_heff_f64emu_matches_fp64(ctx, chem6, k, Dl, Dr):
    m = chem6
    mpo = a2.MPO(ctx, m)
    Lh, Rh, x = _case(m, k, Dl, Dr, 30 + k)
    ref = oracle_heff(Lh, m[k], m[k + 1], Rh, x)
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    y64 = torch.zeros_like(y)
    a2.heff_apply(ctx, mpo, k, dev(Lh), dev(Rh), dev(x), y, prec="f64emu")
    a2.heff_apply(ctx, mpo, k, dev(Lh), dev(Rh), dev(x), y64, prec="fp64")
    got, g64 = host(y, ctx), host(y64, ctx)
    assert rel(got, ref) < 1e-13
    assert rel(got, g64) < 1e-13


def test_heff_f64emu_long_reduction(ctx, chem16):
    """Hand-over bond of the L = 16 MPO (R_r = 444): S4 reduces over 444*Dr indices, split
    into up to 111 K chunks per level; S1 over Dl = 96 (two K blocks)."""
    m = chem16
    k = 7
    mpo = a2.MPO(ctx, m)
    Lh, Rh, x = _case(m, k, 96, 32, 5)
    ref = oracle_heff(Lh, m[k], m[k + 1], Rh, x)
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    op = a2.HeffOp(ctx, mpo, k, dev(Lh), dev(Rh), prec="f64emu")
    op.apply(dev(x), y)
    ctx.synchronize()
    assert rel(host(y, ctx), ref) < 1e-13


def test_heff_f64emu_zero_rows_and_scales(ctx, chem6):
    """Rows of zeros and rows scaled over 2^-60 .. 2^60 (each row has its own exponent)."""
    m = chem6
    k = 2
    mpo = a2.MPO(ctx, m)
    Lh, Rh, x = _case(m, k, 24, 40, 8)
    Lh[3] = 0.0
    Rh[:, 5] = 0.0
    x[:, :, :, 7] = 0.0
    sc = np.exp2(np.linspace(-60, 60, Lh.shape[0]))
    Lh = Lh * sc[:, None, None]
    ref = oracle_heff(Lh, m[k], m[k + 1], Rh, x)
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    a2.heff_apply(ctx, mpo, k, dev(Lh), dev(Rh), dev(x), y, prec="f64emu")
    got = host(y, ctx)
    # each output row a carries the scale of L row a: compare row by row
    for a in range(Lh.shape[0]):
        r = ref[a]
        if np.abs(r).max() == 0.0:
            assert np.abs(got[a]).max() == 0.0
        else:
            assert rel(got[a], r) < 1e-13


def test_f64emu_sweep_matches_fp64(ctx, chem6):
    m = chem6
    raw = random_tt_cores([4] * 6, 8, 23429)
    mpo = a2.MPO(ctx, m)
    out = {}
    for prec in ("fp64", "f64emu"):
        t = a2.TT.from_cores(ctx, raw)
        t.left_orthogonalize()
        rep = a2.additive_sweep(ctx, t, mpo, 3, partition=[2, 2, 1], D_max=16, prec=prec,
                                svd_tol=1e-10, eig_tol=1e-10, coarse_eps=1e-10)
        out[prec] = (rep, a2.energy(ctx, t, mpo)[0])
    r64, re = out["fp64"][0], out["f64emu"][0]
    assert abs(r64["lambda_coarse"] - re["lambda_coarse"]) < 1e-11 * abs(r64["lambda_coarse"])
    assert np.allclose(r64["energy_local"], re["energy_local"], atol=1e-11)
    assert abs(out["fp64"][1] - out["f64emu"][1]) < 1e-11


@pytest.mark.parametrize("j,Dlb,Drb,Dlk,Drk", [(0, 1, 9, 1, 12), (2, 11, 9, 7, 12),
                                               (3, 40, 33, 40, 33), (5, 16, 1, 9, 1)])
def test_env_update_f64emu_matches_oracle(ctx, chem6, j, Dlb, Drb, Dlk, Drk):
    """Environment updates with both GEMMs Ozaki-emulated and the sparse stage in
    double-float arithmetic (the path the mixed and FP64-emulated sweeps use for their
    FP64 environments): bra and ket of different shapes, ragged dims."""
    from oracle.env import env_left_update, env_right_update
    m = chem6
    mpo = a2.MPO(ctx, m)
    W = m[j]
    rng = np.random.default_rng(40 + j)
    bra = rng.standard_normal((Dlb, 4, Drb))
    ket = rng.standard_normal((Dlk, 4, Drk))
    Hin = rng.standard_normal((Dlb, W.shape[0], Dlk))
    ref = env_left_update(Hin, bra, W, ket)
    out = torch.zeros(ref.shape, dtype=torch.float64, device="cuda")
    a2.env_update(ctx, mpo, j, 0, dev(Hin), dev(bra), dev(ket), out, prec="f64emu")
    assert rel(host(out, ctx), ref) < 1e-13
    Hr = rng.standard_normal((Drb, W.shape[3], Drk))
    ref = env_right_update(Hr, bra, W, ket)
    out = torch.zeros(ref.shape, dtype=torch.float64, device="cuda")
    a2.env_update(ctx, mpo, j, 1, dev(Hr), dev(bra), dev(ket), out, prec="f64emu")
    assert rel(host(out, ctx), ref) < 1e-13


def test_env_update_f64emu_large_and_scaled(ctx, chem16):
    """A middle site of the L = 16 MPO (R = 562) at bond 96 with the input environment's
    rows scaled over 2^-40 .. 2^40: sampled output slices against the oracle."""
    from oracle.env import env_left_update_entry
    m = chem16
    j = 8
    mpo = a2.MPO(ctx, m)
    W = m[j]
    rng = np.random.default_rng(77)
    D = 96
    bra = rng.standard_normal((D, 4, D))
    Hin = rng.standard_normal((D, W.shape[0], D))
    Hin *= np.exp2(np.linspace(-40, 40, W.shape[0]))[None, :, None]
    out = torch.zeros((D, W.shape[3], D), dtype=torch.float64, device="cuda")
    a2.env_update(ctx, mpo, j, 0, dev(Hin), dev(bra), dev(bra), out, prec="f64emu")
    got = host(out, ctx)
    for b, bp in [(0, 0), (5, 77), (95, 3), (40, 40)]:
        ref = env_left_update_entry(Hin, bra, W, bra, b, bp)
        assert rel(got[b, :, bp], ref) < 1e-12
