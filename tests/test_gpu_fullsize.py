"""Full-size parity on sampled outputs: the L=16 chemistry MPO (R up to 562, hand-over
core folded) at the benchmarked bond dimension D = 256, through the same C-ABI calls the
benchmark times (H_eff operator handles, environment updates, truncated SVD).  The
oracle computes the sampled outputs one slice at a time (oracle.env.*_entry) or, for
the SVD, LAPACK's singular values of the same matrix."""
import numpy as np
import pytest

from oracle.env import env_left_update_entry, heff_apply_entry
from synthetic import chemistry_integrals, chemistry_mpo, random_tt_cores

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_23429_gb300 as a2  # noqa: E402
from gpu_common import dev, host  # noqa: E402

D = 256
SAMPLES = [(0, 0), (17, 255), (128, 3), (255, 130), (77, 77)]
# FP32-class arithmetic (FP32 SIMT, or split BF16 products with FP32 sums): one output of
# H_eff at D = 256 sums ~1e6 signed products, so rounding at eps32 = 6e-8 leaves an error
# of order eps32 * sqrt(1e6) relative to the output scale.
TOL32 = 6e-8 * 1e3


@pytest.fixture(scope="module")
def ctx():
    c = a2.Context(0)
    yield c
    assert a2.device_error(c) == 0
    c.close()


@pytest.fixture(scope="module")
def chem16(ctx):
    h, eri = chemistry_integrals(16, 2505)
    m = chemistry_mpo(h, eri)
    return m, a2.MPO(ctx, m)


def _scaled_err(got, ref, scale):
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / scale)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("f64emu", 1e-12), ("fp32", TOL32),
                                      ("f32emu", TOL32), ("bf16", 3e-2)])
@pytest.mark.parametrize("k", [5, 7, 8])
def test_heff_full_size_sampled(ctx, chem16, prec, tol, k):
    """Bond 5: a typical middle bond; 7 / 8: the hand-over core on the right / left
    (identity-block fold active).  Errors are measured against the RMS of the output."""
    m, mpo = chem16
    rng = np.random.default_rng(1000 + k)
    Lh = rng.standard_normal((D, m[k].shape[0], D)) / np.sqrt(D)
    Rh = rng.standard_normal((D, m[k + 1].shape[3], D)) / np.sqrt(D)
    x = rng.standard_normal((D, 4, 4, D))
    op = a2.HeffOp(ctx, mpo, k, dev(Lh), dev(Rh), prec=prec)
    xd = dev(x)
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    op.apply(xd, y)
    yh = host(y, ctx)
    op.close()
    assert np.all(np.isfinite(yh))
    scale = float(np.sqrt(np.mean(yh ** 2)))
    for a, b in SAMPLES:
        ref = heff_apply_entry(Lh, m[k], m[k + 1], Rh, x, a, b)
        assert _scaled_err(yh[a, :, :, b], ref, scale) < tol, (a, b)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", TOL32), ("f32emu", TOL32)])
@pytest.mark.parametrize("j", [5, 8])
def test_env_update_full_size_sampled(ctx, chem16, prec, tol, j):
    m, mpo = chem16
    W = m[j]
    rng = np.random.default_rng(2000 + j)
    Hin = rng.standard_normal((D, W.shape[0], D)) / np.sqrt(D)
    bra = rng.standard_normal((D, 4, D)) / np.sqrt(D)
    ket = rng.standard_normal((D, 4, D)) / np.sqrt(D)
    out = torch.zeros((D, W.shape[3], D), dtype=torch.float64, device="cuda")
    a2.env_update(ctx, mpo, j, 0, dev(Hin), dev(bra), dev(ket), out, prec=prec)
    oh = host(out, ctx)
    assert np.all(np.isfinite(oh))
    scale = float(np.sqrt(np.mean(oh ** 2)))
    for b, bp in SAMPLES:
        ref = env_left_update_entry(Hin, bra, W, ket, b, bp)
        assert _scaled_err(oh[b, :, bp], ref, scale) < tol, (b, bp)


def test_svd_split_full_size(ctx):
    """The two-site split at D = 256 of a 1024 x 1024 matrix with a slowly decaying
    spectrum (the regime of the chemistry workload): kept rank, discarded weight and
    reconstruction against LAPACK's singular values of the same matrix."""
    rng = np.random.default_rng(7)
    n = 1024
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = 1.0 / (1.0 + np.arange(n)) ** 0.75
    M = (U * sig) @ V.T
    s = np.linalg.svd(M, compute_uv=False)
    x = dev(M.reshape(D, 4, 4, D))
    kmax = n
    P = torch.zeros((n, kmax), dtype=torch.float64, device="cuda")
    SQ = torch.zeros((kmax, n), dtype=torch.float64, device="cuda")
    r, disc = a2.svd_split(ctx, x, D, 1e-6, P, SQ)
    assert r == D
    assert abs(disc - np.sqrt(np.sum(s[D:] ** 2))) < 1e-10 * np.linalg.norm(s)
    Ph = host(P, ctx).ravel()[: n * r].reshape(n, r)        # [Dl n1][r], row stride r
    SQh = host(SQ, ctx).ravel()[: r * n].reshape(r, n)      # [r][n2 Dr]
    assert np.abs(Ph.T @ Ph - np.eye(r)).max() < 1e-12
    assert np.allclose(np.linalg.svd(SQh, compute_uv=False), s[:r], rtol=1e-10, atol=1e-13)
    assert abs(np.linalg.norm(M - Ph @ SQh) - disc) < 1e-10 * np.linalg.norm(s)


def test_c2_iterate_energy_matches_oracle_rayleigh_quotient(ctx):
    """The L = 16, D = 256, P = 4 workload itself: six global iterations of the BF16
    default path from the seeded TT (the middle bonds reach the cap of 256); the
    library's FP64-class energy of the iterate (a2_energy with Ozaki-emulated
    environments), and the energy_in the next iteration reports, equal the oracle's FP64
    Rayleigh quotient <x, A x> / <x, x> of the same TT contracted on the host."""
    from oracle.env import sandwich
    from oracle.tt import tt_inner
    from synthetic import get_config
    cfg = get_config("chem_L16_D256")
    h, eri = chemistry_integrals(cfg["L"], cfg["seed_int"])
    m = chemistry_mpo(h, eri)
    mpo = a2.MPO(ctx, m)
    t = a2.TT.from_cores(ctx, random_tt_cores([4] * cfg["L"], cfg["r0"], cfg["seed_tt"]))
    t.left_orthogonalize()
    kw = dict(partition=cfg["partition"], D_max=cfg["D"], prec="bf16", svd_tol=1e-6,
              eig_tol=1e-6, coarse_eps=1e-10, max_restarts=50, sequential=True)
    for _ in range(6):
        a2.additive_sweep(ctx, t, mpo, cfg["P"], **kw)
    cores = t.cores()
    assert max(c.shape[2] for c in cores) == cfg["D"]
    E_gpu, _ = a2.energy(ctx, t, mpo, "f64emu")
    E_or = sandwich(cores, m, cores) / tt_inner(cores, cores)
    assert abs(E_gpu - E_or) < 1e-10 * abs(E_or)
    rep = a2.additive_sweep(ctx, t, mpo, cfg["P"], **kw)
    assert abs(rep["energy_in"] - E_or) < 1e-10 * abs(E_or)
