"""GPU parity of the kernel-level entry points against the oracle (C-ABI calls)."""
import numpy as np
import pytest

from oracle.coarse import coarse_solve as oracle_coarse
from oracle.env import env_left_update, env_right_update, heff_apply as oracle_heff
from oracle.tt import left_orthogonalize, tt_full
from synthetic import chemistry_integrals, chemistry_mpo, heisenberg_mpo, random_tt_cores

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_23429_gb300 as a2  # noqa: E402
from gpu_common import dev, host, rel  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 2e-5, "bf16": 3e-2, "f32emu": 5e-6}


@pytest.fixture(scope="module")
def ctx():
    c = a2.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def chem6():
    h, eri = chemistry_integrals(6, 2505)
    return chemistry_mpo(h, eri)


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,Dl,Dr", [(0, 1, 7), (2, 9, 13), (4, 16, 1), (3, 33, 65)])
def test_heff_chemistry(ctx, chem6, prec, k, Dl, Dr):
    mpo = a2.MPO(ctx, chem6)
    W1, W2 = chem6[k], chem6[k + 1]
    Lh = _rand((Dl, W1.shape[0], Dl), 1)
    Rh = _rand((Dr, W2.shape[3], Dr), 2)
    x = _rand((Dl, 4, 4, Dr), 3)
    ref = oracle_heff(Lh, W1, W2, Rh, x)
    y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
    a2.heff_apply(ctx, mpo, k, dev(Lh), dev(Rh), dev(x), y, prec=prec)
    assert rel(host(y, ctx), ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_heff_heisenberg_ragged(ctx, prec):
    m = heisenberg_mpo(12)
    mpo = a2.MPO(ctx, m)
    for k, Dl, Dr in [(0, 1, 31), (5, 32, 32), (10, 29, 1), (7, 130, 67)]:
        Lh = _rand((Dl, m[k].shape[0], Dl), k)
        Rh = _rand((Dr, m[k + 1].shape[3], Dr), k + 1)
        x = _rand((Dl, 2, 2, Dr), k + 2)
        ref = oracle_heff(Lh, m[k], m[k + 1], Rh, x)
        y = torch.zeros(x.shape, dtype=torch.float64, device="cuda")
        a2.heff_apply(ctx, mpo, k, dev(Lh), dev(Rh), dev(x), y, prec=prec)
        assert rel(host(y, ctx), ref) < TOL[prec], (k, Dl, Dr)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f32emu"])
@pytest.mark.parametrize("j", [0, 2, 5])
def test_env_updates_mixed(ctx, chem6, prec, j):
    mpo = a2.MPO(ctx, chem6)
    W = chem6[j]
    Dlb, Drb, Dlk, Drk = (1 if j == 0 else 11), (1 if j == 5 else 9), (1 if j == 0 else 7), (1 if j == 5 else 12)
    bra = _rand((Dlb, 4, Drb), 5)
    ket = _rand((Dlk, 4, Drk), 6)
    Hin = _rand((Dlb, W.shape[0], Dlk), 7)
    ref = env_left_update(Hin, bra, W, ket)
    out = torch.zeros(ref.shape, dtype=torch.float64, device="cuda")
    a2.env_update(ctx, mpo, j, 0, dev(Hin), dev(bra), dev(ket), out, prec=prec)
    assert rel(host(out, ctx), ref) < TOL[prec]
    Hr = _rand((Drb, W.shape[3], Drk), 8)
    ref = env_right_update(Hr, bra, W, ket)
    out = torch.zeros(ref.shape, dtype=torch.float64, device="cuda")
    a2.env_update(ctx, mpo, j, 1, dev(Hr), dev(bra), dev(ket), out, prec=prec)
    assert rel(host(out, ctx), ref) < TOL[prec]


@pytest.mark.parametrize("shape,D,tol", [((4, 2, 2, 4), 100, 1e-14), ((8, 4, 4, 8), 10, 1e-3),
                                         ((16, 2, 2, 3), 100, 1e-8), ((1, 4, 4, 64), 7, 0.0)])
def test_svd_split(ctx, shape, D, tol):
    rng = np.random.default_rng(11)
    # graded spectrum so that the truncation rule is exercised
    m, n = shape[0] * shape[1], shape[2] * shape[3]
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    k = min(m, n)
    s = 10.0 ** (-np.arange(k) * 0.7)
    M = (U[:, :k] * s) @ V[:k]
    Pd = torch.zeros(m * k, dtype=torch.float64, device="cuda")
    SQd = torch.zeros(k * n, dtype=torch.float64, device="cuda")
    r, disc = a2.svd_split(ctx, dev(M.reshape(shape)), D, tol, Pd, SQd)
    from oracle.tt import svd_split as osvd
    P0, s0, Q0, d0 = osvd(M, D, tol)
    assert r == len(s0)
    P = host(Pd)[: m * r].reshape(m, r)
    SQ = host(SQd)[: r * n].reshape(r, n)
    assert np.allclose(P.T @ P, np.eye(r), atol=1e-12)
    best = (P0 * s0) @ Q0
    assert np.linalg.norm(P @ SQ - best) < 1e-10 * np.linalg.norm(M)
    assert abs(disc - d0) < 1e-10 * np.linalg.norm(s)


def test_coarse_solve_matches_oracle_and_eigh(ctx):
    import scipy.linalg
    rng = np.random.default_rng(0)
    for m in (1, 3, 5, 9, 17):
        B = rng.standard_normal((m, m))
        S = B @ B.T + m * np.eye(m)
        A = rng.standard_normal((m, m))
        A = A + A.T
        c, lam, p = a2.coarse_solve(ctx, A, S, 1e-10)
        c0, lam0, p0 = oracle_coarse(A, S, 1e-10)
        w = scipy.linalg.eigh(A, S, eigvals_only=True)[0]
        assert p == p0 == m
        assert abs(lam - w) < 1e-11 * max(1, abs(w)) and abs(lam - lam0) < 1e-11 * max(1, abs(w))
        assert np.allclose(c, c0, atol=1e-9)
    Y = rng.standard_normal((40, 4))
    Y = np.concatenate([Y, Y[:, :1], Y[:, 1:2] * 2.0], axis=1)   # rank deficient
    H = rng.standard_normal((40, 40))
    H = H + H.T
    c, lam, p = a2.coarse_solve(ctx, Y.T @ H @ Y, Y.T @ Y, 1e-10)
    c0, lam0, p0 = oracle_coarse(Y.T @ H @ Y, Y.T @ Y, 1e-10)
    assert p == p0 == 4 and abs(lam - lam0) < 1e-10


def test_tt_create_left_orthogonal(ctx):
    phys = [2] * 9
    cores = random_tt_cores(phys, 6, 42)
    t = a2.TT.from_cores(ctx, cores)
    nrm = t.left_orthogonalize()
    got = t.cores()
    full = tt_full(cores)
    assert abs(nrm - np.linalg.norm(full)) < 1e-12 * nrm
    assert np.allclose(tt_full(got), full / np.linalg.norm(full), atol=1e-13)
    for c in got[:-1]:
        M = c.reshape(-1, c.shape[2])
        assert np.allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-13)
    # seeded constructor: same generator stream as synthetic.random_tt_cores
    t2 = a2.TT.random(ctx, phys, [6] * 8, 42)
    assert np.allclose(tt_full(t2.cores()), full / np.linalg.norm(full), atol=1e-13)
