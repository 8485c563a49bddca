"""The library's own dense factorisations against the oracle and LAPACK (C-ABI calls):
the Householder LQ of Alg. 2 step 1 and of the TT rounding, with diag(L) >= 0 (unique for
full-rank M), on wide, square, tall, ragged, graded and rank-deficient matrices up to the
compression's largest shape at D = 256; the truncated SVD of Alg. 1 step 2
(bidiagonalisation, bisection, inverse iteration) with tolerances down to 1e-10 on
spectra down to 1e-12, degenerate multiplets and edge cases."""
import numpy as np
import pytest

from oracle.tt import lq_pos

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_23429_gb300 as a2  # noqa: E402
from gpu_common import dev, host  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = a2.Context(0)
    yield c
    assert a2.device_error(c) == 0
    c.close()


def _lq(ctx, M):
    rows, cols = M.shape
    k = min(rows, cols)
    L = torch.full((rows, k), float("nan"), dtype=torch.float64, device="cuda")
    Q = torch.full((k, cols), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    a2.lq(ctx, dev(M), L, Q)
    return host(L, ctx), host(Q, ctx)


@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 7), (5, 1), (3, 8), (8, 8), (13, 5),
                                       (32, 64), (100, 37), (256, 1024), (129, 515)])
def test_lq_matches_oracle(ctx, rows, cols):
    rng = np.random.default_rng(rows * 1000 + cols)
    M = rng.standard_normal((rows, cols))
    L, Q = _lq(ctx, M)
    L0, Q0 = lq_pos(M)
    k = min(rows, cols)
    scale = np.abs(M).max()
    assert np.abs(L - L0).max() < 1e-12 * scale * k
    assert np.abs(Q - Q0).max() < 1e-11 * k
    assert np.all(np.diag(L[:k]) >= 0.0)
    assert np.abs(np.tril(L[:k, :k]) - L[:k, :k]).max() == 0.0
    assert np.abs(Q @ Q.T - np.eye(k)).max() < 1e-13 * k


def test_lq_graded_rows(ctx):
    """Rows scaled over 1 .. 1e-12 (a truncated TT core's spectrum)."""
    rng = np.random.default_rng(5)
    M = rng.standard_normal((64, 256)) * np.logspace(0, -12, 64)[:, None]
    L, Q = _lq(ctx, M)
    assert np.abs(L @ Q - M).max() < 1e-14
    assert np.abs(Q @ Q.T - np.eye(64)).max() < 1e-13
    L0, _ = lq_pos(M)
    assert np.allclose(np.diag(L), np.diag(L0), rtol=1e-8, atol=1e-28)


def test_lq_rank_deficient_and_large(ctx):
    """The compression's TT sum has linearly dependent rows (bond 2D + D~ > its rank): L Q
    still reproduces M and Q keeps orthonormal rows.  768 x 3072 is the largest core of
    the compression at D = 256."""
    rng = np.random.default_rng(9)
    B = rng.standard_normal((256, 3072))
    C = rng.standard_normal((768, 256))
    M = C @ B / 16.0                                  # rank 256, 768 rows
    L, Q = _lq(ctx, M)
    assert np.abs(L @ Q - M).max() < 1e-12 * np.abs(M).max()
    assert np.abs(Q @ Q.T - np.eye(768)).max() < 1e-12
    Z = np.zeros((4, 9))
    Lz, Qz = _lq(ctx, Z)
    assert np.abs(Lz).max() == 0.0 and np.abs(Qz @ Qz.T - np.eye(4)).max() < 1e-15


def _svd(ctx, M, D, tol, shape=None):
    rows, cols = M.shape
    shape = shape or (rows, 1, 1, cols)
    k = min(rows, cols)
    P = torch.zeros(rows * k, dtype=torch.float64, device="cuda")
    SQ = torch.zeros(k * cols, dtype=torch.float64, device="cuda")
    r, disc = a2.svd_split(ctx, dev(M.reshape(shape)), D, tol, P, SQ)
    return r, disc, host(P, ctx)[: rows * r].reshape(rows, r), host(SQ)[: r * cols].reshape(r, cols)


def _spectrum_matrix(rows, cols, sig, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((rows, rows)))
    V, _ = np.linalg.qr(rng.standard_normal((cols, cols)))
    k = len(sig)
    return (U[:, :k] * sig) @ V[:, :k].T


@pytest.mark.parametrize("rows,cols", [(64, 64), (256, 128), (96, 300)])
def test_svd_tol_1e10_spectrum_to_1e12(ctx, rows, cols):
    """svd_tol = 1e-10 on a spectrum decaying from 1 to 1e-12: the rank the truncation
    rule picks, the discarded weight and the truncated product agree with LAPACK's SVD of
    the same matrix (a Gram-matrix eigensolver would see only singular values above
    ~1e-8 here)."""
    from oracle.tt import svd_split as osvd
    k = min(rows, cols)
    sig = np.logspace(0, -12, k)
    M = _spectrum_matrix(rows, cols, sig, rows + cols)
    r, disc, P, SQ = _svd(ctx, M, k, 1e-10)
    P0, s0, Q0, d0 = osvd(M, k, 1e-10)
    assert r == len(s0)
    s = np.linalg.svd(M, compute_uv=False)
    assert abs(disc - np.sqrt(np.sum(s[r:] ** 2))) < 1e-3 * np.sqrt(np.sum(s[r:] ** 2)) + 1e-16
    assert np.abs(P.T @ P - np.eye(r)).max() < 1e-12
    assert np.linalg.norm(P @ SQ - (P0 * s0) @ Q0) < 1e-12 * np.linalg.norm(s)
    assert np.allclose(np.linalg.svd(SQ, compute_uv=False), s[:r], rtol=1e-9, atol=1e-15)


def test_svd_degenerate_singular_values(ctx):
    """Exactly degenerate multiplets (spin-degenerate Schmidt values): the kept left
    subspace equals LAPACK's (any basis of a multiplet is a valid set of singular
    vectors), the kept columns are orthonormal."""
    sig = np.repeat([1.0, 0.5, 0.5, 0.25, 0.1, 1e-3], [1, 3, 1, 4, 6, 9])[:24]
    M = _spectrum_matrix(48, 40, sig, 3)
    r, disc, P, SQ = _svd(ctx, M, 9, 1e-12)        # cut between 0.25 (x4) and 0.1
    assert r == 9
    U = np.linalg.svd(M)[0][:, :9]
    assert np.abs(P.T @ P - np.eye(9)).max() < 1e-12
    assert np.abs(P @ P.T - U @ U.T).max() < 1e-12
    assert abs(disc - np.sqrt(6 * 0.01 + 9 * 1e-6)) < 1e-12


def test_svd_edge_cases(ctx):
    r, disc, P, SQ = _svd(ctx, np.zeros((6, 5)), 4, 1e-8)
    assert r == 1 and disc == 0.0 and np.abs(SQ).max() == 0.0
    M = np.outer(np.arange(1.0, 8.0), np.linspace(-1, 1, 3))
    r, disc, P, SQ = _svd(ctx, M, 3, 1e-12)
    assert r == 1 and disc < 1e-13 * np.linalg.norm(M)
    assert np.abs(P @ SQ - M).max() < 1e-13 * np.abs(M).max()
    r, disc, P, SQ = _svd(ctx, np.array([[3.0]]), 1, 0.0)
    assert r == 1 and abs(abs(P[0, 0]) - 1.0) < 1e-15 and abs(abs(SQ[0, 0]) - 3.0) < 1e-15


def test_svd_large_global_memory_path(ctx):
    """2048 x 1800: too large for the shared-memory-resident bidiagonalisation, so the
    global-memory kernel runs; kept rank, discarded weight and truncated product against
    LAPACK."""
    from oracle.tt import svd_split as osvd
    rows, cols, D = 2048, 1800, 200
    sig = 1.0 / (1.0 + np.arange(cols)) ** 0.8
    M = _spectrum_matrix(rows, cols, sig, 21)
    r, disc, P, SQ = _svd(ctx, M, D, 1e-8)
    P0, s0, Q0, d0 = osvd(M, D, 1e-8)
    assert r == len(s0) == D
    assert abs(disc - d0) < 1e-10 * np.linalg.norm(sig)
    assert np.abs(P.T @ P - np.eye(r)).max() < 1e-12
    assert np.linalg.norm(P @ SQ - (P0 * s0) @ Q0) < 1e-10 * np.linalg.norm(sig)


def test_svd_tall_in_place_back_transformation(ctx):
    """3300 x 40: more rows than the back-transformation keeps in shared memory, so the
    kept columns are updated in place in device memory; rank, discarded weight and
    truncated product against LAPACK.  More than 12800 rows is refused."""
    from oracle.tt import svd_split as osvd
    sig = np.logspace(0, -9, 40)
    M = _spectrum_matrix(3300, 40, sig, 33)
    r, disc, P, SQ = _svd(ctx, M, 30, 1e-7)
    P0, s0, Q0, d0 = osvd(M, 30, 1e-7)
    assert r == len(s0)
    assert abs(disc - d0) < 1e-12
    assert np.abs(P.T @ P - np.eye(r)).max() < 1e-12
    assert np.linalg.norm(P @ SQ - (P0 * s0) @ Q0) < 1e-12
    with pytest.raises(a2.A2Error):
        _svd(ctx, np.ones((12801, 2)), 2, 1e-8)
