"""Pins of oracle.tt / oracle.mpo against brute force and linear algebra facts."""
import itertools

import numpy as np
import pytest

from oracle.tt import (left_orthogonalize, right_orthogonalize, tt_add, tt_full,
                       tt_inner, tt_round, truncation_rank, lq_pos, qr_pos)
from synthetic import random_tt_cores


def _brute_full(cores):
    dims = [c.shape[1] for c in cores]
    out = np.zeros(dims)
    for idx in itertools.product(*[range(d) for d in dims]):
        m = np.eye(1)
        for c, x in zip(cores, idx):
            m = m @ c[:, x, :]          # product of slices, Def. TT contraction
        out[idx] = m[0, 0]
    return out.ravel()


def test_tt_full_matches_slice_products():
    cores = random_tt_cores([2, 3, 2, 2], 3, 5)
    assert np.allclose(tt_full(cores), _brute_full(cores), atol=1e-14)


def test_orthogonal_forms_are_orthogonal_and_same_tensor():
    cores = random_tt_cores([2] * 7, 4, 9)
    full = tt_full(cores)
    U = left_orthogonalize(cores)
    V = right_orthogonalize(cores)
    for c in U[:-1]:
        M = c.reshape(-1, c.shape[2])
        assert np.allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-13)
    for c in V[1:]:
        M = c.reshape(c.shape[0], -1)
        assert np.allclose(M @ M.T, np.eye(M.shape[0]), atol=1e-13)
    assert np.allclose(tt_full(U), full, atol=1e-12)
    assert np.allclose(tt_full(V), full, atol=1e-12)
    # ||tau(U)|| = ||last core|| for a left-orthogonal decomposition
    assert np.isclose(np.linalg.norm(U[-1]), np.linalg.norm(full), rtol=1e-13)


def test_qr_lq_sign_convention():
    A = np.random.default_rng(1).standard_normal((6, 4))
    Q, R = qr_pos(A)
    assert np.all(np.diag(R) >= 0) and np.allclose(Q @ R, A)
    L, Q2 = lq_pos(A.T)
    assert np.all(np.diag(L) >= 0) and np.allclose(L @ Q2, A.T)


def test_inner_and_sum():
    a = random_tt_cores([2] * 6, 3, 1)
    b = random_tt_cores([2] * 6, 4, 2)
    assert np.isclose(tt_inner(a, b), tt_full(a) @ tt_full(b), rtol=1e-12)
    s = tt_add([a, b], [0.3, -1.7])
    assert np.allclose(tt_full(s), 0.3 * tt_full(a) - 1.7 * tt_full(b), atol=1e-12)


def test_truncation_rule():
    s = np.array([1.0, 0.1, 0.02, 1e-3])
    r, d = truncation_rank(s, 10, 1e-2)
    # ||s|| = 1.00520; tail after 2 values sqrt(4e-4 + 1e-6) = 0.0200 > 0.0100520,
    # tail after 3 values 1e-3 <= 0.0100520  ->  r = 3, discarded 1e-3
    assert r == 3 and np.isclose(d, 1e-3)
    # boundary: tail exactly below the threshold keeps the smaller rank
    s = np.array([1.0, 0.1, 0.01, 1e-3])
    assert truncation_rank(s, 10, 1e-2)[0] == 2
    assert truncation_rank(s, 2, 0.0)[0] == 2
    assert truncation_rank(s, 10, 0.0)[0] == 4
    assert truncation_rank(np.array([2.0]), 5, 0.5)[0] == 1


def test_round_exact_and_truncated():
    a = random_tt_cores([2] * 6, 4, 3)
    b = random_tt_cores([2] * 6, 4, 4)
    s = tt_add([a, b], [1.0, 1.0])
    r, _ = tt_round(s, 100, 1e-14)
    assert np.allclose(tt_full(r), tt_full(s), atol=1e-12)
    assert max(c.shape[2] for c in r) <= 8
    # two-site tensor: rounding to rank 1 equals the best rank-1 approximation
    M = np.random.default_rng(0).standard_normal((4, 5))
    cores = [M.reshape(1, 4, 5), np.eye(5).reshape(5, 5, 1)]
    r, _ = tt_round(cores, 1, 0.0)
    U, sv, Vt = np.linalg.svd(M)
    assert np.allclose(tt_full(r), (sv[0] * np.outer(U[:, 0], Vt[0])).ravel(), atol=1e-12)
