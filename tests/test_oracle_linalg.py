"""Pins for the oracle's products, Householder QR and one-sided Jacobi SVD."""

import itertools

import numpy as np
import pytest

from oracle import linalg as L

EPS = np.finfo(np.float64).eps


def test_apply_exact_on_small_integers():
    rng = np.random.default_rng(0)
    A = rng.integers(-5, 6, size=(37, 23)).astype(np.float32)
    X = rng.integers(-4, 5, size=(23, 6)).astype(np.float64)
    Yt = rng.integers(-4, 5, size=(37, 6)).astype(np.float64)
    ref = [[sum(int(A[i, t]) * int(X[t, j]) for t in range(23)) for j in range(6)] for i in range(37)]
    assert np.array_equal(L.apply(A, X, block_rows=8), np.array(ref, dtype=np.float64))
    reft = [[sum(int(A[t, i]) * int(Yt[t, j]) for t in range(37)) for j in range(6)] for i in range(23)]
    assert np.array_equal(L.apply(A, Yt, trans=True, block_rows=5), np.array(reft, dtype=np.float64))


@pytest.mark.parametrize("m,r", [(50, 7), (7, 7), (300, 40), (1, 1)])
def test_householder_qr_factorises(m, r):
    rng = np.random.default_rng(m * 31 + r)
    Y = rng.standard_normal((m, r)) * np.logspace(0, -6, r)
    Q, R = L.householder_qr(Y)
    assert np.allclose(np.tril(R, -1), 0)
    assert np.linalg.norm(Q.T @ Q - np.eye(r)) <= 10 * r * EPS * 10
    assert np.linalg.norm(Q @ R - Y) <= 10 * r * EPS * np.linalg.norm(Y) * 10
    # |diag R| equals the Cholesky factor of Y^T Y (library comparator)
    C = np.linalg.cholesky(Y.T @ Y)
    assert np.allclose(np.abs(np.diag(R)), np.diag(C), rtol=1e-6)


def test_householder_qr_rank_deficient():
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((20, 5))
    Y[:, 2] = 0.0
    Q, R = L.householder_qr(Y)
    assert np.linalg.norm(Q @ R - Y) < 1e-13
    assert np.linalg.norm(Q.T @ Q - np.eye(5)) < 1e-13


def test_round_robin_covers_every_pair_once():
    for c in (1, 2, 3, 8, 11, 30):
        rounds = L.round_robin_rounds(c)
        seen = []
        for pairs in rounds:
            idx = [i for p in pairs for i in p]
            assert len(idx) == len(set(idx))  # disjoint within a round
            seen += pairs
        assert sorted(seen) == sorted(itertools.combinations(range(c), 2))


@pytest.mark.parametrize("rows,c", [(3, 3), (8, 5), (5, 8), (2, 2), (8, 8), (6, 1)])
def test_jacobi_matches_library_svd_on_tiny_inputs(rows, c):
    rng = np.random.default_rng(rows * 10 + c)
    M = rng.standard_normal((rows, c))
    U, s, W, _ = L.jacobi_svd(M)
    ref = np.linalg.svd(M, compute_uv=False)
    t = min(rows, c)
    assert np.allclose(s[:t], ref, rtol=1e-13, atol=1e-14)
    assert np.allclose(s[t:], 0, atol=1e-13)
    assert np.linalg.norm(W.T @ W - np.eye(c)) < 1e-13
    assert np.linalg.norm(M @ W - U * s) < 1e-13 * max(1, s[0])
    # squared singular values are the eigenvalues of M^T M
    ev = np.sort(np.linalg.eigvalsh(M.T @ M))[::-1]
    assert np.allclose(s ** 2, np.clip(ev, 0, None), atol=1e-12)


def test_jacobi_closed_forms():
    # permuted diagonal: singular values are |d| sorted
    d = np.array([0.5, -3.0, 2.0, 1e-3])
    P = np.eye(4)[[2, 0, 3, 1]]
    _, s, _, sweeps = L.jacobi_svd(P @ np.diag(d))
    assert np.array_equal(s, np.sort(np.abs(d))[::-1])
    assert sweeps == 1  # orthogonal columns: nothing to rotate
    # 2x2: sigma_1 sigma_2 = |det|, sigma_1^2 + sigma_2^2 = ||M||_F^2
    M = np.array([[3.0, 1.0], [2.0, -4.0]])
    _, s, _, _ = L.jacobi_svd(M)
    assert np.isclose(s[0] * s[1], abs(np.linalg.det(M)), rtol=1e-14)
    assert np.isclose((s ** 2).sum(), (M ** 2).sum(), rtol=1e-14)
    # rotation of the identity's columns by angle a: singular values are 1, 1
    a = 0.3
    Rm = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    _, s, _, _ = L.jacobi_svd(Rm)
    assert np.allclose(s, 1.0, rtol=1e-15)


def test_jacobi_high_relative_accuracy_graded():
    """One-sided Jacobi keeps tiny singular values of a graded matrix to high relative accuracy."""
    rng = np.random.default_rng(11)
    Q1, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    Q2, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    s = np.logspace(0, -10, 12)
    M = (Q1 * s) @ Q2.T
    _, got, _, _ = L.jacobi_svd(M)
    assert np.max(np.abs(got - s) / s) < 1e-5  # far below what sigma_1*eps/sigma_i would allow


def test_normalise_signs_rule():
    U = np.array([[0.1, -0.5], [-0.7, 0.5], [0.2, 0.1]])
    V = np.array([[1.0, 2.0]])
    Un, Vn = L.normalise_signs(U, V)
    assert np.array_equal(Un[:, 0], -U[:, 0]) and Vn[0, 0] == -1.0
    # tie |-0.5| = |0.5|: lowest row index (row 0, negative) decides -> flip
    assert np.array_equal(Un[:, 1], -U[:, 1]) and Vn[0, 1] == -2.0
