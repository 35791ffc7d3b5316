"""Pins for the oracle's SVD adjoint: central finite differences of losses
evaluated through the exact SVD, one loss per cotangent term."""

import numpy as np
import pytest

from oracle import adjoint as AD
from synth import prescribed_dense, spectrum_geometric

LOSSES = ["S", "U", "V", "all"]


def _fd(loss, A, E, h=1e-5):
    return (loss(A + h * E) - loss(A - h * E)) / (2 * h)


def _loss_and_cotangents(which, m, n, k, rng):
    w = rng.uniform(size=k)
    X = rng.standard_normal((m, 3))
    Yv = rng.standard_normal((n, 2))

    def loss_of(U, S, V):
        val = 0.0
        if which in ("S", "all"):
            val += float(w @ S)
        if which in ("U", "all"):
            val += float(np.sum((U.T @ X) ** 2))
        if which in ("V", "all"):
            val += float(np.sum((V.T @ Yv) ** 2))
        return val

    def cot(U, S, V):
        dS = w if which in ("S", "all") else None
        dU = 2 * X @ (X.T @ U) if which in ("U", "all") else None
        dV = 2 * Yv @ (Yv.T @ V) if which in ("V", "all") else None
        return dU, dS, dV

    return loss_of, cot


def _check(A, k, which, grad_fn, seed):
    rng = np.random.default_rng(seed)
    loss_of, cot = _loss_and_cotangents(which, *A.shape, k, rng)
    loss = lambda M: loss_of(*AD.truncated_svd_exact(M, k))
    dA = grad_fn(A, k, *cot(*AD.truncated_svd_exact(A, k)))
    for t in range(4):
        E = rng.standard_normal(A.shape)
        E /= np.linalg.norm(E)
        fd = _fd(loss, A, E)
        an = float(np.sum(dA * E))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (which, t, fd, an)


def _truncated(A, k, dU, dS, dV):
    return AD.svd_adjoint(*AD.truncated_svd_exact(A, k), dU, dS, dV)


@pytest.mark.parametrize("which", LOSSES)
def test_truncated_formula_exact_for_rank_k(which):
    """A of exact rank k: the projector terms are the whole story."""
    k = 6
    s = np.concatenate([10.0 * spectrum_geometric(k, 0.8), np.zeros(16 - k)])
    A, _, _ = prescribed_dense(24, 16, s, 0)
    _check(A, k, which, _truncated, 1)


@pytest.mark.parametrize("which", LOSSES)
def test_thin_formula_exact_for_full_rank(which):
    """k = min(m, n): every pair couples through F."""
    A, _, _ = prescribed_dense(20, 12, 10.0 * spectrum_geometric(12, 0.8), 2)
    _check(A, 12, which, _truncated, 3)


@pytest.mark.parametrize("which", LOSSES)
def test_exact_truncated_gradient_for_full_rank(which):
    """Full-rank A, k < min(m, n): the reference gradient of the GPU comparison."""
    A, _, _ = prescribed_dense(24, 16, 10.0 * spectrum_geometric(16, 0.8), 4)
    _check(A, 6, which, AD.exact_truncated_gradient, 5)


def test_truncated_formula_differs_from_exact_when_tail_is_nonzero():
    A, _, _ = prescribed_dense(24, 16, 10.0 * spectrum_geometric(16, 0.8), 6)
    k = 6
    U, S, V = AD.truncated_svd_exact(A, k)
    rng = np.random.default_rng(7)
    dU = rng.standard_normal(U.shape)
    a = AD.svd_adjoint(U, S, V, dU, None, None)
    b = AD.exact_truncated_gradient(A, k, dU, None, None)
    assert np.linalg.norm(a - b) > 1e-3 * np.linalg.norm(b)


def test_singular_value_gradient_is_u_v_outer():
    """dS only: dA = U diag(dS) V^T exactly (the classical dsigma_i/dA = u_i v_i^T)."""
    A, _, _ = prescribed_dense(12, 9, 10.0 * spectrum_geometric(9, 0.8), 4)
    U, S, V = AD.truncated_svd_exact(A, 4)
    dS = np.array([1.0, -2.0, 0.5, 3.0])
    assert np.allclose(AD.svd_adjoint(U, S, V, None, dS, None), (U * dS) @ V.T, atol=1e-14)
