"""Adjoint (reverse-mode derivative) of the rank-k truncated SVD, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper does not differentiate the SVD.  This follows the truncated-SVD
adjoint of J. Townsend, "Differentiating the Singular Value Decomposition"
(2016): for A ~ U diag(S) V^T (U m x k, V n x k orthonormal, distinct
positive S) and cotangents dU, dS, dV of a loss,

  F_ij = 1 / (S_j^2 - S_i^2) for i != j, F_ii = 0
  J = F o (U^T dU - dU^T U),   K = F o (V^T dV - dV^T V)
  M = J diag(S) + diag(dS) + diag(S) K
  dA = U M V^T + (I - U U^T) dU diag(S)^-1 V^T + U diag(S)^-1 dV^T (I - V V^T)

where o is the elementwise product.  The GPU path evaluates the same formula
as one rank-2k product [U | P] [R | V]^T.

The projector terms treat the discarded part of the spectrum as zero, so the
formula is the exact derivative of a loss of (U, S, V) when A has rank k, or
when k = min(m, n) (thin SVD).  For a full-rank A truncated at k < min(m, n)
the exact derivative also couples the kept singular pairs with the discarded
ones; ``exact_truncated_gradient`` evaluates it through the thin SVD with the
cotangents of the discarded pairs set to zero.
"""

from __future__ import annotations

import numpy as np


def svd_adjoint(U, S, V, dU=None, dS=None, dV=None):
    """dA for the truncated SVD (U, S, V) and cotangents (dU, dS, dV), any of which may be None."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    m, k = U.shape
    n = V.shape[0]
    dU = np.zeros((m, k)) if dU is None else np.asarray(dU, dtype=np.float64)
    dV = np.zeros((n, k)) if dV is None else np.asarray(dV, dtype=np.float64)
    dS = np.zeros(k) if dS is None else np.asarray(dS, dtype=np.float64)
    s2 = S * S
    diff = s2[None, :] - s2[:, None]          # (i, j) -> S_j^2 - S_i^2
    F = np.zeros((k, k))
    off = ~np.eye(k, dtype=bool)
    F[off] = 1.0 / diff[off]
    UtdU = U.T @ dU
    VtdV = V.T @ dV
    J = F * (UtdU - UtdU.T)
    K = F * (VtdV - VtdV.T)
    M = J * S[None, :] + np.diag(dS) + S[:, None] * K
    Sinv = 1.0 / S
    term1 = U @ M @ V.T
    term2 = ((dU - U @ UtdU) * Sinv[None, :]) @ V.T
    term3 = (U * Sinv[None, :]) @ (dV - V @ VtdV).T
    return term1 + term2 + term3


def exact_truncated_gradient(A, k, dU=None, dS=None, dV=None, thin_svd=None):
    """Exact dA of a loss of the top-k singular triplets of a full-rank A.

    The thin SVD (k' = min(m, n)) is differentiated with the formula above,
    which is exact for it, after padding the cotangents of the pairs k..k'-1
    with zeros.  ``thin_svd`` may supply (U, S, V) of A's thin SVD (otherwise
    the oracle's Jacobi SVD computes it).
    """
    A = np.asarray(A, dtype=np.float64)
    U, S, V = thin_svd if thin_svd is not None else truncated_svd_exact(A, min(A.shape))
    kk = len(S)
    pad = lambda X, rows: None if X is None else np.concatenate([np.asarray(X, dtype=np.float64),
                                                                 np.zeros((rows, kk - k))], axis=1)
    dUf = pad(dU, A.shape[0])
    dVf = pad(dV, A.shape[1])
    dSf = None if dS is None else np.concatenate([np.asarray(dS, dtype=np.float64), np.zeros(kk - k)])
    return svd_adjoint(U, S, V, dUf, dSf, dVf)


def truncated_svd_exact(A, k):
    """Rank-k truncated SVD of a small matrix by the oracle's one-sided Jacobi."""
    from .rsvd import full_svd
    U, S, V = full_svd(A)
    return U[:, :k], S[:k], V[:, :k]
