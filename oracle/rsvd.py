"""Randomized SVD with power iterations, FP64 (Section 2.1 steps 1-7, Section 2.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The steps follow the paper's numbered list in Section 2.1:

 1. O in R^{n x r}, r = k + p, i.i.d. N(0,1)           (``oracle.gaussian``)
 2. Y = A O
 3./4. thin QR of Y, Q_r = its first r columns         (Householder)
 5. B = Q_r^T A, held as its transpose B^T = A^T Q_r   (r x n; the paper's
    "B in R^{m x r}" is read as r x n, and the stage list of Section 4.1
    also forms B^T first)
 6. SVD of B: B^T = Q_b R (Householder), one-sided Jacobi on R^T gives
    R^T W = U_R diag(sigma), hence B = U_R diag(sigma) (Q_b W)^T
 7. U_r = Q_r U_B, V = Q_b W; the top k are returned.

Power iterations (Section 2.2, Eq. (2) and (3)): the sketch (A A^T)^q A O is
evaluated from right to left.  The paper states no re-orthonormalisation
between the products; this oracle orthonormalises after every product,
as in Halko, Martinsson & Tropp (2011), Algorithm 4.4, which is the scheme
the GPU path implements:  Q = orth(A O); q times: Z = orth(A^T Q), Q = orth(A Z).
The singular values returned are those of B = Q^T A, i.e. approximations of
A's own singular values: no (2q+1)-th root is taken.

Sign convention: each pair (u_i, v_i) is flipped so that the largest-magnitude
entry of u_i is positive (lowest row index on ties).
"""

from __future__ import annotations

import numpy as np

from .gaussian import gaussian_matrix_as_f64
from .linalg import apply, householder_qr, jacobi_svd, normalise_signs


def range_finder(A, r: int, q: int, seed: int, omega_dtype: str = "f64"):
    """Q with orthonormal columns spanning (A A^T)^q A O (Section 2.2, Eq. (3))."""
    m, n = A.shape
    O = gaussian_matrix_as_f64(n, r, seed, omega_dtype)
    Q, _ = householder_qr(apply(A, O))
    for _ in range(q):
        Z, _ = householder_qr(apply(A, Q, trans=True))
        Q, _ = householder_qr(apply(A, Z))
    return Q


def range_finder_fused(A, r: int, q: int, seed: int, omega_dtype: str = "f64"):
    """Q spanning the same sketch (A A^T)^q A O as ``range_finder``, with each
    power iteration taken as one sweep Z = A^T (A W) and only the n-side
    orthonormalised (Section 2.2 evaluates the product right to left with no
    re-orthonormalisation; here W = orth(Z) after every sweep, Halko,
    Martinsson & Tropp (2011) Algorithm 4.3 with that step added):
        W = O;  q times: W = orth(A^T (A W));  Q = orth(A W).
    Equal to ``range_finder``'s span in exact arithmetic; in floating point
    the sweep squares the spectrum, so directions below about sqrt(eps) of
    sigma_1 are not resolved.  One read of A per sweep when A (A W) and
    A^T (A W) are formed tile by tile."""
    m, n = A.shape
    W = gaussian_matrix_as_f64(n, r, seed, omega_dtype)
    for _ in range(q):
        W, _ = householder_qr(apply(A, apply(A, W), trans=True))
    Q, _ = householder_qr(apply(A, W))
    return Q


def small_svd_of_bt(Bt):
    """SVD of B from B^T (n x r): returns U_B (r x r), sigma (r), V (n x r)."""
    Qb, R = householder_qr(Bt)
    UR, sigma, W, _ = jacobi_svd(R.T)
    return UR, sigma, Qb @ W


def rsvd(A, k: int, p: int, q: int, seed: int, omega_dtype: str = "f64"):
    """Rank-k randomized SVD of an m x n matrix A (numpy array, FP32 or FP64, or an
    ``oracle.linalg.CSR``).

    Returns (U m x k, S k, V n x k) in FP64 with S descending.
    ``omega_dtype`` rounds O to the working type of the path under test
    ("f64", "f32" or "bf16") before it is used.
    """
    m, n = A.shape
    r = k + p
    if not (1 <= k and 0 <= p and r <= min(m, n) and q >= 0):
        raise ValueError("need 1 <= k, 0 <= p, k + p <= min(m, n), q >= 0")
    Q = range_finder(A, r, q, seed, omega_dtype)
    Bt = apply(A, Q, trans=True)
    UB, sigma, V = small_svd_of_bt(Bt)
    U = Q @ UB[:, :k]
    U, V = normalise_signs(U, V[:, :k])
    return U, sigma[:k], V


def rsvd_fused_sweeps(A, k: int, p: int, q: int, seed: int, omega_dtype: str = "f64"):
    """``rsvd`` with the range finder of ``range_finder_fused`` (steps 5-7 as
    in ``rsvd``)."""
    m, n = A.shape
    r = k + p
    if not (1 <= k and 0 <= p and r <= min(m, n) and q >= 0):
        raise ValueError("need 1 <= k, 0 <= p, k + p <= min(m, n), q >= 0")
    Q = range_finder_fused(A, r, q, seed, omega_dtype)
    Bt = apply(A, Q, trans=True)
    UB, sigma, V = small_svd_of_bt(Bt)
    U = Q @ UB[:, :k]
    U, V = normalise_signs(U, V[:, :k])
    return U, sigma[:k], V


def rsvd_auto_q(A, k: int, p: int, q_max: int, seed: int, tol: float = 1e-3, omega_dtype: str = "f64"):
    """Randomized SVD with the iteration parameter chosen automatically
    (Section 2.2 leaves the rule open: q grows while the estimated spectrum
    still moves by more than a threshold).

    Reading taken: after i power iterations the estimates sigma^(i) are the
    singular values of B_i = Q_i^T A (i = 0, 1, ...); the change
    delta_i = ||sigma^(i)_{1..k} - sigma^(i-1)_{1..k}||_2 / ||sigma^(i)_{1..k}||_2
    is monitored and the iterations stop at the first i >= 1 with delta_i <= tol,
    or at i = q_max.  The basis for the next iteration is the orthonormal
    factor of B_i^T = A^T Q_i (as in ``range_finder``), so no product with A is
    spent on the monitoring.  Returns (U, S, V, q_used); the result equals
    ``rsvd(A, k, p, q_used, seed, omega_dtype)``.
    """
    m, n = A.shape
    r = k + p
    if not (1 <= k and 0 <= p and r <= min(m, n) and q_max >= 0):
        raise ValueError("need 1 <= k, 0 <= p, k + p <= min(m, n), q_max >= 0")
    O = gaussian_matrix_as_f64(n, r, seed, omega_dtype)
    Q, _ = householder_qr(apply(A, O))
    prev = None
    i = 0
    while True:
        Bt = apply(A, Q, trans=True)
        UB, sigma, V = small_svd_of_bt(Bt)
        if prev is not None:
            delta = np.linalg.norm(sigma[:k] - prev[:k]) / np.linalg.norm(sigma[:k])
            if delta <= tol:
                break
        if i == q_max:
            break
        prev = sigma
        Z, _ = householder_qr(Bt)
        Q, _ = householder_qr(apply(A, Z))
        i += 1
    U = Q @ UB[:, :k]
    U, V = normalise_signs(U, V[:, :k])
    return U, sigma[:k], V, i


def full_svd(A):
    """Exact thin SVD of a small dense matrix by one-sided Jacobi.

    m >= n: A W = U diag(s) gives A = U diag(s) W^T.  m < n: the same on A^T.
    Returns (U m x t, S t, V n x t), t = min(m, n), S descending, signs normalised.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if m >= n:
        Qa, R = householder_qr(A)
        UR, s, W, _ = jacobi_svd(R)
        U, V = Qa @ UR, W
    else:
        Qa, R = householder_qr(A.T)
        UR, s, W, _ = jacobi_svd(R)
        U, V = W, Qa @ UR
    U, V = normalise_signs(U, V)
    return U, s, V
