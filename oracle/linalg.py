"""Plain FP64 dense linear algebra for the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``apply``           products A X and A^T X in FP64; FP32 entries of A are
                      widened exactly, one block of rows at a time, so an 8 GB
                      FP32 matrix never needs a 16 GB FP64 copy.  numpy's
                      matmul is the library primitive for each block.
* ``householder_qr``  thin QR by Householder reflections, the QR
                      decomposition of Section 2.1 step 3 truncated as in
                      step 4 (Golub & Van Loan, Algorithm 5.2.1).
* ``jacobi_svd``      one-sided (Hestenes) Jacobi SVD with the relative
                      stopping test of Demmel & Veselic (1992), used for the
                      SVD of the small matrix in Section 2.1 step 6.
"""

from __future__ import annotations

import numpy as np

EPS64 = np.finfo(np.float64).eps


class CSR:
    """A sparse m x n matrix in compressed sparse row form (values widened to FP64 on use)."""

    def __init__(self, m, n, rowptr, colidx, val):
        self.m, self.n = int(m), int(n)
        self.rowptr = np.asarray(rowptr, dtype=np.int64)
        self.colidx = np.asarray(colidx, dtype=np.int64)
        self.val = np.asarray(val)

    @property
    def shape(self):
        return (self.m, self.n)


def csr_apply(A: CSR, X, trans: bool = False) -> np.ndarray:
    """A @ X or A.T @ X for a CSR matrix, FP64 (scipy's sparse product as the library primitive)."""
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val.astype(np.float64), A.colidx, A.rowptr), shape=(A.m, A.n))
    X = np.asarray(X, dtype=np.float64)
    return np.asarray((M.T @ X) if trans else (M @ X))


def apply(A, X, trans: bool = False, block_rows: int = 4096) -> np.ndarray:
    """Return A @ X (trans=False) or A.T @ X (trans=True) in FP64.

    A is a dense array or a CSR.  For a dense A with trans=True the partial
    products of the row blocks are added in increasing block order.
    """
    if isinstance(A, CSR):
        return csr_apply(A, X, trans)
    X = np.asarray(X, dtype=np.float64)
    m, n = A.shape
    if not trans:
        assert X.shape[0] == n
        out = np.empty((m, X.shape[1]), dtype=np.float64)
        for i0 in range(0, m, block_rows):
            i1 = min(m, i0 + block_rows)
            out[i0:i1] = np.asarray(A[i0:i1], dtype=np.float64) @ X
        return out
    assert X.shape[0] == m
    out = np.zeros((n, X.shape[1]), dtype=np.float64)
    for i0 in range(0, m, block_rows):
        i1 = min(m, i0 + block_rows)
        out += np.asarray(A[i0:i1], dtype=np.float64).T @ X[i0:i1]
    return out


def householder_qr(Y):
    """Thin QR of an m x r matrix (m >= r): Y = Q R, Q^T Q = I_r, R upper triangular.

    Reflector j maps column j of the trailing block onto alpha*e_1 with
    alpha = -sign(x_0)*||x|| (sign(0) taken as +1); a zero column is left
    unreflected.  Q is formed by applying the reflectors in reverse order to
    the first r columns of the identity.
    """
    A = np.array(Y, dtype=np.float64, copy=True)
    m, r = A.shape
    if m < r:
        raise ValueError("householder_qr needs m >= r")
    vs = []
    for j in range(r):
        x = A[j:, j]
        nx = np.linalg.norm(x)
        if nx == 0.0:
            vs.append(None)
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv == 0.0:
            vs.append(None)
            continue
        v /= nv
        A[j:, j:] -= 2.0 * np.outer(v, v @ A[j:, j:])
        vs.append(v)
    R = np.triu(A[:r, :])
    Q = np.zeros((m, r), dtype=np.float64)
    Q[:r, :r] = np.eye(r)
    for j in reversed(range(r)):
        v = vs[j]
        if v is None:
            continue
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    return Q, R


def round_robin_rounds(c: int):
    """Pairings of c column indices into disjoint pairs, c-1 rounds (c even) per sweep.

    Circle method: position 0 stays, positions 1..c'-1 rotate by one after each
    round; pair i of a round is (pos[i], pos[c'-1-i]).  An odd c gets a dummy
    index -1 whose pairs are dropped.
    """
    pos = list(range(c)) + ([-1] if c % 2 else [])
    cp = len(pos)
    rounds = []
    for _ in range(cp - 1):
        pairs = [(pos[i], pos[cp - 1 - i]) for i in range(cp // 2)]
        pairs = [(min(a, b), max(a, b)) for a, b in pairs if a >= 0 and b >= 0]
        rounds.append(pairs)
        pos = [pos[0], pos[-1]] + pos[1:-1]
    return rounds


def jacobi_svd(M, tol: float | None = None, max_sweeps: int = 80):
    """One-sided Jacobi SVD of a rows x c matrix M: M W = U diag(sigma).

    Each rotation makes a column pair (p, q) orthogonal.  With alpha = |m_p|^2,
    beta = |m_q|^2, gamma = m_p^T m_q, the pair is rotated when
    |gamma| > tol*sqrt(alpha*beta) (Demmel & Veselic) and neither column has
    fallen to rounding level (norm^2 <= (max(rows,c)*eps*||M||_F)^2); zeta = (beta-alpha)/(2 gamma),
    t = sign(zeta)/(|zeta| + sqrt(1+zeta^2)), c = 1/sqrt(1+t^2), s = c t,
    m_p <- c m_p - s m_q, m_q <- s m_p + c m_q, and the same for the columns of
    W.  Sweeps visit all pairs in round-robin order (the pairs of one round are
    disjoint, so their rotations commute) until a sweep rotates nothing.

    Returns (U, sigma, W, sweeps) with sigma sorted in descending order (stable
    for ties) and U's columns the normalised columns of M W (a zero column
    of M W gives a zero column of U).
    """
    M = np.array(M, dtype=np.float64, copy=True)
    rows, c = M.shape
    W = np.eye(c)
    if tol is None:
        tol = max(c, 1) * EPS64
    rounds = round_robin_rounds(c)
    # columns whose norm has fallen to rounding level of ||M||_F are treated as
    # exact zeros (a wide or rank-deficient M would otherwise keep rotating noise)
    zero2 = (max(rows, c, 1) * EPS64 * np.linalg.norm(M)) ** 2
    sweeps = 0
    for sweep in range(max_sweeps):
        rotated = False
        for pairs in rounds:
            if not pairs:
                continue
            P = np.array([a for a, _ in pairs])
            Qi = np.array([b for _, b in pairs])
            mp = M[:, P]
            mq = M[:, Qi]
            alpha = np.einsum("ij,ij->j", mp, mp)
            beta = np.einsum("ij,ij->j", mq, mq)
            gamma = np.einsum("ij,ij->j", mp, mq)
            need = (np.abs(gamma) > tol * np.sqrt(alpha * beta)) & (alpha > zero2) & (beta > zero2)
            if not np.any(need):
                continue
            rotated = True
            P, Qi = P[need], Qi[need]
            alpha, beta, gamma = alpha[need], beta[need], gamma[need]
            zeta = (beta - alpha) / (2.0 * gamma)
            sgn = np.where(zeta >= 0, 1.0, -1.0)
            t = sgn / (np.abs(zeta) + np.hypot(1.0, zeta))
            cs = 1.0 / np.sqrt(1.0 + t * t)
            sn = cs * t
            mp = M[:, P]
            mq = M[:, Qi]
            M[:, P] = cs * mp - sn * mq
            M[:, Qi] = sn * mp + cs * mq
            wp = W[:, P]
            wq = W[:, Qi]
            W[:, P] = cs * wp - sn * wq
            W[:, Qi] = sn * wp + cs * wq
        sweeps = sweep + 1
        if not rotated:
            break
    else:
        raise RuntimeError("one-sided Jacobi did not converge")
    sigma = np.sqrt(np.einsum("ij,ij->j", M, M))
    order = np.argsort(-sigma, kind="stable")
    sigma = sigma[order]
    M = M[:, order]
    W = W[:, order]
    U = np.zeros_like(M)
    nz = sigma > 0
    U[:, nz] = M[:, nz] / sigma[nz]
    return U, sigma, W, sweeps


def normalise_signs(U, V):
    """Flip each pair (u_i, v_i) so that the largest-magnitude entry of u_i is
    positive; among entries of equal magnitude the lowest row index decides."""
    U = np.array(U, dtype=np.float64, copy=True)
    V = np.array(V, dtype=np.float64, copy=True)
    if U.shape[0] == 0:
        return U, V
    idx = np.argmax(np.abs(U), axis=0)  # first occurrence of the maximum
    s = np.sign(U[idx, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return U * s, V * s
