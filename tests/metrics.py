"""Accuracy measures shared by the tests (no method arithmetic)."""

import numpy as np


def max_principal_angle(Ua, Ub) -> float:
    """sin of the largest principal angle between span(Ua) and span(Ub).

    Both inputs have orthonormal columns (up to rounding); the value is
    ||(I - Ub Ub^T) Ua||_2, computed through a re-orthonormalised Ub.
    """
    Ua = np.asarray(Ua, dtype=np.float64)
    Ub = np.asarray(Ub, dtype=np.float64)
    Qb, _ = np.linalg.qr(Ub)
    Qa, _ = np.linalg.qr(Ua)
    resid = Qa - Qb @ (Qb.T @ Qa)
    return float(np.linalg.norm(resid, 2))


def sigma_rel_err(S, S_ref) -> float:
    S = np.asarray(S, dtype=np.float64)
    S_ref = np.asarray(S_ref, dtype=np.float64)
    return float(np.max(np.abs(S - S_ref) / np.abs(S_ref)))


def cluster_safe_angles(U, U_ref, S_ref, k, rel_gap=1e-8):
    """Largest principal angle between leading subspaces, cut where S_ref has no cluster.

    Returns the angle between the first k' columns, k' <= k the largest index
    whose sigma is separated from the next one by more than ``rel_gap``.
    """
    kk = k
    while kk > 1 and kk < len(S_ref) and S_ref[kk - 1] / S_ref[kk] - 1 < rel_gap:
        kk -= 1
    return max_principal_angle(U[:, :kk], U_ref[:, :kk])
