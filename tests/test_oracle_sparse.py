"""Pins for the oracle's sparse products and for the sparse input recipe."""

import numpy as np
import pytest

from oracle import linalg as L
from oracle import rsvd as OR
from synth import zipf_csr


def _dense_of(m, n, rp, ci, v):
    D = np.zeros((m, n), dtype=np.float64)
    for i in range(m):
        for e in range(rp[i], rp[i + 1]):
            D[i, ci[e]] += float(v[e])
    return D


def test_csr_apply_exact_on_small_integers():
    rng = np.random.default_rng(11)
    m, n, r = 37, 23, 5
    D = (rng.random((m, n)) < 0.2) * rng.integers(-9, 10, size=(m, n))
    rp = np.concatenate([[0], np.cumsum((D != 0).sum(1))])
    ci = np.concatenate([np.nonzero(D[i])[0] for i in range(m)])
    v = D[D != 0].astype(np.float32)
    A = L.CSR(m, n, rp, ci, v)
    X = rng.integers(-5, 6, size=(n, r)).astype(np.float64)
    Yt = rng.integers(-5, 6, size=(m, r)).astype(np.float64)
    # integer sums below 2^53 are exact, so the products must equal the triple loop
    ref = np.array([[sum(D[i, j] * X[j, c] for j in range(n)) for c in range(r)] for i in range(m)])
    assert np.array_equal(L.apply(A, X), ref)
    reft = np.array([[sum(D[i, j] * Yt[i, c] for i in range(m)) for c in range(r)] for j in range(n)])
    assert np.array_equal(L.apply(A, Yt, trans=True), reft)


def test_rsvd_of_csr_equals_rsvd_of_its_dense_form():
    m, n = 400, 300
    rp, ci, v = zipf_csr(m, n, 2000, 7)
    A = L.CSR(m, n, rp, ci, v)
    D = _dense_of(m, n, rp, ci, v)
    Us, Ss, Vs = OR.rsvd(A, 10, 5, 2, 2004, "f32")
    Ud, Sd, Vd = OR.rsvd(D, 10, 5, 2, 2004, "f32")
    assert np.max(np.abs(Ss - Sd) / Sd) < 1e-12
    assert np.max(np.abs(Us - Ud)) < 1e-9 and np.max(np.abs(Vs - Vd)) < 1e-9


@pytest.mark.parametrize("m,n,nnz,seed", [(2000, 1000, 20000, 1), (20000, 5000, 400000, 1004)])
def test_zipf_csr_structure(m, n, nnz, seed):
    rp, ci, v = zipf_csr(m, n, nnz, seed)
    assert rp.dtype == np.int32 and ci.dtype == np.int32 and v.dtype == np.float32
    assert rp[0] == 0 and rp[-1] == ci.size == v.size
    lens = np.diff(rp)
    cap = max(1, min(20000, n // 50))
    assert lens.min() >= 1 and lens.max() <= cap           # no empty rows, cap held
    assert abs(int(rp[-1]) - nnz) <= 0.01 * nnz + m        # total close to the target
    assert np.all(v > 0) and np.all(np.isfinite(v))        # zero-truncated Poisson: no stored zeros
    assert ci.min() >= 0 and ci.max() < n
    # colidx strictly ascending inside every row (sorted, no duplicates)
    d = np.diff(ci.astype(np.int64))
    row_start = np.zeros(ci.size, dtype=bool)
    row_start[rp[:-1][lens > 0]] = True
    assert np.all(d[~row_start[1:]] > 0)
    # Zipf(1.0) columns: column 0 is the most frequent, and the head outweighs the tail
    df = np.bincount(ci, minlength=n)
    assert df[0] == df.max()
    assert df[: n // 10].sum() > df[n // 10:].sum()
    # the same seed reproduces the same matrix
    rp2, ci2, v2 = zipf_csr(m, n, nnz, seed)
    assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2) and np.array_equal(v, v2)
