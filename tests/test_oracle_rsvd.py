"""Pins for the oracle's randomized SVD (Section 2.1, Section 2.2)."""

import math

import numpy as np
import pytest

from oracle import rsvd as R
from oracle.linalg import apply, householder_qr
from synth import prescribed_dense, spectrum_geometric
from tests.metrics import max_principal_angle


def test_exact_when_sketch_spans_the_range():
    """A of exact rank 25 and r = 30 >= 25: the randomized SVD is exact."""
    m, n, k, p = 300, 120, 20, 10
    s = np.concatenate([spectrum_geometric(25, 0.8), np.zeros(0)])
    A, U0, V0 = prescribed_dense(m, n, s, seed=11)
    for q in (0, 1, 2):
        U, S, V = R.rsvd(A, k, p, q, seed=21)
        assert np.max(np.abs(S - s[:k]) / s[:k]) < 1e-12
        assert max_principal_angle(U, U0[:, :k]) < 1e-10
        assert max_principal_angle(V, V0[:, :k]) < 1e-10
        # the factors reproduce the rank-k truncation of A
        Ak = (U0[:, :k] * s[:k]) @ V0[:, :k].T
        assert np.linalg.norm((U * S) @ V.T - Ak) < 1e-12 * np.linalg.norm(Ak)


def test_exact_when_r_equals_min_dimension():
    m, n = 80, 40
    s = spectrum_geometric(40, 0.9)
    A, U0, V0 = prescribed_dense(m, n, s, seed=3)
    U, S, V = R.rsvd(A, 30, 10, 0, seed=4)
    assert np.max(np.abs(S - s[:30]) / s[:30]) < 1e-12


def _hmt_factor(k, p, m, n, q):
    return (1 + 11 * math.sqrt(k + p) * math.sqrt(min(m, n))) ** (1.0 / (2 * q + 1))


@pytest.mark.parametrize("q", [0, 1, 2])
def test_hmt_error_bound_over_seeds(q):
    """||A - Q Q^T A||_2 <= [1 + 11 sqrt(k+p) sqrt(min(m,n))]^(1/(2q+1)) sigma_{k+1}
    (Halko, Martinsson & Tropp 2011, Eq. (1.9) and its power-scheme form in
    Section 10.4), which holds with probability >= 1 - 6 p^-p."""
    m, n, k, p = 400, 200, 20, 10
    s = 1.0 / np.arange(1, n + 1)
    A, _, _ = prescribed_dense(m, n, s, seed=5)
    for seed in range(10):
        Q = R.range_finder(A, k + p, q, seed)
        err = np.linalg.norm(A - Q @ (Q.T @ A), 2)
        assert err <= _hmt_factor(k, p, m, n, q) * s[k]
        assert err >= s[k + p] * (1 - 1e-12)  # no rank-r projector beats sigma_{r+1}


def test_power_iterations_shrink_the_error():
    m, n, k, p = 500, 300, 20, 5
    s = 1.0 / np.sqrt(np.arange(1, n + 1))
    A, _, _ = prescribed_dense(m, n, s, seed=6)
    errs = []
    for q in (0, 1, 2):
        Q = R.range_finder(A, k + p, q, seed=7)
        errs.append(np.linalg.norm(A - Q @ (Q.T @ A), 2))
    assert errs[0] > errs[1] > errs[2]


def test_interlacing_and_rayleigh_ritz():
    """sigma_i(Q^T A) <= sigma_i(A); the small SVD equals a library SVD of Q^T A."""
    m, n, k, p, q = 300, 150, 10, 5, 1
    s = spectrum_geometric(150, 0.97)
    A, _, _ = prescribed_dense(m, n, s, seed=8)
    U, S, V = R.rsvd(A, k, p, q, seed=9)
    assert np.all(S <= s[:k] * (1 + 1e-12))
    Q = R.range_finder(A, k + p, q, seed=9)
    ref = np.linalg.svd(Q.T @ A, compute_uv=False)[:k]
    assert np.allclose(S, ref, rtol=1e-12)
    # U = Q U_B: U lies in span(Q); U and V are orthonormal and U^T A V = diag(S)
    assert np.linalg.norm(U - Q @ (Q.T @ U)) < 1e-12
    assert np.linalg.norm(U.T @ U - np.eye(k)) < 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(k)) < 1e-12
    assert np.allclose(U.T @ A @ V, np.diag(S), atol=1e-12)


def test_small_svd_of_bt_reconstructs_b():
    rng = np.random.default_rng(12)
    Bt = rng.standard_normal((90, 12)) * np.logspace(0, -4, 12)
    UB, sig, V = R.small_svd_of_bt(Bt)
    assert np.linalg.norm(V @ np.diag(sig) @ UB.T - Bt) < 1e-13 * np.linalg.norm(Bt)
    assert np.allclose(sig, np.linalg.svd(Bt, compute_uv=False), rtol=1e-12)


def test_full_svd_matches_library():
    rng = np.random.default_rng(13)
    for shape in [(9, 4), (4, 9), (6, 6), (40, 17)]:
        A = rng.standard_normal(shape)
        U, S, V = R.full_svd(A)
        t = min(shape)
        assert np.allclose(S, np.linalg.svd(A, compute_uv=False), rtol=1e-13)
        assert np.linalg.norm((U * S) @ V.T - A) < 1e-13 * np.linalg.norm(A)
        assert np.linalg.norm(U.T @ U - np.eye(t)) < 1e-13 and np.linalg.norm(V.T @ V - np.eye(t)) < 1e-13
    # rank 2 in a 7 x 5: three singular values at rounding level; the vectors
    # of the two nonzero ones are orthonormal (those of the null part are not
    # completed to an orthonormal set)
    A = rng.standard_normal((7, 2)) @ rng.standard_normal((2, 5))
    U, S, V = R.full_svd(A)
    assert np.all(S[2:] < 1e-14 * S[0])
    assert np.linalg.norm(U[:, :2].T @ U[:, :2] - np.eye(2)) < 1e-13
    assert np.linalg.norm(V[:, :2].T @ V[:, :2] - np.eye(2)) < 1e-13
    assert np.linalg.norm((U * S) @ V.T - A) < 1e-13 * np.linalg.norm(A)


def test_signs_are_normalised():
    m, n = 60, 30
    A, _, _ = prescribed_dense(m, n, spectrum_geometric(30, 0.7), seed=14)
    U, S, V = R.rsvd(A, 5, 5, 1, seed=15)
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(5)] > 0)


def test_argument_checks():
    A = np.zeros((10, 5))
    with pytest.raises(ValueError):
        R.rsvd(A, 4, 2, 0, seed=1)  # k + p > min(m, n)
    with pytest.raises(ValueError):
        R.rsvd(A, 0, 2, 0, seed=1)


def test_fp32_input_is_widened_exactly():
    rng = np.random.default_rng(16)
    A32 = rng.standard_normal((50, 20)).astype(np.float32)
    X = rng.standard_normal((20, 3))
    assert np.array_equal(apply(A32, X), A32.astype(np.float64) @ X)
    Q, _ = householder_qr(apply(A32, X))
    assert Q.shape == (50, 3)


def test_auto_q_equals_fixed_q_at_the_chosen_count():
    """The automatic loop is the fixed-q computation stopped early: bit-identical."""
    A, _, _ = prescribed_dense(600, 300, spectrum_geometric(300, 0.97), 21)
    for tol in (1e-1, 1e-3, 1e-6):
        U, S, V, qu = R.rsvd_auto_q(A, 10, 5, 6, 2001, tol)
        Uf, Sf, Vf = R.rsvd(A, 10, 5, qu, 2001)
        assert np.array_equal(S, Sf) and np.array_equal(U, Uf) and np.array_equal(V, Vf)


def test_auto_q_stops_at_one_for_an_exactly_low_rank_matrix():
    """rank(A) <= r: the first sketch already spans the range, sigma^(1) = sigma^(0)
    to rounding, so one iteration is used."""
    s = np.concatenate([spectrum_geometric(12, 0.8), np.zeros(188)])
    A, _, _ = prescribed_dense(400, 200, s, 22)
    _, S, _, qu = R.rsvd_auto_q(A, 8, 6, 5, 2001, 1e-8)
    assert qu == 1
    assert np.max(np.abs(S - s[:8]) / s[:8]) < 1e-12


def test_auto_q_runs_to_the_limit_when_the_spectrum_keeps_moving():
    A, _, _ = prescribed_dense(500, 400, spectrum_geometric(400, 0.999), 23)
    _, _, _, qu = R.rsvd_auto_q(A, 20, 5, 3, 2001, 1e-12)
    assert qu == 3
    with pytest.raises(ValueError):
        R.rsvd_auto_q(A, 20, 5, -1, 2001)


# ---- fused power sweeps: W = orth(A^T (A W)) ------------------------------------

def test_fused_sweeps_exact_when_sketch_spans_the_range():
    m, n, k, p = 300, 120, 20, 10
    s = spectrum_geometric(25, 0.8)
    A, U0, V0 = prescribed_dense(m, n, s, seed=11)
    for q in (0, 1, 2):
        U, S, V = R.rsvd_fused_sweeps(A, k, p, q, seed=21)
        assert np.max(np.abs(S - s[:k]) / s[:k]) < 1e-12
        assert max_principal_angle(U, U0[:, :k]) < 1e-10
        assert max_principal_angle(V, V0[:, :k]) < 1e-10


def test_fused_sweeps_without_iterations_is_the_plain_scheme():
    A, _, _ = prescribed_dense(200, 90, spectrum_geometric(90, 0.93), seed=5)
    a = R.rsvd(A, 10, 5, 0, seed=6)
    b = R.rsvd_fused_sweeps(A, 10, 5, 0, seed=6)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("q", [1, 2])
def test_fused_sweeps_span_the_same_sketch(q):
    """(A A^T)^q A O has one span however the products are grouped: with the
    spectrum far above sqrt(eps) the two range finders agree to rounding."""
    m, n, k, p = 400, 150, 12, 8
    s = 1.0 / np.arange(1, n + 1)          # sigma_n / sigma_1 ~ 7e-3, squared 4e-5 >> eps
    A, _, _ = prescribed_dense(m, n, s, seed=8)
    Qa = R.range_finder(A, k + p, q, 9)
    Qb = R.range_finder_fused(A, k + p, q, 9)
    assert max_principal_angle(Qa, Qb) < 1e-9
    Ua, Sa, Va = R.rsvd(A, k, p, q, seed=9)
    Ub, Sb, Vb = R.rsvd_fused_sweeps(A, k, p, q, seed=9)
    assert np.max(np.abs(Sa - Sb) / Sa) < 1e-12
    assert max_principal_angle(Ua, Ub) < 1e-9 and max_principal_angle(Va, Vb) < 1e-9


@pytest.mark.parametrize("q", [1, 2])
def test_fused_sweeps_meet_the_hmt_bound(q):
    m, n, k, p = 300, 200, 10, 5
    s = spectrum_geometric(200, 0.95)
    A, _, _ = prescribed_dense(m, n, s, seed=17)
    bound = _hmt_factor(k, p, m, n, q) * s[k]
    for seed in range(5):
        U, S, V = R.rsvd_fused_sweeps(A, k + p, 0, q, seed=100 + seed)
        Q = U  # the rank-(k+p) basis
        err = np.linalg.norm(A - Q @ (Q.T @ A), 2)
        assert err <= bound


def test_fused_sweeps_accuracy_under_bf16_rounding():
    """The accuracy cost of the fused reading where the arithmetic is BF16: the
    range finder run with A, the panels and (fused) the intermediate A W
    rounded to BF16, on the harmonic-plus-noise spectrum of the dense
    workload, against the FP64 per-product result.  Rounding A W to BF16 costs
    up to a few times the per-product error; carrying A W as two BF16 parts
    (hi + lo, as the split panel of the tensor-core passes does) removes it."""
    from oracle.gaussian import bf16_bits_to_f64, gaussian_matrix_as_f64, to_bf16_bits
    from synth import spectrum_harmonic_noisy

    def bf(x):
        return bf16_bits_to_f64(to_bf16_bits(x))

    def orth(Y):
        return householder_qr(Y)[0]

    m, n, k, p, q = 3000, 1500, 50, 10, 2
    A, _, _ = prescribed_dense(m, n, spectrum_harmonic_noisy(n, 1e-4, 7), 8)
    Ab = bf(A)
    O = gaussian_matrix_as_f64(n, k + p, 9, "bf16")

    def top_sigma(Q):
        return np.linalg.svd(A.T @ Q, compute_uv=False)[:k]

    ref = top_sigma(R.range_finder(A, k + p, q, 9, "bf16"))
    Q = orth(Ab @ O)
    for _ in range(q):
        Q = orth(Ab @ bf(orth(Ab.T @ bf(Q))))
    per_product = np.max(np.abs(top_sigma(Q) - ref) / ref)
    W = O
    for _ in range(q):
        W = orth(Ab.T @ bf(Ab @ bf(W)))
    fused = np.max(np.abs(top_sigma(orth(Ab @ bf(W))) - ref) / ref)
    W = O
    for _ in range(q):
        Y = Ab @ bf(W)
        hi = bf(Y)
        W = orth(Ab.T @ (hi + bf(Y - hi)))
    fused_split = np.max(np.abs(top_sigma(orth(Ab @ bf(W))) - ref) / ref)
    assert per_product < 1e-3
    assert fused <= 4 * per_product and fused < 5e-4
    assert fused_split <= 1.3 * per_product
