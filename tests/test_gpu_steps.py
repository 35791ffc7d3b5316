"""GPU parity of the individual steps against the oracle (through the C ABI)."""

import numpy as np
import pytest

from oracle import gaussian as OG
from oracle import linalg as OL
from oracle import rsvd as OR

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1907_06470_gb300 as g
    g.load()
    return g


# ---- Section 2.1 step 1: Gaussian test matrix, bit-exact --------------------------

@pytest.mark.parametrize("n,r,seed", [(1000, 30, 2001), (257, 13, 7), (1, 1, 0), (33, 7, 0xFFFFFFFFFFFFFFFF),
                                      (20000, 120, 2002)])
def test_gaussian_f64_bit_exact(g, n, r, seed):
    got = g.gaussian(n, r, seed, "f64").cpu().numpy()
    ref = OG.gaussian_matrix(n, r, seed, "f64")
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("n,r,seed", [(999, 31, 5), (20000, 120, 2002)])
def test_gaussian_f32_and_layouts_bit_exact(g, n, r, seed):
    ref = OG.gaussian_matrix(n, r, seed, "f32")
    got = g.gaussian(n, r, seed, "f32", layout=0).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    got_t = g.gaussian(n, r, seed, "f32", layout=1).cpu().numpy()
    assert np.array_equal(got_t.T.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("n,r,seed", [(1001, 17, 3), (4096, 128, 2002)])
def test_gaussian_bf16_bit_exact(g, n, r, seed):
    ref = OG.gaussian_matrix(n, r, seed, "bf16")
    got = g.gaussian(n, r, seed, "bf16", layout=1).cpu().view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got.T, ref)


@pytest.mark.parametrize("n,r,seed", [(20000, 120, 2002), (1_000_000, 8, 11), (4_000_000, 1, 0xDEADBEEF)])
def test_gaussian_bf16_fp32_first_equals_fp64_rounding(g, n, r, seed):
    """bfloat16 entries are evaluated in FP32 first and go to FP64 only within
    a relative 2^-19 of a rounding boundary: over millions of entries, the near-
    boundary ones included, they are the FP64 entries (bit-exact with the
    oracle above) rounded once by the oracle's to_bf16_bits."""
    f64 = g.gaussian(n, r, seed, "f64").cpu().numpy()
    ref = OG.to_bf16_bits(f64)
    for layout in (0, 1):
        got = g.gaussian(n, r, seed, "bf16", layout=layout).cpu().view(torch.int16).numpy().view(np.uint16)
        assert np.array_equal(got if layout == 0 else got.T, ref)
    # the FP64 decisions are exercised: entries within 2^-19 (relative) of the
    # midpoint between two bfloat16 neighbours
    a = np.abs(f64).ravel()
    e = np.floor(np.log2(a))
    spacing = np.exp2(e - 7)
    frac = a / spacing - np.floor(a / spacing)
    near = np.abs(frac - 0.5) * spacing <= 2.0 ** -19 * a
    assert near.sum() >= 100


def test_gaussian_sample_at_full_size(g):
    """1e6 x 350 stream (the sparse workload's width): sampled entries match the oracle."""
    n, r, seed = 1_000_000, 350, 2004
    got = g.gaussian(n, r, seed, "f32")
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.integers(0, n * r, 2000), [0, 1, n * r - 2, n * r - 1]])
    flat = got.reshape(-1)[torch.as_tensor(idx, device=got.device)].cpu().numpy()
    ref = np.array([OG.gaussian_stream(int(e), 1, seed)[0] for e in idx]).astype(np.float32)
    assert np.array_equal(flat.view(np.uint32), ref.view(np.uint32))


# ---- A-passes (Section 2.1 steps 2 and 5) --------------------------------------------

@pytest.mark.parametrize("m,n,r,mb,nb", [(700, 300, 30, 0, 0), (1037, 517, 13, 256, 128), (64, 2000, 5, 16, 300)])
def test_apass_fp64_matches_oracle(g, m, n, r, mb, nb):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    X = rng.standard_normal((n, r))
    Yt = rng.standard_normal((m, r))
    Ad = torch.as_tensor(A, device="cuda")
    y = g.apass(Ad, torch.as_tensor(X, device="cuda"), False, "fp64", mb, nb).cpu().numpy()
    z = g.apass(Ad, torch.as_tensor(Yt, device="cuda"), True, "fp64", mb, nb).cpu().numpy()
    ry, rz = OL.apply(A, X), OL.apply(A, Yt, trans=True)
    assert np.max(np.abs(y - ry)) <= 1e-13 * np.max(np.abs(ry)) * np.sqrt(n)
    assert np.max(np.abs(z - rz)) <= 1e-13 * np.max(np.abs(rz)) * np.sqrt(m)


def test_apass_exact_on_small_integers(g):
    rng = np.random.default_rng(3)
    A = rng.integers(-8, 9, size=(513, 389)).astype(np.float32)
    X = rng.integers(-8, 9, size=(389, 17)).astype(np.float32)
    Yt = rng.integers(-8, 9, size=(513, 17)).astype(np.float32)
    Ad = torch.as_tensor(A, device="cuda")
    y = g.apass(Ad, torch.as_tensor(X, device="cuda"), False, "fp32", 128, 100).cpu().numpy()
    z = g.apass(Ad, torch.as_tensor(Yt, device="cuda"), True, "fp32", 100, 128).cpu().numpy()
    assert np.array_equal(y, OL.apply(A, X).astype(np.float32))
    assert np.array_equal(z, OL.apply(A, Yt, trans=True).astype(np.float32))


@pytest.mark.parametrize("m,n,r,mb,nb", [(3000, 1500, 120, 1024, 1024), (1111, 777, 31, 300, 200)])
def test_apass_fp32_matches_oracle(g, m, n, r, mb, nb):
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, n)).astype(np.float32)
    X = rng.standard_normal((n, r)).astype(np.float32)
    Ad = torch.as_tensor(A, device="cuda")
    y = g.apass(Ad, torch.as_tensor(X, device="cuda"), False, "fp32", mb, nb).cpu().numpy().astype(np.float64)
    ry = OL.apply(A, X)
    # FP32 accumulation over n terms: |error| <= ~ n * eps32 * sum |a||x| (worst case)
    bound = n * 6e-8 * OL.apply(np.abs(A), np.abs(X))
    assert np.all(np.abs(y - ry) <= bound)
    assert np.max(np.abs(y - ry)) / np.max(np.abs(ry)) < 1e-5


# ---- CholeskyQR2 (Section 2.1 steps 3-4) ---------------------------------------------

@pytest.mark.parametrize("dtype,M,r", [("f64", 2000, 30), ("f64", 257, 256), ("f32", 100000, 120),
                                       ("f32", 20000, 120), ("f32", 513, 65), ("f64", 500, 1),
                                       ("f64", 3000, 112), ("f64", 3000, 113), ("f32", 5000, 17),
                                       ("f32", 5000, 128), ("f32", 5000, 129), ("f32", 6000, 350),
                                       ("f64", 4000, 512)])
def test_orth_is_orthonormal_and_spans_y(g, dtype, M, r):
    rng = np.random.default_rng(M + r)
    Y = rng.standard_normal((M, r)) * np.logspace(0, -2, r)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Yd = torch.as_tensor(Y, dtype=tdt, device="cuda")
    Q, R = g.orth(Yd, want_R=True)
    Q = Q.cpu().numpy().astype(np.float64)
    R = R.cpu().numpy()
    eps = 2.2e-16 if dtype == "f64" else 6e-8
    assert np.linalg.norm(Q.T @ Q - np.eye(r)) <= 50 * r * eps
    Yr = Yd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(Q @ R - Yr) <= 50 * r * eps * np.linalg.norm(Yr)
    assert np.allclose(np.tril(R, -1), 0)
    Qo, _ = OL.householder_qr(Yr)
    from tests.metrics import max_principal_angle
    assert max_principal_angle(Q, Qo) < 1e3 * eps


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_orth_rank_deficient_panel_is_completed(g, dtype):
    """Dependent columns are deflated and replaced: Q stays orthonormal, spans Y, and
    R (Y = Q R) has zero rows at the deflated pivots."""
    rng = np.random.default_rng(5)
    B = rng.standard_normal((3000, 3))
    Y = np.concatenate([B, B @ rng.standard_normal((3, 4)), B[:, :1]], axis=1)  # rank 3, r = 8
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Yd = torch.as_tensor(Y, dtype=tdt, device="cuda")
    Q, R = g.orth(Yd, want_R=True)
    Q, R = Q.cpu().numpy().astype(np.float64), R.cpu().numpy()
    eps = 2.2e-16 if dtype == "f64" else 6e-8
    assert np.linalg.norm(Q.T @ Q - np.eye(8)) <= 1e3 * eps
    Yr = Yd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(Q @ R - Yr) <= 1e3 * eps * np.linalg.norm(Yr)
    assert np.sum(np.abs(np.diag(R)) > 1e-6 * np.abs(R).max()) == 3


def test_orth_reports_non_finite_panel(g):
    Y = torch.ones(100, 4, dtype=torch.float64, device="cuda")
    Y[3, 1] = float("nan")
    with pytest.raises(g.RsvdError) as e:
        g.orth(Y)
    assert "NOT_SPD" in str(e.value)


# ---- one-sided Jacobi (Section 2.1 step 6) ------------------------------------------

def _graded_r_factor(r, seed):
    """R of the QR of a Gaussian panel with graded columns: the kind of factor the
    range finder hands to the small SVD (its column-scaled condition is small)."""
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((4 * r + 8, r)) * np.logspace(0, -4, r)
    return np.linalg.qr(Y)[1]


@pytest.mark.parametrize("r", [1, 2, 7, 30, 120, 256])
def test_small_svd_matches_oracle(g, r):
    M = _graded_r_factor(r, r)
    # the library takes M column-major, i.e. the row-major storage of M^T
    sig, U, W = g.small_svd(torch.as_tensor(np.ascontiguousarray(M.T), device="cuda"))
    sig, U, W = sig.cpu().numpy(), U.cpu().numpy(), W.cpu().numpy()
    Uo, so, Wo, _ = OL.jacobi_svd(M)
    assert np.max(np.abs(sig - so) / so) < 1e-12
    assert np.linalg.norm(M @ W - U * sig) < 1e-13 * so[0] * r
    assert np.linalg.norm(W.T @ W - np.eye(r)) < 1e-13 * r


def test_small_svd_ill_conditioned_triangle_is_backward_stable(g):
    """A random triangle has exponentially small singular values: only the
    absolute bound |sigma_i - sigma_i'| <= c r eps sigma_1 applies."""
    r = 120
    rng = np.random.default_rng(12)
    M = np.triu(rng.standard_normal((r, r)))
    sig, U, W = (t.cpu().numpy() for t in g.small_svd(torch.as_tensor(np.ascontiguousarray(M.T), device="cuda")))
    so = OL.jacobi_svd(M)[1]
    assert np.max(np.abs(sig - so)) <= 10 * r * 2.2e-16 * so[0]
    assert np.linalg.norm(M @ W - U * sig) < 1e-13 * so[0] * r


# ---- exact small SVD ------------------------------------------------------------------

@pytest.mark.parametrize("m,n,dtype", [(300, 40, "f64"), (40, 300, "f64"), (256, 256, "f64"),
                                       (500, 100, "f32"), (60, 90, "f32")])
def test_full_svd_matches_oracle(g, m, n, dtype):
    rng = np.random.default_rng(m * n)
    A = rng.standard_normal((m, n))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Ad = torch.as_tensor(A, dtype=tdt, device="cuda")
    U, S, V = (t.cpu().numpy().astype(np.float64) for t in g.full_svd(Ad))
    Uo, So, Vo = OR.full_svd(Ad.cpu().numpy().astype(np.float64))
    tol = 1e-12 if dtype == "f64" else 1e-5
    assert np.max(np.abs(S - So) / So) < tol
    assert np.linalg.norm((U * S) @ V.T - Ad.cpu().numpy()) < 10 * tol * np.linalg.norm(A)


# min(m, n) above 256 or more than 2^24 entries: CholeskyQR2 of A (or A^T) and
# the square Jacobi on R
@pytest.mark.parametrize("m,n,dtype", [(6000, 264, "f64"), (264, 6000, "f32")])
def test_full_svd_large_path_matches_oracle(g, m, n, dtype):
    rng = np.random.default_rng(m + 7 * n)
    A = rng.standard_normal((m, n))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Ad = torch.as_tensor(A, dtype=tdt, device="cuda")
    U, S, V = (t.cpu().numpy().astype(np.float64) for t in g.full_svd(Ad))
    Ah = Ad.cpu().numpy().astype(np.float64)
    Uo, So, Vo = OR.full_svd(Ah)
    tol = 1e-11 if dtype == "f64" else 1e-5
    t = min(m, n)
    assert np.max(np.abs(S - So) / So) < tol
    assert np.linalg.norm(U.T @ U - np.eye(t)) < 10 * tol and np.linalg.norm(V.T @ V - np.eye(t)) < 10 * tol
    assert np.linalg.norm((U * S) @ V.T - Ah) < 10 * tol * np.linalg.norm(Ah)


@pytest.mark.parametrize("m,n,dtype", [(200000, 88, "f32"), (600, 512, "f64")])
def test_full_svd_large_path_properties(g, m, n, dtype):
    # sizes beyond what the oracle finishes in seconds: orthonormal factors,
    # descending S and A V = U S, A^T U = V S, which fix the SVD
    tdt = torch.float64 if dtype == "f64" else torch.float32
    gen = torch.Generator(device="cuda").manual_seed(m * n)
    Ad = torch.randn(m, n, generator=gen, dtype=tdt, device="cuda")
    U, S, V = (t.double() for t in g.full_svd(Ad))
    A64 = Ad.double()
    tol = 1e-12 if dtype == "f64" else 1e-6
    t = min(m, n)
    eye = torch.eye(t, dtype=torch.float64, device="cuda")
    assert bool((S[:-1] >= S[1:]).all()) and float(S[-1]) > 0
    assert float(torch.linalg.norm(U.T @ U - eye)) < 100 * tol
    assert float(torch.linalg.norm(V.T @ V - eye)) < 100 * tol
    nA = float(torch.linalg.norm(A64))
    assert float(torch.linalg.norm(A64 @ V - U * S)) < 100 * tol * nA
    assert float(torch.linalg.norm(A64.T @ U - V * S)) < 100 * tol * nA
