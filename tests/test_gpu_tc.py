"""Tensor-core (tcgen05) A-passes: exactness on small integers, accuracy of the
BF16 and split-BF16 modes against FP64 products, split-K balance, and the
BF16 randomized SVD against the oracle."""

import numpy as np
import pytest

from oracle import linalg as OL
from oracle import rsvd as OR
from synth import prescribed_dense, spectrum_harmonic_noisy
from tests.metrics import max_principal_angle, sigma_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1907_06470_gb300 as g
    g.load()
    return g


def _bf16(x):
    return torch.as_tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


# row strides are multiples of 4 floats (the TMA rule the library enforces)
SHAPES = [(300, 200, 17), (128, 64, 1), (513, 388, 120), (1000, 132, 128), (257, 1000, 200), (640, 320, 256),
          (129, 68, 30)]


@pytest.mark.parametrize("m,n,r", SHAPES)
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_tc_apass_exact_on_small_integers(g, m, n, r, trans, prec):
    if prec == "bf16x3" and r > 192:
        pytest.skip("split mode supports r <= 192")
    rng = np.random.default_rng(m * 7 + n * 3 + r)
    A = rng.integers(-4, 5, size=(m, n)).astype(np.float32)
    K = m if trans else n
    X = rng.integers(-4, 5, size=(K, r)).astype(np.float32)
    got = g.apass(torch.as_tensor(A, device="cuda"), torch.as_tensor(X, device="cuda"), trans, prec).cpu().numpy()
    ref = OL.apply(A, X, trans=trans).astype(np.float32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("trans", [False, True])
def test_tc_apass_bf16_error_model(g, trans):
    """BF16 mode = exact product of the BF16-rounded operands, accumulated in FP32."""
    m, n, r = 2000, 1500, 120
    rng = np.random.default_rng(1 + trans)
    A = rng.standard_normal((m, n)).astype(np.float32)
    K = m if trans else n
    X = rng.standard_normal((K, r)).astype(np.float32)
    got = g.apass(torch.as_tensor(A, device="cuda"), torch.as_tensor(X, device="cuda"), trans, "bf16").cpu().numpy()
    Ab, Xb = _bf16(A), _bf16(X)
    ref = OL.apply(Ab, Xb, trans=trans)
    bound = (K + 2) * 2.0 ** -24 * OL.apply(np.abs(Ab), np.abs(Xb), trans=trans)
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("trans", [False, True])
def test_tc_apass_split_mode_is_near_fp32(g, trans):
    m, n, r = 1500, 1100, 64
    rng = np.random.default_rng(5 + trans)
    A = rng.standard_normal((m, n)).astype(np.float32)
    K = m if trans else n
    X = rng.standard_normal((K, r)).astype(np.float32)
    got = g.apass(torch.as_tensor(A, device="cuda"), torch.as_tensor(X, device="cuda"), trans, "bf16x3").cpu().numpy()
    ref = OL.apply(A, X, trans=trans)
    scale = OL.apply(np.abs(A), np.abs(X), trans=trans)
    rel = np.max(np.abs(got - ref) / scale)
    assert rel < 2.0 ** -14  # BF16 alone sits near 2^-9
    bf = g.apass(torch.as_tensor(A, device="cuda"), torch.as_tensor(X, device="cuda"), trans, "bf16").cpu().numpy()
    assert rel < np.max(np.abs(bf - ref) / scale) / 30


def test_tc_apass_split_k_matches_unsplit_reference(g):
    """Long K with few output tiles forces the K range to be split over CTAs."""
    m, n, r = 60000, 256, 32
    rng = np.random.default_rng(9)
    A = rng.integers(-2, 3, size=(m, n)).astype(np.float32)
    Y = rng.integers(-2, 3, size=(m, r)).astype(np.float32)
    got = g.apass(torch.as_tensor(A, device="cuda"), torch.as_tensor(Y, device="cuda"), True, "bf16").cpu().numpy()
    assert np.array_equal(got, OL.apply(A, Y, trans=True).astype(np.float32))


def test_tc_apass_rejects_misaligned_rows(g):
    A = torch.zeros(64, 67, device="cuda")
    X = torch.zeros(67, 8, device="cuda")
    with pytest.raises(g.RsvdError):
        g.apass(A, X, False, "bf16")


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_bf16_rsvd_against_oracle(g, prec):
    """BF16 path (reported, not pinned to FP32 tolerances): errors against the
    FP64 oracle run with the same BF16-rounded test matrix."""
    m, n, k, p, q, seed = 8000, 4000, 100, 20, 2, 2002
    s = spectrum_harmonic_noisy(n, 1e-4, 3002)
    A, _, _ = prescribed_dense(m, n, s, 1002, dtype=np.float32)
    U, S, V = (t.cpu().numpy().astype(np.float64) for t in
               g.rsvd(torch.as_tensor(A, device="cuda"), k, p, q, seed, prec=prec))
    Uo, So, Vo = OR.rsvd(A, k, p, q, seed, "bf16")
    es, eu, ev = sigma_rel_err(S, So), max_principal_angle(U, Uo), max_principal_angle(V, Vo)
    print(f"{prec}: sigma rel err {es:.2e}, U angle {eu:.2e}, V angle {ev:.2e}")
    # the BF16 plan's small SVD stops at FP32 convergence: U and V stay
    # orthonormal far below the BF16 error
    I = np.eye(k)
    assert np.abs(U.T @ U - I).max() <= 1e-4 and np.abs(V.T @ V - I).max() <= 1e-4
    if prec == "bf16x3":
        assert es <= 1e-4 and eu <= 1e-2
    else:
        assert es <= 1e-2


def test_bf16_copy_of_a_gives_the_same_bits(g):
    """In-core BF16 plans read a BF16 copy of A that the first forward pass
    writes: the same operands as converting the FP32 A in every pass, hence
    the same result bit for bit.  A memory cap with no room for the copy makes
    every pass read the FP32 A.  Ragged sizes: a partial last row tile and
    columns padded to whole 64-column tiles in the copy."""
    m, n, k, p, q, seed = 6007, 3004, 40, 8, 2, 11
    A, _, _ = prescribed_dense(m, n, spectrum_harmonic_noisy(n, 1e-4, 5), 7, dtype=np.float32)
    Ad = torch.as_tensor(A, device="cuda")
    p1 = g.Plan(m, n, k, p, q, seed, prec="bf16")
    U1, S1, V1 = p1.run(Ad)
    ws = p1.info()["workspace_bytes"]
    p1.close()
    p2 = g.Plan(m, n, k, p, q, seed, mem_cap=ws + 4096, prec="bf16")
    U2, S2, V2 = p2.run(Ad)
    p2.close()
    assert torch.equal(S1, S2) and torch.equal(U1, U2) and torch.equal(V1, V2)


@pytest.mark.parametrize("r", [48, 120])
def test_split_copy_of_a_gives_the_same_bits(g, r):
    """In-core BF16X3 plans keep BF16(A) and BF16(A - BF16(A)) from the first
    forward pass and read the two parts in the later passes (three products,
    no conversion): the operands the FP32 A splits into, so the same bits as
    a plan without room for the copy."""
    m, n, q, seed = 6007, 3004, 2, 11
    k, p = r - 8, 8
    A, _, _ = prescribed_dense(m, n, spectrum_harmonic_noisy(n, 1e-4, 5), 7, dtype=np.float32)
    Ad = torch.as_tensor(A, device="cuda")
    p1 = g.Plan(m, n, k, p, q, seed, prec="bf16x3")
    U1, S1, V1 = p1.run(Ad)
    assert p1.info()["bf16_copy"] == 1
    ws = p1.info()["workspace_bytes"]
    p1.close()
    p2 = g.Plan(m, n, k, p, q, seed, mem_cap=ws + 4096, prec="bf16x3")
    U2, S2, V2 = p2.run(Ad)
    assert p2.info()["bf16_copy"] == 0
    p2.close()
    assert torch.equal(S1, S2) and torch.equal(U1, U2) and torch.equal(V1, V2)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
@pytest.mark.parametrize("M,r", [(100000, 120), (5003, 36), (4096, 128)])
def test_gram_of_a_panel_matches_the_general_path(g, prec, M, r):
    """Y^T Y with one row tile of output uses the converted tile of Y^T as the
    panel operand too: the same rounded operands as converting the panel
    separately, so the same bits."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(M + r)
    Y = torch.randn(M, r, generator=gen, device="cuda")
    G1 = g.apass(Y, Y, True, prec)            # X is A: the Gram path
    G2 = g.apass(Y, Y.clone(), True, prec)    # a separate panel
    assert torch.equal(G1, G2)
    ref = (Y.double().T @ Y.double()).cpu().numpy()
    assert np.abs(G1.double().cpu().numpy() - ref).max() <= (2e-2 if prec == "bf16" else 1e-4) * np.abs(ref).max()


# ---- A stored in 16 bits (BF16 or IEEE FP16) --------------------------------------

TDT16 = {"bf16": torch.bfloat16, "f16": torch.float16}


def _round16(x, fmt):
    """x rounded to the 16-bit format (round to nearest even), as FP64."""
    if fmt == "f16":
        return np.asarray(x, np.float32).astype(np.float16).astype(np.float64)
    return _bf16(x)


# row strides are multiples of 8 values (16 bytes) for a 16-bit A
SHAPES16 = [(300, 200, 17), (513, 392, 120), (257, 1000, 200), (129, 72, 30), (640, 320, 256)]


@pytest.mark.parametrize("m,n,r", SHAPES16)
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_16bit_source_exact_on_small_integers(g, m, n, r, trans, prec, fmt):
    rng = np.random.default_rng(m * 7 + n * 3 + r + (fmt == "f16"))
    A = rng.integers(-4, 5, size=(m, n)).astype(np.float32)
    K = m if trans else n
    X = rng.integers(-4, 5, size=(K, r)).astype(np.float32)
    A16 = torch.as_tensor(A, device="cuda").to(TDT16[fmt])
    got = g.apass(A16, torch.as_tensor(X, device="cuda"), trans, prec).cpu().numpy()
    ref = OL.apply(A, X, trans=trans).astype(np.float32)
    assert got.dtype == np.float32 and np.array_equal(got, ref)


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_16bit_source_many_units_per_cta(g, trans, prec):
    """Enough 128-row output tiles that every CTA of the persistent grid takes
    three or more of them (the accumulator double buffer cycles), exact on
    small integers."""
    rng = np.random.default_rng(11 + trans)
    m, n = (60000, 1024) if not trans else (1024, 60000)
    A = rng.integers(-4, 5, size=(m, n)).astype(np.float32)
    K = m if trans else n
    X = rng.integers(-4, 5, size=(K, 64)).astype(np.float32)
    A16 = torch.as_tensor(A, device="cuda").to(torch.bfloat16)
    got = g.apass(A16, torch.as_tensor(X, device="cuda"), trans, prec).cpu().numpy()
    ref = (A.T if trans else A).astype(np.float64) @ X.astype(np.float64)
    assert np.array_equal(got, ref.astype(np.float32))


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_16bit_source_error_model(g, trans, fmt):
    """prec BF16 on a 16-bit A: the exact product of A and the panel rounded to
    A's format, accumulated in FP32.  prec BF16X3: the panel split in two
    16-bit parts, close to the FP32 product of the stored A."""
    m, n, r = 2000, 1504, 120
    rng = np.random.default_rng(3 + trans + 2 * (fmt == "f16"))
    A16 = torch.as_tensor(rng.standard_normal((m, n)).astype(np.float32)).to(TDT16[fmt])
    Ad = A16.double().numpy()
    K = m if trans else n
    X = rng.standard_normal((K, r)).astype(np.float32)
    Xd = torch.as_tensor(X, device="cuda")
    got = g.apass(A16.to("cuda"), Xd, trans, "bf16").cpu().numpy()
    Xr = _round16(X, fmt)
    ref = OL.apply(Ad, Xr, trans=trans)
    bound = (K + 2) * 2.0 ** -24 * OL.apply(np.abs(Ad), np.abs(Xr), trans=trans)
    assert np.all(np.abs(got - ref) <= bound)
    split = g.apass(A16.to("cuda"), Xd, trans, "bf16x3").cpu().numpy()
    ref = OL.apply(Ad, X.astype(np.float64), trans=trans)
    scale = OL.apply(np.abs(Ad), np.abs(X.astype(np.float64)), trans=trans)
    rel = np.max(np.abs(split - ref) / scale)
    assert rel < 2.0 ** -14
    assert rel < np.max(np.abs(got - ref) / scale) / 30


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_16bit_storage_rsvd_against_oracle(g, fmt):
    """rsvd of a matrix stored in 16 bits against the FP64 oracle on the
    values that matrix holds (the same BF16-rounded test matrix)."""
    m, n, k, p, q, seed = 8000, 4000, 100, 20, 2, 2002
    s = spectrum_harmonic_noisy(n, 1e-4, 3002)
    A, _, _ = prescribed_dense(m, n, s, 1002, dtype=np.float32)
    A16 = torch.as_tensor(A * np.float32(256.0)).to(TDT16[fmt])   # entries in FP16's normal range
    Ad = A16.double().numpy()
    U, S, V = (t.cpu().numpy().astype(np.float64) for t in g.rsvd(A16.to("cuda"), k, p, q, seed))
    Uo, So, Vo = OR.rsvd(Ad, k, p, q, seed, "bf16")
    es, eu, ev = sigma_rel_err(S, So), max_principal_angle(U, Uo), max_principal_angle(V, Vo)
    print(f"{fmt}: sigma rel err {es:.2e}, U angle {eu:.2e}, V angle {ev:.2e}")
    I = np.eye(k)
    assert np.abs(U.T @ U - I).max() <= 1e-4 and np.abs(V.T @ V - I).max() <= 1e-4
    assert es <= 1e-4 and eu <= 1e-2


def test_16bit_storage_host_copy_and_row_stride(g):
    """A host 16-bit A with n not a multiple of 8 is copied with padded rows:
    the same bits as the device A with the same padded stride; a device A
    whose stride is not a multiple of 8 values is rejected."""
    m, n, k, p, q, seed = 3001, 1003, 30, 10, 1, 5
    A, _, _ = prescribed_dense(m, n, spectrum_harmonic_noisy(n, 1e-4, 8), 9, dtype=np.float32)
    A16 = torch.as_tensor(A * np.float32(256.0)).to(torch.float16)
    pad = torch.zeros(m, 1008, dtype=torch.float16, device="cuda")
    pad[:, :n] = A16.to("cuda")
    a = g.rsvd(A16, k, p, q, seed)
    b = g.rsvd(pad[:, :n], k, p, q, seed)
    for s_, t_ in zip(a, b):
        assert torch.equal(s_, t_)
    with pytest.raises(g.RsvdError):
        g.rsvd(A16.to("cuda"), k, p, q, seed)
