"""Sparse (CSR) A-passes and the randomized SVD of a CSR matrix (Section 3.3
sparse x dense products, Section 2.1 steps 1-7) against the FP64 oracle."""

import numpy as np
import pytest

from oracle import linalg as OL
from oracle import panel as OP
from oracle import rsvd as OR
from oracle import tiles as OT
from synth import zipf_csr
from tests.metrics import cluster_safe_angles, sigma_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1907_06470_gb300 as g
    g.load()
    return g


@pytest.fixture(scope="module")
def zipf():
    """The sparse workload's recipe scaled to 20000 x 5000 with 4e5 entries."""
    m, n = 20000, 5000
    rp, ci, v = zipf_csr(m, n, 400000, 1004)
    return m, n, rp, ci, v


@pytest.fixture(scope="module")
def zipf_abs(zipf):
    """|A| and |A|^T (oracle CSR) for the rounding bounds."""
    m, n, rp, ci, v = zipf
    trp, tci, tv = OT.csr_transpose(m, n, rp, ci, np.abs(v))
    return OL.CSR(m, n, rp, ci, np.abs(v)), OL.CSR(n, m, trp, tci, tv)


def _torch_csr(m, n, rp, ci, v, device):
    return torch.sparse_csr_tensor(torch.as_tensor(rp), torch.as_tensor(ci), torch.as_tensor(v),
                                   size=(m, n), device=device)


def _fp32_product_bound(A_abs_csr, X):
    """Per-entry bound on the FP32 accumulation error: gamma_L |A| |X| with L the
    longest row, gamma_L = L u / (1 - L u), u = 2^-24."""
    L = int(np.max(np.diff(A_abs_csr.rowptr)))
    u = 2.0 ** -24
    gam = (L + 1) * u / (1 - (L + 1) * u)
    return gam * OL.csr_apply(A_abs_csr, np.abs(X))


@pytest.mark.parametrize("r", [1, 7, 120, 350, 512])
@pytest.mark.parametrize("aligned", [True, False])
def test_csr_apass_matches_oracle(g, zipf, zipf_abs, r, aligned):
    m, n, rp, ci, v = zipf
    A = OL.CSR(m, n, rp, ci, v)
    Aabs, Atabs = zipf_abs
    rng = np.random.default_rng(r)
    # the panel is rounded to FP32 first, so both sides multiply the same numbers
    X = rng.standard_normal((n, r)).astype(np.float32)
    Yt = rng.standard_normal((m, r)).astype(np.float32)
    Ad = _torch_csr(m, n, rp, ci, v, "cuda")
    Atd = g.csr_transpose(_torch_csr(m, n, rp, ci, v, "cpu")).to("cuda")
    if aligned:
        Xd = torch.as_tensor(X, device="cuda")
        Ytd = torch.as_tensor(Yt, device="cuda")
    else:  # leading dimension r + 1: the scalar kernel
        Xd = torch.zeros(n, r + 1, device="cuda")[:, :r]
        Xd.copy_(torch.as_tensor(X))
        Ytd = torch.zeros(m, r + 1, device="cuda")[:, :r]
        Ytd.copy_(torch.as_tensor(Yt))
    Y = g.apass(Ad, Xd, trans=False).cpu().numpy().astype(np.float64)
    Z = g.apass(Ad, Ytd, trans=True, At=Atd).cpu().numpy().astype(np.float64)
    Yo = OL.csr_apply(A, X.astype(np.float64))
    Zo = OL.csr_apply(A, Yt.astype(np.float64), trans=True)
    assert np.all(np.abs(Y - Yo) <= _fp32_product_bound(Aabs, X) + 1e-30)
    assert np.all(np.abs(Z - Zo) <= _fp32_product_bound(Atabs, Yt) + 1e-30)


@pytest.mark.parametrize("prec,bits", [("bf16", 8), ("bf16x3", 16)])
@pytest.mark.parametrize("r", [7, 120, 350])
def test_csr_compact_panel_pass_matches_oracle(g, zipf, zipf_abs, prec, bits, r):
    """BF16 and 24-bit panels: the pass equals the FP64 product of A with the
    panel rounded by the oracle (8 / 16 significant bits, ties to even),
    within the FP32 accumulation bound -- forward, and transposed over the
    long rows of A^T (split into segments)."""
    m, n, rp, ci, v = zipf
    A = OL.CSR(m, n, rp, ci, v)
    Aabs, Atabs = zipf_abs
    rng = np.random.default_rng(100 + r)
    X = rng.standard_normal((n, r)).astype(np.float32)
    Yt = (rng.standard_normal((m, r)) * 1e-3).astype(np.float32)
    Ad = _torch_csr(m, n, rp, ci, v, "cuda")
    Atd = g.csr_transpose(_torch_csr(m, n, rp, ci, v, "cpu")).to("cuda")
    Y = g.apass(Ad, torch.as_tensor(X, device="cuda"), prec=prec).cpu().numpy().astype(np.float64)
    Z = g.apass(Ad, torch.as_tensor(Yt, device="cuda"), trans=True, At=Atd, prec=prec).cpu().numpy()
    Xr = OP.round_significant(X, bits).astype(np.float64)
    Ytr = OP.round_significant(Yt, bits).astype(np.float64)
    assert np.all(np.abs(Y - OL.csr_apply(A, Xr)) <= _fp32_product_bound(Aabs, Xr) + 1e-30)
    Zo = OL.csr_apply(A, Ytr, trans=True)
    assert np.all(np.abs(Z.astype(np.float64) - Zo) <= _fp32_product_bound(Atabs, Ytr) + 1e-30)
    # the rounding is what moved the result: the FP32 panel's product differs
    Yf = OL.csr_apply(A, X.astype(np.float64))
    rel = np.abs(Y - Yf).max() / np.abs(Yf).max()
    assert rel <= 2.0 ** -bits


def test_csr_apass_is_deterministic(g, zipf):
    m, n, rp, ci, v = zipf
    Ad = _torch_csr(m, n, rp, ci, v, "cuda")
    X = torch.randn(n, 120, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    Y1 = g.apass(Ad, X)
    Y2 = g.apass(Ad, X)
    assert torch.equal(Y1, Y2)


def test_csr_rsvd_scaled_sparse_workload_matches_oracle(g, zipf):
    """k=64 p=16 q=3 on the scaled recipe; FP32 path against the FP64 oracle."""
    m, n, rp, ci, v = zipf
    k, p, q, seed = 64, 16, 3, 2004
    U, S, V = g.rsvd(_torch_csr(m, n, rp, ci, v, "cuda"), k, p, q, seed)
    U, S, V = (t.cpu().numpy().astype(np.float64) for t in (U, S, V))
    Uo, So, Vo = OR.rsvd(OL.CSR(m, n, rp, ci, v), k, p, q, seed, "f32")
    assert sigma_rel_err(S, So) <= 1e-5
    assert cluster_safe_angles(U, Uo, So, 8, rel_gap=1e-2) <= 1e-4
    assert cluster_safe_angles(V, Vo, So, 8, rel_gap=1e-2) <= 1e-4


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_csr_rsvd_compact_panels_against_oracle(g, zipf, prec):
    """CSR plans whose range finder gathers compact panels, the final
    B^T = A^T Q an FP32 panel: 24-bit panels (BF16X3) meet the FP32 bars;
    BF16 panels are reported against looser ones."""
    m, n, rp, ci, v = zipf
    k, p, q, seed = 64, 16, 3, 2004
    U, S, V = g.rsvd(_torch_csr(m, n, rp, ci, v, "cuda"), k, p, q, seed, prec=prec)
    U, S, V = (t.cpu().numpy().astype(np.float64) for t in (U, S, V))
    Uo, So, Vo = OR.rsvd(OL.CSR(m, n, rp, ci, v), k, p, q, seed, "f32" if prec == "bf16x3" else "bf16")
    es = sigma_rel_err(S, So)
    eu = cluster_safe_angles(U, Uo, So, 8, rel_gap=1e-2)
    ev = cluster_safe_angles(V, Vo, So, 8, rel_gap=1e-2)
    print(f"CSR {prec} panels: sigma {es:.2e} U {eu:.2e} V {ev:.2e}")
    if prec == "bf16x3":
        assert es <= 1e-5 and eu <= 1e-4 and ev <= 1e-4
    else:
        assert es <= 1e-3 and eu <= 1e-1 and ev <= 1e-1


def test_csr_input_locations_agree_bitwise(g, zipf):
    """Device CSR with the library-built transpose, device CSR with a caller
    transpose, and host CSR: the same kernels on the same arrays."""
    m, n, rp, ci, v = zipf
    k, p, q, seed = 20, 10, 2, 7
    host = _torch_csr(m, n, rp, ci, v, "cpu")
    At = g.csr_transpose(host)
    a = g.rsvd(host.to("cuda"), k, p, q, seed)
    b = g.rsvd(host.to("cuda"), k, p, q, seed, At=At.to("cuda"))
    c = g.rsvd(host, k, p, q, seed)
    d = g.rsvd(host, k, p, q, seed, At=At)
    for x in (b, c, d):
        for s, t in zip(a, x):
            assert torch.equal(s, t)


def test_coo_input(g, zipf):
    """A COO matrix (Section 3.3's format) is converted to the CSR of A and of
    A^T: in row order it runs bitwise like the CSR input; shuffled, with 2% of
    the entries split in two, it is the same matrix summed in another order
    and agrees with the FP64 oracle to the FP32 bar."""
    m, n, rp, ci, v = zipf
    k, p, q, seed = 20, 10, 2, 7
    rows = np.repeat(np.arange(m), np.diff(rp))
    idx = torch.as_tensor(np.stack([rows, np.asarray(ci)]), dtype=torch.int64)
    coo = torch.sparse_coo_tensor(idx, torch.as_tensor(v), size=(m, n))
    a = g.rsvd(_torch_csr(m, n, rp, ci, v, "cpu"), k, p, q, seed)
    b = g.rsvd(coo, k, p, q, seed)
    c = g.rsvd(coo.to("cuda"), k, p, q, seed)
    for x in (b, c):
        for s_, t_ in zip(a, x):
            assert torch.equal(s_, t_)
    rng = np.random.default_rng(11)
    order = rng.permutation(rows.size)
    ri, cj, vv = rows[order], np.asarray(ci)[order], np.asarray(v, np.float32)[order].copy()
    dup = rng.choice(ri.size, size=ri.size // 50, replace=False)
    half = (vv[dup] * np.float32(0.5)).astype(np.float32)
    vv[dup] = half
    idx = torch.as_tensor(np.stack([np.concatenate([ri, ri[dup]]), np.concatenate([cj, cj[dup]])]),
                          dtype=torch.int64)
    shuffled = torch.sparse_coo_tensor(idx, torch.as_tensor(np.concatenate([vv, half])), size=(m, n))
    U, S, V = (t.cpu().numpy().astype(np.float64) for t in g.rsvd(shuffled, k, p, q, seed))
    Uo, So, Vo = OR.rsvd(OL.CSR(m, n, rp, ci, v), k, p, q, seed, "f32")
    assert sigma_rel_err(S, So) <= 1e-5
    assert cluster_safe_angles(U, Uo, So, 8, rel_gap=1e-2) <= 1e-4


def test_csr_rsvd_r350_matches_oracle(g):
    """r = k + p = 350 (the sparse workload's sketch width): the FP64-only Jacobi
    and the global-memory Cholesky."""
    m, n = 6000, 3000
    rp, ci, v = zipf_csr(m, n, 120000, 1005)
    k, p, q, seed = 300, 50, 1, 2005
    U, S, V = g.rsvd(_torch_csr(m, n, rp, ci, v, "cuda"), k, p, q, seed)
    S = S.cpu().numpy().astype(np.float64)
    Uo, So, Vo = OR.rsvd(OL.CSR(m, n, rp, ci, v), k, p, q, seed, "f32")
    assert sigma_rel_err(S, So) <= 1e-5
    U = U.cpu().numpy().astype(np.float64)
    assert cluster_safe_angles(U, Uo, So, 4, rel_gap=1e-2) <= 1e-4


def test_csr_with_empty_rows_and_columns(g):
    rng = np.random.default_rng(5)
    m, n = 3000, 1000
    D = (rng.random((m, n)) < 0.01) * rng.random((m, n))
    D[::7] = 0.0          # empty rows
    D[:, ::5] = 0.0       # empty columns
    D = D.astype(np.float32)
    Ssp = torch.as_tensor(D).to_sparse_csr()
    k, p, q, seed = 16, 8, 2, 11
    U, S, V = g.rsvd(Ssp.to("cuda"), k, p, q, seed)
    Uo, So, Vo = OR.rsvd(D, k, p, q, seed, "f32")
    assert sigma_rel_err(S.cpu().numpy(), So) <= 1e-5
    # V has no weight on the empty columns
    assert float(V[::5].abs().max()) < 1e-6


def test_csr_zero_matrix_gives_zero_spectrum(g):
    m, n = 500, 300
    Z = torch.sparse_csr_tensor(torch.zeros(m + 1, dtype=torch.int32), torch.zeros(0, dtype=torch.int32),
                                torch.zeros(0), size=(m, n))
    U, S, V = g.rsvd(Z.to("cuda"), 5, 5, 1, 3)
    assert float(S.abs().max()) == 0.0
    assert torch.isfinite(U).all() and torch.isfinite(V).all()


def test_csr_cap_too_small_for_the_copies(g, zipf):
    m, n, rp, ci, v = zipf
    from paper_1907_06470_gb300 import _lib
    import ctypes as C
    o = _lib.RsvdOpts(prec=1, refine=1, mb=0, nb=0, n_slots=2, dtype=1, kind=1)
    out = C.c_size_t()
    assert g.load().rsvd_plan_min_cap(m, n, 10, 5, C.byref(o), C.byref(out)) == 0
    plan = g.Plan(m, n, 10, 5, 1, 0, mem_cap=out.value + 4096, kind="csr")
    with pytest.raises(g.RsvdError) as e:
        plan.run(_torch_csr(m, n, rp, ci, v, "cpu"))
    assert "CAP_TOO_SMALL" in str(e.value)
    plan.close()


def _csr_min_cap(g, m, n, k, p, prec="fp32"):
    from paper_1907_06470_gb300 import _lib
    import ctypes as C
    o = _lib.RsvdOpts(prec=_lib.PREC[prec], refine=1, mb=0, nb=0, n_slots=2, dtype=1, kind=1)
    out = C.c_size_t()
    assert g.load().rsvd_plan_min_cap(m, n, k, p, C.byref(o), C.byref(out)) == 0
    return out.value


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_csr_streamed_full_width_blocks_match_in_core_bits(g, zipf, prec):
    """A host CSR over the cap is streamed in full-width row blocks (of A for
    the forward products, of A^T for the transposed ones): every output row is
    summed by the same kernel over the same entries as in core, so the result
    is the same bits (FP32 and 24-bit panels); and it meets the oracle at the
    FP32 bars."""
    m, n, rp, ci, v = zipf
    k, p, q, seed = 20, 10, 2, 2004
    A_bytes = (m + 1) * 4 + len(v) * 8
    cap = _csr_min_cap(g, m, n, k, p, prec) + A_bytes // 2
    Ah = _torch_csr(m, n, rp, ci, v, "cpu")
    plan = g.Plan(m, n, k, p, q, seed, mem_cap=cap, kind="csr", prec=prec)
    Us, Ss, Vs = plan.run(Ah)
    st = plan.stream_stats()
    assert st["tiles_streamed_per_pass"] > 0 and st["h2d_bytes"] > A_bytes
    plan.close()
    Ui, Si, Vi = g.rsvd(_torch_csr(m, n, rp, ci, v, "cuda"), k, p, q, seed, prec=prec)
    assert torch.equal(Ss, Si) and torch.equal(Us, Ui) and torch.equal(Vs, Vi)
    Uo, So, Vo = OR.rsvd(OL.CSR(m, n, rp, ci, v), k, p, q, seed, "f32")
    assert sigma_rel_err(Ss.cpu().numpy(), So) <= 1e-5
    assert cluster_safe_angles(Us.cpu().numpy().astype(np.float64), Uo, So, k) <= 1e-4


@pytest.mark.parametrize("mb,nb", [(3000, 1500), (7001, 5000), (20000, 999)])
def test_csr_streamed_block_cyclic_grid_matches_oracle(g, zipf, mb, nb):
    """Streamed on the block-cyclic grid mb x nb (blocks cut on the host,
    partial products of a row block added in block order), against the oracle:
    under a cap that holds the slots and some resident blocks, and with no cap
    (the block-cyclic map in core: every block resident after the first pass)."""
    m, n, rp, ci, v = zipf
    k, p, q, seed = 20, 10, 2, 2004
    A_bytes = (m + 1) * 4 + len(v) * 8
    cap = _csr_min_cap(g, m, n, k, p) + A_bytes * 3
    plan = g.Plan(m, n, k, p, q, seed, mem_cap=cap, kind="csr", mb=mb, nb=nb)
    U, S, V = (t.cpu().numpy().astype(np.float64) for t in plan.run(_torch_csr(m, n, rp, ci, v, "cpu")))
    st = plan.stream_stats()
    assert st["h2d_bytes"] > 0 and st["tiles_resident"] > 0
    plan.close()
    free = g.Plan(m, n, k, p, q, seed, kind="csr", mb=mb, nb=nb)
    Uf, Sf, Vf = (t.cpu().numpy().astype(np.float64) for t in free.run(_torch_csr(m, n, rp, ci, v, "cpu")))
    stf = free.stream_stats()
    assert stf["tiles_streamed_per_pass"] == 0 and stf["h2d_bytes"] < 3 * A_bytes  # each block copied once
    free.close()
    assert np.array_equal(Sf, S)
    Uo, So, Vo = OR.rsvd(OL.CSR(m, n, rp, ci, v), k, p, q, seed, "f32")
    assert sigma_rel_err(S, So) <= 1e-5
    assert cluster_safe_angles(U, Uo, So, k) <= 1e-4 and cluster_safe_angles(V, Vo, So, k) <= 1e-4


@pytest.mark.parametrize("split,prec", [(True, "fp32"), (False, "fp32"), (True, "bf16x3")])
def test_csr_long_rows_at_segment_boundaries(g, split, prec):
    """Rows of 0, 1, 1023, 1024, 1025, 2048, 2049, 4097 and 30000 entries: the
    segment split (1024 entries per warp, partials added in order) against the
    oracle, with and without the split workspace, FP32 and 24-bit panels."""
    rng = np.random.default_rng(17)
    n, r = 40000, 130
    lens = [0, 1, 1023, 1024, 1025, 2048, 2049, 4097, 30000, 5, 12000]
    rows_c, rows_v = [], []
    for L in lens:
        c = np.sort(rng.choice(n, size=L, replace=False))
        rows_c.append(c)
        rows_v.append(rng.standard_normal(L).astype(np.float32))
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    ci = np.concatenate(rows_c).astype(np.int32)
    v = np.concatenate(rows_v).astype(np.float32)
    m = len(lens)
    X = rng.standard_normal((n, r)).astype(np.float32)
    rnd = (lambda x: x) if prec == "fp32" else OP.round_p24  # the panel both sides multiply
    Ad = _torch_csr(m, n, rp, ci, v, "cuda")
    Y = g.apass(Ad, torch.as_tensor(X, device="cuda"), prec=prec,
                split_long_rows=split).cpu().numpy().astype(np.float64)
    A = OL.CSR(m, n, rp, ci, v)
    Yo = OL.csr_apply(A, rnd(X).astype(np.float64))
    bound = _fp32_product_bound(OL.CSR(m, n, rp, ci, np.abs(v)), rnd(X))
    assert np.all(np.abs(Y - Yo) <= bound + 1e-30)
    assert np.all(Y[0] == 0.0)
    # the transposed pass over the same long rows (columns of A^T)
    At = g.csr_transpose(_torch_csr(m, n, rp, ci, v, "cpu")).to("cuda")
    Yt = rng.standard_normal((n, r)).astype(np.float32)
    Z = g.apass(At, torch.as_tensor(Yt, device="cuda"), trans=True, At=Ad, prec=prec,
                split_long_rows=split).cpu().numpy().astype(np.float64)
    Zo = OL.csr_apply(A, rnd(Yt).astype(np.float64))
    assert np.all(np.abs(Z - Zo) <= _fp32_product_bound(OL.CSR(m, n, rp, ci, np.abs(v)), rnd(Yt)) + 1e-30)
