"""Host-side checks of the C ABI: the library loads, exports every declared
symbol, and its host-only logic (tile map, argument checks, planner sizes)
matches the oracle.  No GPU compute is called here."""

import ctypes as C
import os
import re

import pytest

from oracle import tiles as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = ""
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            with open(os.path.join(ROOT, "include", name)) as fh:
                text += fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:rsvd_status|size_t|void|const char\*|unsigned long long)\s+(rsvd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "rsvd_plan" in names and "rsvd_run" in names and len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1907_06470_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared_functions()


@pytest.mark.parametrize("m,n,mb,nb,S", [(10, 7, 3, 2, 2), (100000, 20000, 4096, 4096, 2),
                                         (600000, 100000, 8192, 8192, 3), (1, 1, 5, 5, 1), (0, 4, 2, 2, 2)])
def test_tile_map_is_bit_exact_with_oracle(m, n, mb, nb, S):
    import paper_1907_06470_gb300 as g
    assert g.tile_map(m, n, mb, nb, S) == T.tile_map(m, n, mb, nb, S)


def test_tile_map_rejects_bad_arguments(lib):
    cnt = C.c_int64()
    assert lib.rsvd_tile_map(10, 10, 0, 2, 1, None, 0, C.byref(cnt)) == 1
    assert lib.rsvd_tile_map(10, 10, 2, 2, 0, None, 0, C.byref(cnt)) == 1
    assert b"rsvd_tile_map" in lib.rsvd_last_error()


def test_plan_argument_rules_checked_before_any_device_call(lib):
    from paper_1907_06470_gb300 import _lib
    h = C.c_void_p()
    # k + p > min(m, n)
    assert lib.rsvd_plan(100, 20, 15, 10, 2, 1, 0, None, C.byref(h)) == 1
    # k + p > 256
    assert lib.rsvd_plan(10000, 10000, 250, 10, 2, 1, 0, None, C.byref(h)) == 1
    # FP64 precision with FP32 data
    o = _lib.RsvdOpts(prec=0, refine=1, mb=0, nb=0, n_slots=2, dtype=1)
    assert lib.rsvd_plan(100, 50, 5, 5, 1, 1, 0, C.byref(o), C.byref(h)) == 1
    assert h.value is None


def test_min_cap_grows_with_the_problem(lib):
    from paper_1907_06470_gb300 import _lib
    out = C.c_size_t()
    o = _lib.RsvdOpts(prec=1, refine=1, mb=4096, nb=4096, n_slots=2, dtype=1)
    assert lib.rsvd_plan_min_cap(100000, 20000, 100, 20, C.byref(o), C.byref(out)) == 0
    big = out.value
    assert lib.rsvd_plan_min_cap(10000, 2000, 100, 20, C.byref(o), C.byref(out)) == 0
    assert out.value < big
    # the panels alone: 2 m-panels + 3 n-panels of r=120 FP32 columns
    assert big >= (2 * 100000 + 3 * 20000) * 120 * 4


def test_status_strings(lib):
    for code, name in {0: b"RSVD_OK", 5: b"RSVD_ERR_NOT_SPD", 7: b"RSVD_ERR_TIMEOUT"}.items():
        assert lib.rsvd_status_str(code) == name


def _csr_ptrs(rp, ci, v):
    import numpy as np
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    return rp, ci, v


def _lib_transpose(lib, m, n, rp, ci, v):
    import numpy as np
    rp, ci, v = _csr_ptrs(rp, ci, v)
    nnz = int(rp[-1]) if rp.size else 0
    trp = np.full(n + 1, -7, dtype=np.int32)
    tci = np.full(max(nnz, 1), -7, dtype=np.int32)
    tv = np.full(max(nnz, 1), np.nan, dtype=np.float32)
    P = lambda a: a.ctypes.data_as(C.c_void_p)
    st = lib.rsvd_csr_transpose(m, n, P(rp), P(ci), P(v), P(trp), P(tci), P(tv))
    return st, trp, tci[:nnz], tv[:nnz]


@pytest.mark.parametrize("m,n,nnz,seed", [(300, 200, 1000, 3), (20000, 5000, 400000, 1004),
                                          (200000, 50000, 4_000_000, 1104)])
def test_csr_transpose_is_bit_exact_with_oracle(lib, m, n, nnz, seed):
    """The library's host transpose (threaded for large nnz) against the oracle's
    entry-by-entry scatter, on the sparse workload's generator."""
    import numpy as np
    from synth import zipf_csr
    rp, ci, v = zipf_csr(m, n, nnz, seed)
    st, trp, tci, tv = _lib_transpose(lib, m, n, rp, ci, v)
    assert st == 0
    if nnz <= 400000:
        orp, oci, ov = T.csr_transpose(m, n, rp, ci, v)
    else:  # the oracle's Python scatter is slow at 4e6 entries: use its definition via a stable sort
        order = np.lexsort((np.repeat(np.arange(m), np.diff(rp)), ci))
        oci = np.repeat(np.arange(m), np.diff(rp))[order]
        ov = v[order]
        orp = np.concatenate([[0], np.cumsum(np.bincount(ci, minlength=n))])
    assert np.array_equal(trp, orp) and np.array_equal(tci, oci) and np.array_equal(tv.view(np.uint32), np.asarray(ov, np.float32).view(np.uint32))


def test_csr_transpose_edge_cases(lib):
    import numpy as np
    # empty rows and columns, one dense row, nnz = 0
    rp = [0, 0, 3, 3, 4]
    ci = [0, 2, 5, 5]
    v = [1.0, 2.0, 3.0, 4.0]
    st, trp, tci, tv = _lib_transpose(lib, 4, 6, rp, ci, v)
    assert st == 0
    assert trp.tolist() == [0, 1, 1, 2, 2, 2, 4]
    assert tci.tolist() == [1, 1, 1, 3] and tv.tolist() == [1.0, 2.0, 3.0, 4.0]
    st, trp, tci, tv = _lib_transpose(lib, 3, 2, [0, 0, 0, 0], [], [])
    assert st == 0 and trp.tolist() == [0, 0, 0]
    # a column index out of range and a decreasing rowptr are rejected
    assert _lib_transpose(lib, 2, 3, [0, 1, 2], [0, 3], [1.0, 1.0])[0] == 1
    assert _lib_transpose(lib, 2, 3, [0, 2, 1], [0, 1], [1.0, 1.0])[0] == 1


def _lib_coo(lib, m, n, ri, ci, v, bits):
    import numpy as np
    it = np.int32 if bits == 32 else np.int64
    ri = np.ascontiguousarray(ri, dtype=it)
    ci = np.ascontiguousarray(ci, dtype=it)
    v = np.ascontiguousarray(v, dtype=np.float32)
    nnz = v.size
    rp = np.full(m + 1, -7, dtype=np.int32)
    oci = np.full(max(nnz, 1), -7, dtype=np.int32)
    ov = np.full(max(nnz, 1), np.nan, dtype=np.float32)
    P = lambda a: a.ctypes.data_as(C.c_void_p)
    st = lib.rsvd_coo_to_csr(m, n, nnz, bits, P(ri), P(ci), P(v), P(rp), P(oci), P(ov))
    return st, rp, oci[:nnz], ov[:nnz]


@pytest.mark.parametrize("m,n,nnz,bits,seed", [(300, 200, 1000, 32, 3), (300, 200, 1000, 64, 4),
                                               (20000, 5000, 400000, 64, 1004),
                                               (200000, 50000, 4_000_000, 32, 1104)])
def test_coo_to_csr_is_bit_exact_with_oracle(lib, m, n, nnz, bits, seed):
    """The library's host COO -> CSR (threaded for large nnz) against the
    oracle's row-by-row bucketing, on the sparse workload's entries given in a
    shuffled order with some of them split into repeated entries."""
    import numpy as np
    from synth import zipf_csr
    rp, ci, v = zipf_csr(m, n, nnz, seed)
    rows = np.repeat(np.arange(m), np.diff(rp))
    rng = np.random.default_rng(seed)
    order = rng.permutation(rows.size)
    ri, cj, vv = rows[order], np.asarray(ci)[order], np.asarray(v, np.float32)[order]
    dup = rng.choice(ri.size, size=ri.size // 50, replace=False)   # split 2% of the entries in two
    ri = np.concatenate([ri, ri[dup]])
    cj = np.concatenate([cj, cj[dup]])
    half = (vv[dup] * np.float32(0.5)).astype(np.float32)
    vv = vv.copy()
    vv[dup] = half
    vv = np.concatenate([vv, half])
    st, orp, oci, ov = _lib_coo(lib, m, n, ri, cj, vv, bits)
    assert st == 0
    if nnz <= 400000:
        erp, eci, ev = T.coo_to_csr(m, n, ri, cj, vv)
    else:  # the oracle's Python loop is slow at 4e6 entries: its definition via a stable sort
        perm = np.argsort(ri, kind="stable")
        eci, ev = cj[perm], vv[perm]
        erp = np.concatenate([[0], np.cumsum(np.bincount(ri, minlength=m))])
    assert np.array_equal(orp, erp) and np.array_equal(oci, eci)
    assert np.array_equal(ov.view(np.uint32), np.asarray(ev, np.float32).view(np.uint32))


def test_coo_to_csr_edge_cases(lib):
    import numpy as np
    st, rp, ci, v = _lib_coo(lib, 3, 2, [], [], [], 32)
    assert st == 0 and rp.tolist() == [0, 0, 0, 0]
    st, rp, ci, v = _lib_coo(lib, 0, 4, [], [], [], 64)
    assert st == 0 and rp.tolist() == [0]
    # the hand example of the oracle's pin
    st, rp, ci, v = _lib_coo(lib, 3, 4, [2, 0, 2, 1, 2, 0], [1, 3, 0, 2, 1, 0], [1, 2, 3, 4, 5, 6], 64)
    assert st == 0 and rp.tolist() == [0, 2, 3, 6]
    assert ci.tolist() == [3, 0, 2, 1, 0, 1] and v.tolist() == [2.0, 6.0, 4.0, 1.0, 3.0, 5.0]
    # indices out of range (row, column, negative, 64-bit beyond 2^32) and bad index widths
    assert _lib_coo(lib, 3, 4, [3], [0], [1.0], 32)[0] == 1
    assert _lib_coo(lib, 3, 4, [0], [4], [1.0], 32)[0] == 1
    assert _lib_coo(lib, 3, 4, [-1], [0], [1.0], 64)[0] == 1
    assert _lib_coo(lib, 3, 4, [0], [(1 << 32) + 1], [1.0], 64)[0] == 1
    z = np.zeros(1, dtype=np.int32)
    P = lambda a: a.ctypes.data_as(C.c_void_p)
    rp = np.zeros(4, dtype=np.int32)
    f = np.zeros(1, dtype=np.float32)
    assert lib.rsvd_coo_to_csr(3, 4, 1, 16, P(z), P(z), P(f), P(rp), P(z), P(f)) == 1
    assert lib.rsvd_coo_to_csr(3, 4, 1, 32, None, P(z), P(f), P(rp), P(z), P(f)) == 1


def test_coo_binding_converts_torch_coo(lib):
    """The binding's coo_to_csr on an uncoalesced host torch COO tensor (int64
    indices, repeats): the CSR of A and of A^T the library builds, against the
    oracle (host only, no GPU call)."""
    import numpy as np
    torch = pytest.importorskip("torch")
    import paper_1907_06470_gb300 as g
    rng = np.random.default_rng(21)
    m, n, nnz = 40, 25, 300
    ri = rng.integers(0, m, nnz)
    ci = rng.integers(0, n, nnz)
    v = rng.standard_normal(nnz).astype(np.float32)
    coo = torch.sparse_coo_tensor(torch.as_tensor(np.stack([ri, ci])), torch.as_tensor(v), size=(m, n))
    assert not coo.is_coalesced()
    A = g.coo_to_csr(coo)
    At = g.coo_to_csr(coo, transpose=True)
    for got, (erp, eci, ev), shape in ((A, T.coo_to_csr(m, n, ri, ci, v), (m, n)),
                                       (At, T.coo_to_csr(n, m, ci, ri, v), (n, m))):
        assert tuple(got.shape) == shape
        assert np.array_equal(got.crow_indices().numpy(), erp)
        assert np.array_equal(got.col_indices().numpy(), eci)
        assert np.array_equal(got.values().numpy().view(np.uint32), ev.view(np.uint32))
    with pytest.raises(TypeError):
        g.coo_to_csr(coo.double())


def test_binding_maps_16bit_dtypes():
    torch = pytest.importorskip("torch")
    import paper_1907_06470_gb300 as g
    from paper_1907_06470_gb300 import _lib
    codes = {t: g._dtype_code(torch.zeros(1, dtype=t)) for t in
             (torch.float64, torch.float32, torch.bfloat16, torch.float16)}
    assert codes == {torch.float64: _lib.DTYPE["f64"], torch.float32: _lib.DTYPE["f32"],
                     torch.bfloat16: _lib.DTYPE["bf16"], torch.float16: _lib.DTYPE["f16"]}
    with open(os.path.join(ROOT, "include", "rsvd.h")) as fh:
        hdr = fh.read()
    for name, val in (("F64", 0), ("F32", 1), ("BF16", 2), ("F16", 3)):
        assert re.search(rf"RSVD_{name} = {val}\b", hdr)
        assert _lib.DTYPE[name.lower()] == val
    with pytest.raises(TypeError):
        g._dtype_code(torch.zeros(1, dtype=torch.int32))


def test_csr_plan_rules(lib):
    from paper_1907_06470_gb300 import _lib
    h = C.c_void_p()
    # CSR plans take r up to 512, FP32 values, and FP32, BF16 or BF16X3 precision
    o = _lib.RsvdOpts(prec=1, refine=1, mb=0, nb=0, n_slots=2, dtype=1, kind=1)
    out = C.c_size_t()
    assert lib.rsvd_plan_min_cap(100000, 50000, 300, 50, C.byref(o), C.byref(out)) == 0
    fp32_cap = out.value
    o513 = _lib.RsvdOpts(prec=1, refine=1, mb=0, nb=0, n_slots=2, dtype=1, kind=1)
    assert lib.rsvd_plan_min_cap(100000, 50000, 500, 13, C.byref(o513), C.byref(out)) == 1
    # the compact panels on top, for the larger side (ldr 352): BF16 2 bytes per
    # value; 24 bits in 384-byte groups of 128 values (3 groups per row)
    for prec, row_bytes in ((2, 352 * 2), (3, 3 * 384)):
        oc = _lib.RsvdOpts(prec=prec, refine=1, mb=0, nb=0, n_slots=2, dtype=1, kind=1)
        assert lib.rsvd_plan_min_cap(100000, 50000, 300, 50, C.byref(oc), C.byref(out)) == 0
        assert 0 <= out.value - fp32_cap - 100000 * row_bytes <= 2048
    for prec, dtype in ((4, 1), (0, 0), (1, 0)):  # FP8, FP64
        ob = _lib.RsvdOpts(prec=prec, refine=1, mb=0, nb=0, n_slots=2, dtype=dtype, kind=1)
        assert lib.rsvd_plan(1000, 500, 10, 5, 1, 1, 0, C.byref(ob), C.byref(h)) in (1, 8)
        assert h.value is None


def test_csr_apass_workspace_sizes(lib):
    """FP32 passes need the split-row workspace only; BF16 / BF16X3 passes add
    the compact panel (K rows: round_up(r, 4) BF16 values, or 384 bytes per
    group of 128 values at 24 bits)."""
    nnz, K, r = 10_000_000, 40000, 350
    base = lib.rsvd_spmm_workspace(nnz, r)
    assert lib.rsvd_csr_apass_workspace(nnz, K, r, 1) == base
    for prec, row_bytes in ((2, 352 * 2), (3, 3 * 384)):
        extra = lib.rsvd_csr_apass_workspace(nnz, K, r, prec) - base
        assert K * row_bytes <= extra <= K * row_bytes + 1024
    assert lib.rsvd_csr_apass_workspace(nnz, K, 0, 2) == 0


def _ckpt_header(step=3, corrupt=False, **kw):
    """A checkpoint header in the library's layout, with its FNV-1a checksum."""
    import struct
    f = dict(m=1000, n=800, k=20, p=10, q=2, r=30, ldr=32, prec=1, dtype=1, kind=0, seed=7, fingerprint=99,
             step=step, panel_rows=800, panel_bytes=800 * 32 * 4, panel_checksum=0)
    f.update(kw)
    fmt = "<8sII" + "qq" + "8i" + "QQ" + "ii" + "q" + "QQQ"
    def pack(hc):
        return struct.pack(fmt, b"RSVDCKP1", 1, struct.calcsize(fmt), f["m"], f["n"], f["k"], f["p"], f["q"],
                           f["r"], f["ldr"], f["prec"], f["dtype"], f["kind"], f["seed"], f["fingerprint"],
                           f["step"], 0, f["panel_rows"], f["panel_bytes"], f["panel_checksum"], hc)
    h = 1469598103934665603
    for b in pack(0):
        h = ((h ^ b) * 1099511628211) & (2 ** 64 - 1)
    data = bytearray(pack(h))
    if corrupt:
        data[20] ^= 1
    return bytes(data)


def test_checkpoint_header_is_read_and_validated(lib, tmp_path):
    """Section 3.8 persistence: the header places the basis in the execution plan."""
    import paper_1907_06470_gb300 as g
    path = tmp_path / "ck.bin"
    path.write_bytes(_ckpt_header(step=3))
    info = g.checkpoint_info(path)
    assert (info["m"], info["n"], info["k"], info["p"], info["q"], info["r"]) == (1000, 800, 20, 10, 2, 30)
    assert info["step"] == 3 and info["seed"] == 7 and info["fingerprint"] == 99 and info["panel_rows"] == 800
    for bad in (_ckpt_header(corrupt=True), _ckpt_header()[:40], b"garbage" * 20):
        path.write_bytes(bad)
        with pytest.raises(g.RsvdError):
            g.checkpoint_info(path)
    with pytest.raises(g.RsvdError):
        g.checkpoint_info(tmp_path / "missing.bin")


def test_fused_sweep_plan_rules(lib):
    """Fused sweeps: dense plans with a fixed q and a precision other than FP8
    (checked on the host before any device call)."""
    from paper_1907_06470_gb300 import _lib
    h = C.c_void_p()
    out = C.c_size_t()
    ok = _lib.RsvdOpts(prec=1, refine=1, mb=0, nb=0, n_slots=2, dtype=1, fused=1)
    assert lib.rsvd_plan_min_cap(1000, 500, 10, 5, C.byref(ok), C.byref(out)) == 0
    for bad in (dict(kind=1), dict(prec=4), dict(auto_q=1)):
        kw = dict(prec=1, refine=1, mb=0, nb=0, n_slots=2, dtype=1, fused=1)
        kw.update(bad)
        o = _lib.RsvdOpts(**kw)
        assert lib.rsvd_plan(1000, 500, 10, 5, 1, 1, 0, C.byref(o), C.byref(h)) == 8
        assert h.value is None


def test_opts_layout_matches_the_header():
    """The binding's rsvd_opts mirrors the header's field order and size."""
    from paper_1907_06470_gb300 import _lib
    assert [f for f, _ in _lib.RsvdOpts._fields_] == ["prec", "refine", "mb", "nb", "n_slots", "dtype", "kind",
                                                      "auto_q", "auto_q_tol", "fused", "reserved"]
    assert C.sizeof(_lib.RsvdOpts) == 56


def test_prefetch_rejects_null_arguments_on_the_host(lib):
    """rsvd_plan_prefetch checks its arguments before touching a plan or a GPU."""
    from paper_1907_06470_gb300 import _lib
    d = _lib.RsvdMatrix()
    assert lib.rsvd_plan_prefetch(None, None) == 1
    assert lib.rsvd_plan_prefetch(None, C.byref(d)) == 1
