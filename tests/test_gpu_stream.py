"""Out-of-core runs (host matrix streamed in block-cyclic tiles under a device
memory cap) against the oracle and against the in-core path."""

import ctypes as C

import numpy as np
import pytest

from oracle import rsvd as OR
from synth import prescribed_dense, spectrum_geometric
from tests.metrics import max_principal_angle, sigma_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1907_06470_gb300 as g
    g.load()
    return g


def _min_cap(g, m, n, k, p, prec, dtype, mb=0, nb=0):
    from paper_1907_06470_gb300 import _lib
    o = _lib.RsvdOpts(prec=_lib.PREC[prec], refine=1, mb=mb, nb=nb, n_slots=2, dtype=_lib.DTYPE[dtype])
    out = C.c_size_t()
    assert g.load().rsvd_plan_min_cap(m, n, k, p, C.byref(o), C.byref(out)) == 0
    return out.value


@pytest.mark.parametrize("tile", [512, 700])
def test_streamed_fp64_matches_oracle(g, tile):
    m, n, k, p, q, seed = 3000, 2000, 20, 10, 2, 2001
    A, _, _ = prescribed_dense(m, n, spectrum_geometric(n, 0.9), 1001)
    a_bytes = A.nbytes
    cap = _min_cap(g, m, n, k, p, "fp64", "f64", tile, tile) + a_bytes // 2
    plan = g.Plan(m, n, k, p, q, seed, mem_cap=cap, dtype="f64", mb=tile, nb=tile)
    Ah = torch.as_tensor(A).pin_memory()
    U, S, V = (t.cpu().numpy() for t in plan.run(Ah))
    st = plan.stream_stats()
    assert st["h2d_bytes"] > 0 and st["tiles_resident"] > 0 and st["tiles_streamed_per_pass"] > 0
    # every pass re-streams the non-resident tiles; resident ones are copied once
    Uo, So, Vo = OR.rsvd(A, k, p, q, seed, "f64")
    assert sigma_rel_err(S, So) <= 1e-11
    assert max_principal_angle(U, Uo) <= 1e-9 and max_principal_angle(V, Vo) <= 1e-9


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_streamed_matches_in_core(g, prec):
    m, n, k, p, q, seed = 4000, 3000, 40, 12, 2, 77
    A, _, _ = prescribed_dense(m, n, spectrum_geometric(n, 0.97), 5, dtype=np.float32)
    cap = _min_cap(g, m, n, k, p, prec, "f32", 1024, 1024) + A.nbytes // 3
    Ah = torch.as_tensor(A).pin_memory()
    plan = g.Plan(m, n, k, p, q, seed, mem_cap=cap, prec=prec, mb=1024, nb=1024)
    Us, Ss, Vs = (t.cpu().numpy().astype(np.float64) for t in plan.run(Ah))
    assert plan.stream_stats()["h2d_bytes"] > A.nbytes  # more than one pass went over the link
    Ui, Si, Vi = (t.cpu().numpy().astype(np.float64) for t in
                  g.rsvd(torch.as_tensor(A, device="cuda"), k, p, q, seed, prec=prec))
    tol = 1e-5 if prec == "fp32" else 5e-4
    assert sigma_rel_err(Ss, Si) <= tol
    assert max_principal_angle(Us, Ui) <= (1e-4 if prec == "fp32" else 1e-2)


def test_bf16_plan_keeps_bf16_copies_resident(g):
    """A streamed BF16 plan keeps its resident tiles as BF16 copies: 12 MB
    more of cap hold six more 1024 x 1024 tiles (2 MB each, not 4 MB), the
    link carries fewer bytes, and the result is the same bits as with fewer
    resident tiles (the copy holds the very operands the FP32 tile is
    converted to)."""
    m, n, k, p, q, seed = 8192, 3072, 40, 12, 2, 77
    A, _, _ = prescribed_dense(m, n, spectrum_geometric(n, 0.97), 5, dtype=np.float32)
    Ah = torch.as_tensor(A).pin_memory()
    base = _min_cap(g, m, n, k, p, "bf16", "f32", 1024, 1024) + 24 * 2**20
    runs = []
    for cap in (base, base + 12 * 2**20):
        plan = g.Plan(m, n, k, p, q, seed, mem_cap=cap, prec="bf16", mb=1024, nb=1024)
        out = [t.cpu() for t in plan.run(Ah)]
        runs.append((out, plan.stream_stats()))
        plan.close()
    (a, sa), (b, sb) = runs
    assert 5 <= sb["tiles_resident"] - sa["tiles_resident"] <= 7
    assert sb["h2d_bytes"] < sa["h2d_bytes"]
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_tiles_smaller_than_a_row(g):
    """A cap so small that a tile is 16 x 16, less than one row of A."""
    m, n, k, p, q, seed = 100, 80, 6, 4, 1, 3
    A, _, _ = prescribed_dense(m, n, spectrum_geometric(n, 0.8), 9)
    cap = _min_cap(g, m, n, k, p, "fp64", "f64", 16, 16) + 3 * 16 * 16 * 8 + 4096
    plan = g.Plan(m, n, k, p, q, seed, mem_cap=cap, dtype="f64", mb=16, nb=16)
    U, S, V = (t.cpu().numpy() for t in plan.run(torch.as_tensor(A).pin_memory()))
    assert plan.stream_stats()["tiles_streamed_per_pass"] > 0
    Uo, So, Vo = OR.rsvd(A, k, p, q, seed, "f64")
    assert sigma_rel_err(S, So) <= 1e-11


def test_cap_below_the_workspace_is_rejected(g):
    m, n = 2000, 1000
    ws = _min_cap(g, m, n, 10, 5, "fp32", "f32")
    with pytest.raises(g.RsvdError) as e:
        g.Plan(m, n, 10, 5, 1, 0, mem_cap=ws // 2)
    assert "CAP_TOO_SMALL" in str(e.value)
