"""Fused power sweeps (Section 2.2, Eq. (3) evaluated right to left with the
products A^T (A W) grouped, only the n-side orthonormalised) in core and over
streamed row panels, against the oracle's fused range finder."""

import ctypes as C

import numpy as np
import pytest

from oracle import rsvd as OR
from synth import lowrank_plus_noise_torch, prescribed_dense, spectrum_geometric
from tests.metrics import cluster_safe_angles, sigma_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1907_06470_gb300 as g
    g.load()
    return g


def _np(t):
    return t.cpu().numpy().astype(np.float64)


def _min_cap(g, m, n, k, p, prec, dtype):
    from paper_1907_06470_gb300 import _lib
    o = _lib.RsvdOpts(prec=_lib.PREC[prec], refine=1, mb=0, nb=0, n_slots=2, dtype=_lib.DTYPE[dtype], fused=1)
    out = C.c_size_t()
    assert g.load().rsvd_plan_min_cap(m, n, k, p, C.byref(o), C.byref(out)) == 0
    return out.value


@pytest.mark.parametrize("q", [0, 1, 3])
def test_fused_in_core_fp64_matches_oracle(g, q):
    m, n, k, p, seed = 3000, 1200, 20, 10, 2001
    A, _, _ = prescribed_dense(m, n, spectrum_geometric(n, 0.93), 1001)
    plan = g.Plan(m, n, k, p, q, seed, dtype="f64", fused=True)
    U, S, V = (_np(t) for t in plan.run(torch.as_tensor(A, device="cuda")))
    Uo, So, Vo = OR.rsvd_fused_sweeps(A, k, p, q, seed, "f64")
    assert sigma_rel_err(S, So) <= 1e-11
    assert cluster_safe_angles(U, Uo, So, k) <= 1e-9 and cluster_safe_angles(V, Vo, So, k) <= 1e-9


@pytest.fixture(scope="module")
def ooc_case():
    """The out-of-core recipe (low rank + 1e-3 floor) at 12288 x 5000, k 60 p 20 q 2."""
    m, n = 12288, 5000
    A = lowrank_plus_noise_torch(m, n, 2000, 50.0, 1e-3, 1003, 3003).cpu().numpy()
    return m, n, 60, 20, 2, 2003, A


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16"])
def test_fused_streamed_matches_oracle_and_reads_a_q_plus_2_times(g, ooc_case, prec):
    """Streamed fused sweeps: each sweep copies every row panel not resident
    once, so a run moves (q + 2) x the streamed bytes of one pass, and the
    result meets the oracle's fused range finder (FP32 bars for the FP32 and
    split-BF16 plans; reported for BF16)."""
    m, n, k, p, q, seed, A = ooc_case
    Ah = torch.as_tensor(A).pin_memory()
    cap = _min_cap(g, m, n, k, p, prec, "f32") + A.nbytes // 3
    plan = g.Plan(m, n, k, p, q, seed, mem_cap=cap, prec=prec, fused=True)
    U, S, V = (_np(t) for t in plan.run(Ah))
    st = plan.stream_stats()
    per_pass = st["tiles_streamed_per_pass"]
    assert per_pass > 0 and st["tiles_resident"] > 0
    plan.close()
    # the same plan without fusion moves 2q + 2 passes' worth
    plain = g.Plan(m, n, k, p, q, seed, mem_cap=cap, prec=prec)
    plain.run(Ah)
    st2 = plain.stream_stats()
    plain.close()
    # resident tiles cross the link once per run, the others once per pass:
    # h2d = resident + passes x streamed, with q + 2 passes fused, 2q + 2 not.
    # (A plain BF16 plan keeps BF16 copies resident, twice as many tiles, and
    # streams them again for its split-BF16 B^T: there only the total is
    # compared.)
    if prec == "bf16":
        assert st["h2d_bytes"] < st2["h2d_bytes"]
    else:
        streamed = (st2["h2d_bytes"] - st["h2d_bytes"]) // q
        resident = st["h2d_bytes"] - (q + 2) * streamed
        assert streamed > 0 and resident > 0 and resident + streamed == A.nbytes
    Uo, So, Vo = OR.rsvd_fused_sweeps(A, k, p, q, seed, "f32" if prec == "fp32" else "bf16")
    es = sigma_rel_err(S, So)
    eu, ev = cluster_safe_angles(U, Uo, So, k), cluster_safe_angles(V, Vo, So, k)
    print(f"fused streamed {prec}: sigma {es:.2e} U {eu:.2e} V {ev:.2e}")
    if prec == "bf16":
        assert es <= 1e-3
    else:
        assert es <= 1e-5 and eu <= 1e-4 and ev <= 1e-4


def test_fused_streamed_equals_fused_in_core(g, ooc_case):
    """The streamed sweep adds A_I^T (A_I W) panel by panel, the in-core sweep
    forms A W and then A^T (A W): the same sums in another order (FP32 bars)."""
    m, n, k, p, q, seed, A = ooc_case
    cap = _min_cap(g, m, n, k, p, "fp32", "f32") + A.nbytes // 3
    a = g.Plan(m, n, k, p, q, seed, mem_cap=cap, fused=True).run(torch.as_tensor(A).pin_memory())
    b = g.Plan(m, n, k, p, q, seed, fused=True).run(torch.as_tensor(A, device="cuda"))
    Sa, Sb = _np(a[1]), _np(b[1])
    assert sigma_rel_err(Sa, Sb) <= 1e-5
    assert cluster_safe_angles(_np(a[0]), _np(b[0]), Sb, k) <= 1e-4


def test_fused_rejects_narrow_streamed_tiles(g):
    m, n = 4000, 3000
    A, _, _ = prescribed_dense(m, n, spectrum_geometric(n, 0.9), 5, dtype=np.float32)
    cap = _min_cap(g, m, n, 20, 10, "fp32", "f32") + A.nbytes // 3
    plan = g.Plan(m, n, 20, 10, 1, 3, mem_cap=cap, mb=512, nb=512, fused=True)
    with pytest.raises(g.RsvdError) as e:
        plan.run(torch.as_tensor(A).pin_memory())
    assert "UNSUPPORTED" in str(e.value)
