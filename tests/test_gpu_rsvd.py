"""End-to-end parity of the randomized SVD (Section 2.1 steps 1-7, Section 2.2)
against the FP64 oracle on the same seeded inputs."""

import numpy as np
import pytest

from oracle import rsvd as OR
from synth import WORKLOADS, prescribed_dense, spectrum_geometric, spectrum_harmonic_noisy
from tests.metrics import max_principal_angle, sigma_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1907_06470_gb300 as g
    g.load()
    return g


def _run(g, A_np, k, p, q, seed, prec, mb=0, nb=0):
    tdt = torch.float64 if A_np.dtype == np.float64 else torch.float32
    Ad = torch.as_tensor(A_np, dtype=tdt, device="cuda")
    U, S, V = g.rsvd(Ad, k, p, q, seed, prec=prec, mb=mb, nb=nb)
    return (U.cpu().numpy().astype(np.float64), S.cpu().numpy().astype(np.float64),
            V.cpu().numpy().astype(np.float64))


def test_dense_fp64_2000x1000_matches_oracle(g):
    """Full-size FP64 workload: sigma within 1e-11 relative, vectors to FP64 accuracy."""
    w = WORKLOADS["dense_fp64_2000x1000"]
    A, _, _ = prescribed_dense(w.m, w.n, spectrum_geometric(w.n, 0.9), w.data_seed)
    U, S, V = _run(g, A, w.k, w.p, w.q, w.seed, "fp64", mb=w.tile, nb=w.tile)
    Uo, So, Vo = OR.rsvd(A, w.k, w.p, w.q, w.seed, "f64")
    assert sigma_rel_err(S, So) <= 1e-11
    assert max_principal_angle(U, Uo) <= 1e-9
    assert max_principal_angle(V, Vo) <= 1e-9
    # well separated spectrum: vectors agree column by column after the sign rule
    assert np.max(np.abs(U - Uo)) < 1e-9 and np.max(np.abs(V - Vo)) < 1e-9


@pytest.mark.parametrize("tile", [0, 1024])
def test_dense_fp32_scaled_c2_recipe_matches_oracle(g, tile):
    """The 100000x20000 recipe scaled to 8000x4000 (ragged 1024 tiles), FP32 path."""
    m, n, k, p, q, seed = 8000, 4000, 100, 20, 2, 2002
    s = spectrum_harmonic_noisy(n, 1e-4, 3002)
    A, _, _ = prescribed_dense(m, n, s, 1002, dtype=np.float32)
    U, S, V = _run(g, A, k, p, q, seed, "fp32", mb=tile, nb=tile)
    Uo, So, Vo = OR.rsvd(A, k, p, q, seed, "f32")
    assert sigma_rel_err(S, So) <= 1e-5
    assert max_principal_angle(U, Uo) <= 1e-4
    assert max_principal_angle(V, Vo) <= 1e-4


def test_dense_fp32_exact_rank_recovers_spectrum(g):
    m, n, k, p, q = 3000, 1000, 20, 10, 1
    s = np.concatenate([spectrum_geometric(25, 0.8), np.zeros(n - 25)])
    A, U0, V0 = prescribed_dense(m, n, s, 5, dtype=np.float32)
    U, S, V = _run(g, A, k, p, q, 77, "fp32")
    assert sigma_rel_err(S, s[:k]) <= 1e-5
    assert max_principal_angle(U, U0[:, :k]) <= 1e-4


@pytest.mark.parametrize("q", [0, 1, 3])
def test_power_iteration_counts(g, q):
    m, n, k, p = 900, 500, 10, 6
    A, _, _ = prescribed_dense(m, n, 1.0 / np.arange(1, n + 1), 9)
    U, S, V = _run(g, A, k, p, q, 123, "fp64")
    Uo, So, Vo = OR.rsvd(A, k, p, q, 123, "f64")
    assert sigma_rel_err(S, So) <= 1e-11


def test_signs_follow_the_rule(g):
    m, n = 700, 300
    A, _, _ = prescribed_dense(m, n, spectrum_geometric(n, 0.85), 31)
    U, S, V = _run(g, A, 10, 5, 1, 1, "fp64")
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(10)] > 0)


def test_host_resident_input_runs_in_core(g):
    m, n = 1200, 600
    A, _, _ = prescribed_dense(m, n, spectrum_geometric(n, 0.9), 41, dtype=np.float32)
    Ah = torch.as_tensor(A).pin_memory()
    U, S, V = g.rsvd(Ah, 12, 8, 2, 5)
    Ud, Sd, Vd = g.rsvd(torch.as_tensor(A, device="cuda"), 12, 8, 2, 5)
    assert torch.equal(S, Sd) and torch.equal(U, Ud) and torch.equal(V, Vd)


def test_repeated_runs_are_bit_identical(g):
    m, n = 2000, 900
    A, _, _ = prescribed_dense(m, n, spectrum_geometric(n, 0.95), 51, dtype=np.float32)
    Ad = torch.as_tensor(A, device="cuda")
    plan = g.Plan(m, n, 30, 10, 2, 9, mb=512, nb=256)
    a = [t.clone() for t in plan.run(Ad)]
    b = plan.run(Ad)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_automatic_q_matches_oracle(g, prec):
    """Section 2.2 automatic iteration parameter: the same stopping point as the
    oracle (tolerance 1e-3 sits between consecutive changes by a factor >= 1.7)
    and the oracle's result at that point."""
    if prec == "fp64":
        A, _, _ = prescribed_dense(2000, 1000, spectrum_geometric(1000, 0.97), 1001)
        k, p, seed, od, qexp = 20, 10, 2001, "f64", 4
    else:
        A, _, _ = prescribed_dense(4000, 2000, spectrum_harmonic_noisy(2000, 1e-4, 3002), 1002, dtype=np.float32)
        k, p, seed, od, qexp = 50, 10, 2002, "f32", 3
    Ad = torch.as_tensor(A, device="cuda")
    plan = g.Plan(A.shape[0], A.shape[1], k, p, 6, seed, prec=prec, dtype="f64" if prec == "fp64" else "f32",
                  auto_q=True, auto_q_tol=1e-3)
    U, S, V = (t.cpu().numpy().astype(np.float64) for t in plan.run(Ad))
    qu = plan.info()["q_used"]
    plan.close()
    Uo, So, Vo, quo = OR.rsvd_auto_q(A, k, p, 6, seed, 1e-3, od)
    assert quo == qexp and qu == quo
    assert sigma_rel_err(S, So) <= (1e-11 if prec == "fp64" else 1e-5)
    assert max_principal_angle(U, Uo) <= (1e-9 if prec == "fp64" else 1e-4)
    # and the same as a fixed-q plan with that count
    Uf, Sf, Vf = (t.cpu().numpy().astype(np.float64) for t in g.rsvd(Ad, k, p, qu, seed, prec=prec))
    assert sigma_rel_err(S, Sf) <= (1e-12 if prec == "fp64" else 1e-6)


def test_automatic_q_bf16_refines_the_final_pass(g):
    A, _, _ = prescribed_dense(4000, 2000, spectrum_harmonic_noisy(2000, 1e-4, 3002), 1002, dtype=np.float32)
    Ad = torch.as_tensor(A, device="cuda")
    plan = g.Plan(4000, 2000, 50, 10, 6, 2002, prec="bf16", auto_q=True, auto_q_tol=1e-3)
    U, S, V = plan.run(Ad)
    qu = plan.info()["q_used"]
    plan.close()
    assert 2 <= qu <= 4
    Uo, So, Vo = OR.rsvd(A, 50, 10, qu, 2002, "bf16")
    assert sigma_rel_err(S.cpu().numpy(), So) <= 5e-4


def test_bf16_plan_on_device_then_host_input(g):
    """One BF16 plan run first on a device A (which makes the plan's BF16 copy
    of A) and then on the same A in pinned host memory (copied to the device
    in core): both runs read the same operands, so the results are the same
    bits, and both meet the oracle at the BF16 plan's bound."""
    m, n, k, p, q, seed = 3000, 1500, 30, 10, 2, 77
    A, _, _ = prescribed_dense(m, n, spectrum_harmonic_noisy(n, 1e-4, 3), 4, dtype=np.float32)
    plan = g.Plan(m, n, k, p, q, seed, prec="bf16")
    a = [t.clone() for t in plan.run(torch.as_tensor(A, device="cuda"))]
    assert plan.info()["bf16_copy"] == 1
    b = plan.run(torch.as_tensor(A).pin_memory())
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    Uo, So, Vo = OR.rsvd(A, k, p, q, seed, "bf16")
    assert sigma_rel_err(b[1].cpu().numpy(), So) <= 1e-3
    plan.close()
