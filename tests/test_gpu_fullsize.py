"""Parity at the full sizes of the five workloads, in the configuration the
benchmark times (Section 2.1 steps 1-7 with the power scheme of Section 2.2;
Section 3.3 for the sparse workload).

* dense 100000 x 20000 FP32 (8 GB), k 100, p 20, q 2, 4096^2 tiles: the FP32
  plan and the split-BF16 plan against the FP64 oracle at the FP32 bars
  (sigma 1e-5 relative, largest principal angle 1e-4), the BF16 plan
  reported (its passes round A to 8 significant bits);
* differentiable 20000 x 10000: the forward rSVD against the oracle, and the
  adjoint on identical inputs against the oracle's adjoint;
* sparse 5e6 x 1e6 with 5e8 entries, r = 350: the oracle cannot run the
  whole rSVD in seconds, so sampled rows of A O and of A^T Y are computed
  entry by entry by the oracle, and the final factors are checked through
  properties that hold at any size (orthonormality, A^T U = V S);
* the out-of-core recipe (low rank + 1e-3 floor, r = 240) streamed under a
  cap, scaled to a size the oracle finishes quickly.
"""

import ctypes as C

import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import gaussian as OG
from oracle import rsvd as OR
from synth import WORKLOADS, lowrank_plus_noise_torch, prescribed_dense_torch, spectrum_harmonic_noisy
from tests.metrics import cluster_safe_angles, max_principal_angle, sigma_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1907_06470_gb300 as g
    g.load()
    return g


def _np(t):
    return t.cpu().numpy().astype(np.float64)


# ---- dense 100000 x 20000 ----------------------------------------------------------

@pytest.fixture(scope="module")
def dense_full():
    w = WORKLOADS["dense_fp32_100000x20000"]
    A = prescribed_dense_torch(w.m, w.n, spectrum_harmonic_noisy(w.n, 1e-4, w.noise_seed), w.data_seed)
    torch.cuda.synchronize()
    A_host = A.cpu().numpy()
    return w, A, A_host


@pytest.fixture(scope="module")
def oracle_f32(dense_full):
    w, _, A_host = dense_full
    return OR.rsvd(A_host, w.k, w.p, w.q, w.seed, "f32")


@pytest.fixture(scope="module")
def oracle_bf16(dense_full):
    w, _, A_host = dense_full
    return OR.rsvd(A_host, w.k, w.p, w.q, w.seed, "bf16")


def _dense_run(g, w, A, prec):
    plan = g.Plan(w.m, w.n, w.k, w.p, w.q, w.seed, prec=prec, mb=w.tile, nb=w.tile)
    U, S, V = plan.run(A)
    out = _np(U), _np(S), _np(V)
    plan.close()
    return out


def _errors(U, S, V, ref, k):
    Uo, So, Vo = ref
    return (sigma_rel_err(S, So), cluster_safe_angles(U, Uo, So, k), cluster_safe_angles(V, Vo, So, k))


def test_dense_full_fp32_matches_oracle(g, dense_full, oracle_f32):
    w, A, _ = dense_full
    U, S, V = _dense_run(g, w, A, "fp32")
    es, eu, ev = _errors(U, S, V, oracle_f32, w.k)
    print(f"fp32: sigma {es:.2e} U {eu:.2e} V {ev:.2e}")
    assert es <= 1e-5 and eu <= 1e-4 and ev <= 1e-4


def test_dense_full_split_bf16_meets_the_fp32_bars(g, dense_full, oracle_bf16):
    """Every A-pass in split BF16 (three tensor-core products, about 16
    significant bits per operand): the accuracy-matched tensor-core schedule."""
    w, A, _ = dense_full
    U, S, V = _dense_run(g, w, A, "bf16x3")
    es, eu, ev = _errors(U, S, V, oracle_bf16, w.k)
    print(f"bf16x3: sigma {es:.2e} U {eu:.2e} V {ev:.2e}")
    assert es <= 1e-5 and eu <= 1e-4 and ev <= 1e-4


def test_dense_full_bf16_reported(g, dense_full, oracle_bf16):
    """The BF16 plan (the benchmark's headline path): BF16 range finder, split-BF16
    B^T.  Reported against the oracle; bounded at the level the 8000 x 4000
    instance of the recipe shows, with orthonormal factors."""
    w, A, _ = dense_full
    U, S, V = _dense_run(g, w, A, "bf16")
    es, eu, ev = _errors(U, S, V, oracle_bf16, w.k)
    print(f"bf16: sigma {es:.2e} U {eu:.2e} V {ev:.2e}")
    I = np.eye(w.k)
    assert np.abs(U.T @ U - I).max() <= 1e-4 and np.abs(V.T @ V - I).max() <= 1e-4
    assert es <= 1e-3 and eu <= 5e-2 and ev <= 5e-2


# ---- differentiable 20000 x 10000 --------------------------------------------------

def test_diff_full_forward_matches_oracle(g):
    w = WORKLOADS["dense_fp32_20000x10000_diff"]
    s = 10.0 * 0.95 ** np.arange(w.n)
    A = prescribed_dense_torch(w.m, w.n, s, w.data_seed)
    U, S, V = _dense_run(g, w, A, "fp32")
    Uo, So, Vo = OR.rsvd(A.cpu().numpy(), w.k, w.p, w.q, w.seed, "f32")
    assert sigma_rel_err(S, So) <= 1e-5
    assert max_principal_angle(U, Uo) <= 1e-4 and max_principal_angle(V, Vo) <= 1e-4


def test_diff_full_adjoint_on_identical_inputs(g):
    """dA (20000 x 10000) of the workload's loss sum_i w_i s_i + ||U_k^T X||_F^2
    at orthonormal U (20000 x 64), V (10000 x 64) and s_i = 10 0.95^(i-1):
    dU = 2 X X^T U, dS = w, dV = 0, the same FP32 inputs on both sides."""
    w = WORKLOADS["dense_fp32_20000x10000_diff"]
    m, n, k = w.m, w.n, w.k
    rng = np.random.default_rng(w.data_seed)
    U = np.linalg.qr(rng.standard_normal((m, k)))[0].astype(np.float32)
    V = np.linalg.qr(rng.standard_normal((n, k)))[0].astype(np.float32)
    S = (10.0 * 0.95 ** np.arange(k)).astype(np.float32)
    X = np.random.default_rng(4005).standard_normal((m, 32))
    dU = (2.0 * X @ (X.T @ U.astype(np.float64))).astype(np.float32)
    dS = np.random.default_rng(5005).uniform(size=k).astype(np.float32)
    plan = g.Plan(m, n, k, w.p, w.q, w.seed, prec="fp32", mb=w.tile, nb=w.tile)
    dev = lambda x: torch.as_tensor(x, device="cuda")
    dA = plan.backward(dev(U), dev(S), dev(V), dev(dU), dev(dS), None).cpu().numpy().astype(np.float64)
    plan.close()
    ref = AD.svd_adjoint(*(x.astype(np.float64) for x in (U, S, V, dU, dS)), None)
    assert np.linalg.norm(dA - ref) <= 2e-5 * np.linalg.norm(ref)


# ---- sparse 5e6 x 1e6, 5e8 entries -------------------------------------------------

@pytest.fixture(scope="module")
def sparse_full(g):
    from synth import zipf_csr_torch
    w = WORKLOADS["csr_fp32_5000000x1000000"]
    rp, ci, v = zipf_csr_torch(w.m, w.n, 500_000_000, w.data_seed)
    host = (rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy())
    A = torch.sparse_csr_tensor(rp, ci, v, size=(w.m, w.n))
    At = g.csr_transpose(torch.sparse_csr_tensor(*(torch.as_tensor(x) for x in host), size=(w.m, w.n))).to("cuda")
    return w, A, At, host


def _row_entries(host, i):
    rp, ci, v = host
    return ci[rp[i]:rp[i + 1]].astype(np.int64), v[rp[i]:rp[i + 1]].astype(np.float64)


def _fp32_bound(L, absprod):
    u = 2.0 ** -24
    return (L + 1) * u / (1 - (L + 1) * u) * absprod


def test_sparse_full_forward_pass_sampled_rows(g, sparse_full):
    """Rows of Y = A O at full size: the oracle sums each sampled row entry by
    entry with its own O rows (the same stream, FP32-rounded)."""
    w, A, At, host = sparse_full
    r = w.k + w.p
    rp = host[0]
    lens = np.diff(rp.astype(np.int64))
    rng = np.random.default_rng(7)
    rows = np.concatenate([np.argsort(-lens, kind="stable")[:3], rng.choice(w.m, 40, replace=False)])
    ldr = (r + 3) // 4 * 4  # the panel stride of the plan (vector kernel)
    O = torch.zeros(w.n, ldr, device="cuda")
    O[:, :r] = g.gaussian(w.n, r, w.seed, "f32")
    Y = g.apass(A, O[:, :r], trans=False, out=torch.empty(w.m, ldr, device="cuda")[:, :r])
    Yg = Y[torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    for t, i in enumerate(rows):
        cols, vals = _row_entries(host, i)
        Orows = OG.gaussian_rows(cols, r, w.seed, "f32")
        ref = vals @ Orows
        bound = _fp32_bound(len(cols), np.abs(vals) @ np.abs(Orows))
        assert np.all(np.abs(Yg[t] - ref) <= bound + 1e-30), i


def test_sparse_full_transposed_pass_sampled_columns(g, sparse_full):
    """Rows j of Z = A^T Y (columns of A) for a seeded panel Y, entry by entry."""
    w, A, At, host = sparse_full
    r = w.k + w.p
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w.noise_seed)
    ldr = (r + 3) // 4 * 4
    Yin = torch.randn(w.m, ldr, generator=gen, device="cuda")[:, :r]
    Z = g.apass(A, Yin, trans=True, At=At, out=torch.empty(w.n, ldr, device="cuda")[:, :r])
    rp, ci, v = host
    for j in (150, 700, 20000, 999_999):
        pos = np.flatnonzero(ci == j)
        rows = np.searchsorted(rp, pos, side="right") - 1
        Yr = Yin[torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
        vals = v[pos].astype(np.float64)
        ref = vals @ Yr
        bound = _fp32_bound(len(pos), np.abs(vals) @ np.abs(Yr))
        got = Z[j].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - ref) <= bound + 1e-30), j


def test_sparse_full_rsvd_properties(g, sparse_full):
    """The full sparse rSVD: orthonormal U and V, descending positive S, and
    A^T U = V diag(S), which holds exactly for U = Q U_B, V = Q_b W (checked
    with torch's own sparse product)."""
    w, A, At, host = sparse_full
    plan = g.Plan(w.m, w.n, w.k, w.p, w.q, w.seed, prec="fp32", kind="csr")
    U, S, V = plan.run(A, At=At)
    plan.close()
    Uh, Sh, Vh = _np(U), _np(S), _np(V)
    assert np.all(Sh > 0) and np.all(np.diff(Sh) <= 0)
    I = np.eye(w.k)
    assert np.abs(Uh.T @ Uh - I).max() <= 1e-4 and np.abs(Vh.T @ Vh - I).max() <= 1e-4
    AtU = (At @ U).cpu().numpy().astype(np.float64)
    assert np.linalg.norm(AtU - Vh * Sh) <= 1e-4 * np.linalg.norm(Sh)


# ---- out-of-core recipe, scaled ------------------------------------------------------

def _min_cap(g, m, n, k, p, prec, mb, nb):
    from paper_1907_06470_gb300 import _lib
    o = _lib.RsvdOpts(prec=_lib.PREC[prec], refine=1, mb=mb, nb=nb, n_slots=2, dtype=_lib.DTYPE["f32"])
    out = C.c_size_t()
    assert g.load().rsvd_plan_min_cap(m, n, k, p, C.byref(o), C.byref(out)) == 0
    return out.value


@pytest.fixture(scope="module")
def ooc_recipe():
    w = WORKLOADS["dense_fp32_600000x100000_ooc"]
    m, n = 16384, 6000
    A = lowrank_plus_noise_torch(m, n, 2000, 50.0, 1e-3, w.data_seed, w.noise_seed)
    A_host = A.cpu().numpy()
    return w, m, n, A_host


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16"])
def test_ooc_recipe_streamed_matches_oracle(g, ooc_recipe, prec):
    """The out-of-core recipe (k 200, p 40, q 2) at 16384 x 6000, streamed in
    2048^2 tiles under a cap that holds about a third of A."""
    w, m, n, A_host = ooc_recipe
    tile = 2048
    cap = _min_cap(g, m, n, w.k, w.p, prec, tile, tile) + A_host.nbytes // 3
    plan = g.Plan(m, n, w.k, w.p, w.q, w.seed, mem_cap=cap, prec=prec, mb=tile, nb=tile)
    U, S, V = (_np(t) for t in plan.run(torch.as_tensor(A_host).pin_memory()))
    st = plan.stream_stats()
    plan.close()
    assert st["tiles_streamed_per_pass"] > 0 and st["h2d_bytes"] > A_host.nbytes
    ref = OR.rsvd(A_host, w.k, w.p, w.q, w.seed, "f32" if prec == "fp32" else "bf16")
    es, eu, ev = _errors(U, S, V, ref, w.k)
    print(f"ooc {prec}: sigma {es:.2e} U {eu:.2e} V {ev:.2e}")
    if prec == "bf16":
        assert es <= 1e-3
    else:
        assert es <= 1e-5 and eu <= 1e-4 and ev <= 1e-4
