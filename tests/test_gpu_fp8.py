"""The FP8 variant of the A-passes: E4M3 codes with per-tile power-of-two
scales (bit-exact against the oracle's encoding), the tensor-core pass on the
codes (against the oracle's product of the decoded matrix), and the
randomized SVD on the FP8 path (reported accuracy)."""

import numpy as np
import pytest

from oracle import fp8 as OF
from oracle import linalg as OL
from oracle import rsvd as OR
from oracle.gaussian import bf16_bits_to_f64, to_bf16_bits
from synth import prescribed_dense, spectrum_harmonic_noisy
from tests.metrics import sigma_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1907_06470_gb300 as g
    g.load()
    return g


def _graded(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * np.logspace(-4, 3, n)[None, :] * np.logspace(0, -2, m)[:, None]
    return A.astype(np.float32)


@pytest.mark.parametrize("m,n,qm,qn", [(300, 260, 128, 128), (1000, 700, 1000, 256), (4113, 513, 128, 512),
                                       (256, 256, 0, 0), (129, 1, 128, 128)])
def test_codes_and_scales_bit_exact(g, m, n, qm, qn):
    A = _graded(m, n, m + n)
    A[:40, :40] = 0.0  # an all-zero corner (and, for 128-tiles, part of a tile)
    codes, scales = g.fp8_quantize(torch.as_tensor(A, device="cuda"), qm, qn)
    qm_, qn_ = min(qm or m, m), min(qn or n, n)
    oc, osc = OF.quantize_tiles(A, qm_, qn_)
    assert np.array_equal(scales.cpu().numpy().astype(np.float64), osc)
    assert np.array_equal(codes.cpu().numpy(), oc)


def test_zero_tile_and_rejected_tile_edges(g):
    A = np.zeros((256, 256), dtype=np.float32)
    codes, scales = g.fp8_quantize(torch.as_tensor(A, device="cuda"), 128, 128)
    assert np.all(scales.cpu().numpy() == 1.0) and np.all(codes.cpu().numpy() == 0)
    with pytest.raises(g.RsvdError):
        g.fp8_quantize(torch.as_tensor(np.ones((300, 300), dtype=np.float32), device="cuda"), 100, 128)


def _bf16(x):
    return bf16_bits_to_f64(to_bf16_bits(np.asarray(x, dtype=np.float64)))


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("tile", [0, 512])
def test_fp8_apass_is_the_product_of_the_decoded_matrix(g, trans, tile):
    """FP8 pass = exact product of decode(codes) * scale and the BF16 panel, FP32 accumulation."""
    m, n, r = 1500, 1100, 100
    A = _graded(m, n, 7 + trans)
    K = m if trans else n
    X = np.random.default_rng(3).standard_normal((K, r)).astype(np.float32)
    got = g.apass(torch.as_tensor(A, device="cuda"), torch.as_tensor(X, device="cuda"), trans, "fp8",
                  mb=tile, nb=tile).cpu().numpy().astype(np.float64)
    q = tile or max(m, n)
    codes, scales = OF.quantize_tiles(A, min(q, m), min(q, n))
    D = OF.dequantize_tiles(codes, scales, min(q, m), min(q, n))
    Xb = _bf16(X)
    ref = OL.apply(D, Xb, trans=trans)
    bound = (K + 2) * 2.0 ** -24 * OL.apply(np.abs(D), np.abs(Xb), trans=trans)
    assert np.all(np.abs(got - ref) <= bound + 1e-30)


def test_fp8_rsvd_reported_accuracy(g):
    """The randomized SVD on the FP8 path with the split-BF16 refinement of B^T
    (the 100000 x 20000 dense recipe scaled to 8000 x 4000): reported against the FP64 oracle; the
    bound only guards against a broken path."""
    m, n, k, p, q, seed = 8000, 4000, 100, 20, 2, 2002
    A, _, _ = prescribed_dense(m, n, spectrum_harmonic_noisy(n, 1e-4, 3002), 1002, dtype=np.float32)
    Ad = torch.as_tensor(A, device="cuda")
    U, S, V = g.rsvd(Ad, k, p, q, seed, prec="fp8", mb=1024, nb=1024)
    Uo, So, Vo = OR.rsvd(A, k, p, q, seed, "bf16")
    err = sigma_rel_err(S.cpu().numpy(), So)
    print(f"fp8 path: sigma relative error vs oracle {err:.2e}")
    assert err < 1e-2
    # the same plan without refinement is worse than with it
    U2, S2, V2 = g.rsvd(Ad, k, p, q, seed, prec="fp8", mb=1024, nb=1024, refine=False)
    assert sigma_rel_err(S2.cpu().numpy(), So) >= err


def test_fp8_plan_rules(g):
    with pytest.raises(g.RsvdError):  # FP8 takes F32 data
        g.Plan(1000, 500, 10, 5, 1, 0, prec="fp8", dtype="f64")
