"""Prefetched host inputs (rsvd_plan_prefetch; Section 3.7, transfers
overlapped with the computation): a run that takes a prefetched copy of its A
gives the bits of a run that copies A itself, for every matrix of a stream
factored with the next copy in flight, and the results are the oracle's."""

import numpy as np
import pytest

from oracle import rsvd as OR

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1907_06470_gb300 as g
    g.load()
    return g


def _host(seed, m, n):
    gen = torch.Generator().manual_seed(seed)
    # a decaying spectrum: A = G diag(1/i) H with Gaussian G, H
    G = torch.randn(m, 64, generator=gen, dtype=torch.float64)
    H = torch.randn(64, n, generator=gen, dtype=torch.float64)
    A = (G / torch.arange(1, 65, dtype=torch.float64)) @ H + 1e-3 * torch.randn(m, n, generator=gen,
                                                                               dtype=torch.float64)
    return A.to(torch.float32).pin_memory()


def _cpu(res):
    return [t.cpu() for t in res]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_prefetched_runs_give_the_bits_of_plain_runs(g, prec):
    m, n, k, p, q, seed = 5000, 3000, 40, 8, 1, 7
    A1, A2 = _host(1, m, n), _host(2, m, n)
    plain = g.Plan(m, n, k, p, q, seed, prec=prec)
    ref1, ref2 = _cpu(plain.run(A1)), _cpu(plain.run(A2))
    plain.close()
    pl = g.Plan(m, n, k, p, q, seed, prec=prec)
    pl.prefetch(A1)
    pl.prefetch(A2)              # in flight while A1 is factored
    r1 = _cpu(pl.run(A1))
    pl.prefetch(A1)
    r2 = _cpu(pl.run(A2))
    r3 = _cpu(pl.run(A1))
    for got, ref in ((r1, ref1), (r2, ref2), (r3, ref1)):
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    # a run of another matrix drops the pending prefetch and copies its own A
    pl.prefetch(A2)
    for a, b in zip(_cpu(pl.run(A1)), ref1):
        assert torch.equal(a, b)
    # at most two pending prefetches
    pl.prefetch(A1)
    pl.prefetch(A2)
    with pytest.raises(g._lib.RsvdError):
        pl.prefetch(A1)
    for a, b in zip(_cpu(pl.run(A1)), ref1):
        assert torch.equal(a, b)
    for a, b in zip(_cpu(pl.run(A2)), ref2):
        assert torch.equal(a, b)
    pl.close()
    if prec == "fp32":  # the stream's results are the oracle's at the FP32 bar
        _, s_ref, _ = OR.rsvd(A2.numpy(), k, p, q, seed, "f32")
        s = r2[1].numpy().astype(np.float64)
        assert np.max(np.abs(s - s_ref) / s_ref) <= 1e-5


def test_prefetch_refuses_what_a_run_would_not_take_in_core(g):
    m, n = 2000, 1000
    A = _host(3, m, n)
    pl = g.Plan(m, n, 20, 4, 1, 0)
    with pytest.raises(ValueError):
        pl.prefetch(A.cuda())                            # a device tensor
    with pytest.raises(g._lib.RsvdError):
        pl.prefetch(_host(4, m, n + 8)[:, :n + 8])       # not the plan's shape
    pl.close()
