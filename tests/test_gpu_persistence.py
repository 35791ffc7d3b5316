"""Persistence and resumption of the range finder (Section 3.8): a run stopped
after a checkpoint and resumed by a new plan gives the uninterrupted result."""

import os

import numpy as np
import pytest

from synth import prescribed_dense, spectrum_geometric

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1907_06470_gb300 as g
    g.load()
    return g


def _A(seed, dtype=np.float32):
    A, _, _ = prescribed_dense(3000, 1500, spectrum_geometric(1500, 0.98), seed, dtype=dtype)
    return torch.as_tensor(A, device="cuda")


@pytest.mark.parametrize("prec,dtype,stop", [("fp32", "f32", 0), ("fp32", "f32", 3), ("bf16", "f32", 2),
                                             ("fp64", "f64", 1)])
def test_interrupted_run_resumes_to_the_same_result(g, tmp_path, prec, dtype, stop):
    A = _A(5, np.float64 if dtype == "f64" else np.float32)
    k, p, q, seed = 20, 10, 2, 11
    ref = [t.cpu() for t in g.Plan(3000, 1500, k, p, q, seed, prec=prec, dtype=dtype).run(A)]
    path = str(tmp_path / "rsvd.ckpt")
    p1 = g.Plan(3000, 1500, k, p, q, seed, prec=prec, dtype=dtype)
    p1.set_checkpoint(path, stop_after_step=stop)
    with pytest.raises(g.RsvdError) as e:
        p1.run(A)
    assert "INTERRUPTED" in str(e.value)
    assert g.checkpoint_info(path)["step"] == stop
    p1.close()
    # a new plan (as after a restart) finds the checkpoint and continues after it
    p2 = g.Plan(3000, 1500, k, p, q, seed, prec=prec, dtype=dtype)
    p2.set_checkpoint(path)
    out = [t.cpu() for t in p2.run(A)]
    assert p2.info()["resumed_from"] == stop
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    assert not os.path.exists(path)  # removed once the run completed


def test_checkpoint_of_another_matrix_or_a_damaged_file_is_not_used(g, tmp_path):
    k, p, q, seed = 20, 10, 2, 11
    path = str(tmp_path / "rsvd.ckpt")
    p1 = g.Plan(3000, 1500, k, p, q, seed)
    p1.set_checkpoint(path, stop_after_step=2)
    with pytest.raises(g.RsvdError):
        p1.run(_A(5))
    # another A: the fingerprint differs, the run starts afresh
    B = _A(6)
    p2 = g.Plan(3000, 1500, k, p, q, seed)
    p2.set_checkpoint(path, stop_after_step=-1)
    out = [t.cpu() for t in p2.run(B)]
    assert p2.info()["resumed_from"] == -1
    ref = [t.cpu() for t in g.Plan(3000, 1500, k, p, q, seed).run(B)]
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    # a damaged panel: the checksum fails, the run starts afresh
    p1.run  # noqa: B018
    with pytest.raises(g.RsvdError):
        p1.run(_A(5))
    raw = bytearray(open(path, "rb").read())
    raw[-5] ^= 0xFF
    open(path, "wb").write(bytes(raw))
    p3 = g.Plan(3000, 1500, k, p, q, seed)
    p3.set_checkpoint(path)
    p3.run(_A(5))
    assert p3.info()["resumed_from"] == -1


def test_checkpoints_are_refused_with_automatic_q(g, tmp_path):
    pl = g.Plan(3000, 1500, 20, 10, 3, 11, auto_q=True)
    with pytest.raises(g.RsvdError):
        pl.set_checkpoint(str(tmp_path / "x"))
