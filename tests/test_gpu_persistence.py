"""Persistence and resumption of the range finder (Section 3.8): a run stopped
after a checkpoint and resumed by a new plan gives the uninterrupted result."""

import os

import numpy as np
import pytest

from oracle import rsvd as OR
from synth import prescribed_dense, spectrum_geometric, zipf_csr
from tests.metrics import max_principal_angle, sigma_rel_err

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
    # and the resumed result is the oracle's (the bars of the plan's precision)
    Uo, So, Vo = OR.rsvd(A.cpu().numpy(), k, p, q, seed, {"fp64": "f64", "fp32": "f32", "bf16": "bf16"}[prec])
    U, S, V = (t.numpy().astype(np.float64) for t in out)
    es, eu = sigma_rel_err(S, So), max_principal_angle(U, Uo)
    if prec == "fp64":
        assert es <= 1e-11 and eu <= 1e-9
    elif prec == "fp32":
        assert es <= 1e-5 and eu <= 1e-4
    else:
        assert es <= 1e-3


def test_a_new_process_resumes_after_the_first_one_ended(g, tmp_path):
    """The interrupted run happens in a child process that ends abruptly after
    the checkpoint of step 3 (os._exit, no teardown; none of its work is left
    on the GPU); this process then resumes from the file and gets the
    uninterrupted result, bit for bit, and the oracle's at the FP32 bars."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = str(tmp_path / "rsvd.ckpt")
    k, p, q, seed = 20, 10, 2, 11
    child = (
        "import os, sys, numpy as np, torch\n"
        f"sys.path.insert(0, {root!r})\n"
        "import paper_1907_06470_gb300 as g\n"
        "from synth import prescribed_dense, spectrum_geometric\n"
        "A, _, _ = prescribed_dense(3000, 1500, spectrum_geometric(1500, 0.98), 5, dtype=np.float32)\n"
        f"plan = g.Plan(3000, 1500, {k}, {p}, {q}, {seed})\n"
        f"plan.set_checkpoint({path!r}, stop_after_step=3)\n"
        "try:\n"
        "    plan.run(torch.as_tensor(A, device='cuda'))\n"
        "except g.RsvdError as e:\n"
        "    torch.cuda.synchronize()\n"
        "    os._exit(17 if 'INTERRUPTED' in str(e) else 2)\n"
        "os._exit(1)\n")
    r = subprocess.run([sys.executable, "-c", child], cwd=root, timeout=900)
    assert r.returncode == 17 and os.path.exists(path)
    assert g.checkpoint_info(path)["step"] == 3
    A = _A(5)
    ref = [t.cpu() for t in g.Plan(3000, 1500, k, p, q, seed).run(A)]
    plan = g.Plan(3000, 1500, k, p, q, seed)
    plan.set_checkpoint(path)
    out = [t.cpu() for t in plan.run(A)]
    assert plan.info()["resumed_from"] == 3
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    Uo, So, Vo = OR.rsvd(A.cpu().numpy(), k, p, q, seed, "f32")
    U, S, V = (t.numpy().astype(np.float64) for t in out)
    assert sigma_rel_err(S, So) <= 1e-5 and max_principal_angle(U, Uo) <= 1e-4


def test_host_csr_resumes_from_its_checkpoint(g, tmp_path):
    """A CSR matrix held in host memory: the checkpoint's fingerprint is taken
    from the host arrays, so a restarted plan given the same host CSR resumes."""
    m, n, k, p, q, seed = 6000, 2000, 20, 10, 2, 2004
    rp, ci, v = zipf_csr(m, n, 60000, 1004)
    Ah = torch.sparse_csr_tensor(torch.as_tensor(rp), torch.as_tensor(ci), torch.as_tensor(v), size=(m, n))
    ref = [t.cpu() for t in g.Plan(m, n, k, p, q, seed, kind="csr").run(Ah)]
    path = str(tmp_path / "csr.ckpt")
    p1 = g.Plan(m, n, k, p, q, seed, kind="csr")
    p1.set_checkpoint(path, stop_after_step=2)
    with pytest.raises(g.RsvdError):
        p1.run(Ah)
    p1.close()
    p2 = g.Plan(m, n, k, p, q, seed, kind="csr")
    p2.set_checkpoint(path)
    out = [t.cpu() for t in p2.run(Ah)]
    assert p2.info()["resumed_from"] == 2
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    from oracle.linalg import CSR
    Uo, So, Vo = OR.rsvd(CSR(m, n, rp, ci, v), k, p, q, seed, "f32")
    assert sigma_rel_err(out[1].numpy(), So) <= 1e-5


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
