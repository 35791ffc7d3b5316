"""rsvd_small_svd_noalloc: the Jacobi SVD entry point for callers that cannot
allocate device memory (it uses the library's static scratch array instead of
a caller workspace).  Checked against rsvd_small_svd, the entry point that
takes a workspace, on consecutive calls that reuse the shared scratch.  This
file is collected last on purpose."""

import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _graded_r_factor(r, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((4 * r + 8, r)) * np.logspace(0, -4, r)
    return np.linalg.qr(Y)[1]


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    import paper_1907_06470_gb300 as g
    g.load()
    # two calls in a row on different sizes: the second reuses the scratch the
    # first left behind (flags and status must be cleared by each call)
    for r, seed in [(120, 1), (37, 2), (256, 3)]:
        M = _graded_r_factor(r, seed)
        Mc = torch.as_tensor(np.ascontiguousarray(M.T), device="cuda")
        s_ref, U_ref, W_ref = (t.cpu().numpy() for t in g.small_svd(Mc))
        s_na, U_na, W_na = (t.cpu().numpy() for t in g.small_svd_noalloc(Mc))
        assert np.max(np.abs(s_na - s_ref) / s_ref) < 1e-12
        assert np.max(np.abs(U_na - U_ref)) < 1e-12
        assert np.max(np.abs(W_na - W_ref)) < 1e-12
        assert np.linalg.norm(M @ W_na - U_na * s_na) < 1e-13 * s_na[0] * r


def test_noalloc_rejects_r_above_the_static_limit():
    import paper_1907_06470_gb300 as g
    from paper_1907_06470_gb300 import _lib
    lib = g.load()
    r = _lib.NOALLOC_MAX_R + 1
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = C.c_void_p(d.data_ptr())
    st = lib.rsvd_small_svd_noalloc(r, p, p, p, p, None)
    assert st == 1
    assert b"RSVD_NOALLOC_MAX_R" in lib.rsvd_last_error()
