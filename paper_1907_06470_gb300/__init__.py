"""GB300-native randomized SVD (Demchik, Bacak, Bordag, arXiv:1907.06470).

Thin PyTorch binding over librsvd_gb300.so: torch provides device memory and
the current stream; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the library cannot be built or loaded
on a GPU machine, these functions raise.

Main entry points
-----------------
rsvd(A, k, p, q, seed, ...)   rank-k randomized SVD (Section 2.1, Section 2.2)
Plan                          reusable plan + workspace for repeated runs
full_svd(A)                   exact SVD, min(m, n) <= 512
gaussian / tile_map / apass / orth / small_svd
                              the individual steps (Section 2.1 steps 1-6,
                              Section 3.1 tile map)
csr_transpose                 host CSR of A^T for the sparse A-passes (Section 3.3)
coo_to_csr                    host CSR of a COO matrix (or of its transpose)
fp8_quantize                  E4M3 codes of A with per-tile scales (the FP8 variant)
"""

from __future__ import annotations

import ctypes as C

from . import _lib
from ._lib import RsvdError, load  # noqa: F401

__all__ = ["rsvd", "Plan", "full_svd", "gaussian", "tile_map", "apass", "orth", "small_svd",
           "small_svd_noalloc", "csr_transpose", "coo_to_csr", "fp8_quantize", "checkpoint_info", "RsvdError", "load"]


def _torch():
    import torch
    return torch


def _stream_ptr():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float64:
        return _lib.DTYPE["f64"]
    if t.dtype == torch.float32:
        return _lib.DTYPE["f32"]
    if t.dtype == torch.bfloat16:
        return _lib.DTYPE["bf16"]
    if t.dtype == torch.float16:
        return _lib.DTYPE["f16"]
    raise TypeError(f"A must be float64, float32, bfloat16 or float16, got {t.dtype}")


def _dense_desc(A) -> _lib.RsvdMatrix:
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a 2-D tensor with unit column stride (row-major)")
    d = _lib.RsvdMatrix()
    d.kind = _lib.DENSE
    d.dtype = _dtype_code(A)
    d.location = _lib.ON_DEVICE if A.is_cuda else _lib.ON_HOST
    d.m, d.n = A.shape
    d.data = A.data_ptr()
    d.ld = A.stride(0)
    return d


def _is_csr(A) -> bool:
    torch = _torch()
    return getattr(A, "layout", None) == torch.sparse_csr


def _csr_arrays(A):
    """(rowptr int32, colidx int32, val float32) of a torch sparse CSR tensor, contiguous."""
    torch = _torch()
    rp = A.crow_indices().to(torch.int32).contiguous()
    ci = A.col_indices().to(torch.int32).contiguous()
    v = A.values()
    if v.dtype != torch.float32:
        raise TypeError(f"CSR values must be float32, got {v.dtype}")
    return rp, ci, v.contiguous()


def _is_coo(A) -> bool:
    torch = _torch()
    return getattr(A, "layout", None) == torch.sparse_coo


def _coo_pair(A):
    """Host CSR of a torch sparse COO matrix and of its transpose (library conversion)."""
    return coo_to_csr(A), coo_to_csr(A, transpose=True)


def _csr_desc(A, At=None):
    """Descriptor of a torch sparse CSR matrix (and optionally the CSR of its
    transpose).  Returns (descriptor, tensors to keep alive during the call)."""
    if A.dim() != 2:
        raise ValueError("A must be a 2-D sparse CSR tensor")
    rp, ci, v = _csr_arrays(A)
    d = _lib.RsvdMatrix()
    d.kind = _lib.CSR
    d.dtype = _lib.DTYPE["f32"]
    d.location = _lib.ON_DEVICE if A.is_cuda else _lib.ON_HOST
    d.m, d.n = A.shape
    d.rowptr, d.colidx, d.val = rp.data_ptr(), ci.data_ptr(), v.data_ptr()
    d.nnz = v.numel()
    keep = [rp, ci, v]
    if At is not None:
        if tuple(At.shape) != (A.shape[1], A.shape[0]) or At.is_cuda != A.is_cuda:
            raise ValueError("At must be the n x m CSR of A^T, on the same device as A")
        trp, tci, tv = _csr_arrays(At)
        d.t_rowptr, d.t_colidx, d.t_val = trp.data_ptr(), tci.data_ptr(), tv.data_ptr()
        keep += [trp, tci, tv]
    return d, keep


def _check(st):
    _lib.check(st)


class Plan:
    """A planned rank-k randomized SVD (rsvd_plan); owns its device workspace."""

    def __init__(self, m, n, k, p=10, q=2, seed=0, mem_cap=0, prec=None, dtype="f32",
                 mb=0, nb=0, refine=True, n_slots=2, kind="dense", auto_q=False, auto_q_tol=0.0, fused=False):
        lib = load()
        if prec is None:
            prec = "fp64" if dtype == "f64" else "fp32"
        o = _lib.RsvdOpts()
        o.prec = _lib.PREC[prec]
        o.refine = 1 if refine else 0
        o.mb, o.nb = mb, nb
        o.n_slots = n_slots
        o.dtype = _lib.DTYPE[dtype]
        o.kind = {"dense": _lib.DENSE, "csr": _lib.CSR}[kind]
        o.auto_q = 1 if auto_q else 0
        o.auto_q_tol = float(auto_q_tol)
        o.fused = 1 if fused else 0
        self.kind = kind
        h = C.c_void_p()
        _check(lib.rsvd_plan(m, n, k, p, q, seed, mem_cap, C.byref(o), C.byref(h)))
        self._h = h
        self.m, self.n, self.k, self.p, self.q, self.seed = m, n, k, p, q, seed
        self.dtype = dtype
        self.prec = prec

    def info(self) -> dict:
        i = _lib.RsvdPlanInfo()
        _check(load().rsvd_plan_info(self._h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in i._fields_}

    def run(self, A, U=None, S=None, V=None, At=None):
        """Factor A (device tensor, or pinned host tensor; for CSR plans a torch
        sparse CSR tensor, with the CSR of A^T in `At` if the caller has it, or a
        torch sparse COO tensor);
        returns (U, S, V) on the device."""
        torch = _torch()
        tdt = torch.float64 if self.dtype == "f64" else torch.float32
        dev = A.device if A.is_cuda else torch.device("cuda", torch.cuda.current_device())
        if U is None:
            U = torch.empty(self.m, self.k, dtype=tdt, device=dev)
        if S is None:
            S = torch.empty(self.k, dtype=tdt, device=dev)
        if V is None:
            V = torch.empty(self.n, self.k, dtype=tdt, device=dev)
        if _is_coo(A):
            A, At = _coo_pair(A)
        if _is_csr(A):
            d, keep = _csr_desc(A, At)
        else:
            d, keep = _dense_desc(A), [A]
        _check(load().rsvd_run(self._h, C.byref(d), C.c_void_p(U.data_ptr()), C.c_void_p(S.data_ptr()),
                               C.c_void_p(V.data_ptr()), _stream_ptr()))
        del keep
        return U, S, V

    def prefetch(self, A):
        """Start copying the pinned host tensor A to the device for a later
        run(A) of this plan and return at once (rsvd_plan_prefetch): a stream
        of host matrices keeps the link busy while the previous one is being
        factored.  A must stay unchanged until that run has returned."""
        if A.is_cuda:
            raise ValueError("prefetch takes a host tensor")
        d = _dense_desc(A)
        self._prefetched = getattr(self, "_prefetched", [])[-1:] + [A]  # alive until the run
        _check(load().rsvd_plan_prefetch(self._h, C.byref(d)))

    def backward(self, U, S, V, dU=None, dS=None, dV=None):
        """dA of the truncated SVD (see rsvd_backward) for cotangents dU, dS, dV (None = zero)."""
        torch = _torch()
        dA = torch.empty(self.m, self.n, dtype=U.dtype, device=U.device)
        p = lambda t: C.c_void_p(t.contiguous().data_ptr() if t is not None else None)
        keep = [t.contiguous() if t is not None else None for t in (U, S, V, dU, dS, dV)]
        ptrs = [C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(None) for t in keep]
        _check(load().rsvd_backward(self._h, *ptrs, C.c_void_p(dA.data_ptr()), _stream_ptr()))
        del p
        return dA

    def stream_stats(self) -> dict:
        """Out-of-core statistics of the last run (zeros when it ran in core)."""
        h2d, per_pass, resident = C.c_uint64(), C.c_int64(), C.c_int64()
        _check(load().rsvd_plan_stream_stats(self._h, C.byref(h2d), C.byref(per_pass), C.byref(resident)))
        return {"h2d_bytes": h2d.value, "tiles_streamed_per_pass": per_pass.value, "tiles_resident": resident.value}

    def set_checkpoint(self, path, stop_after_step=-1):
        """Persist the range finder's basis after each step to `path` and resume
        from a matching checkpoint there (Section 3.8); None turns it off."""
        _check(load().rsvd_plan_set_checkpoint(self._h, path.encode() if path else None, stop_after_step))

    def set_profiling(self, on=True):
        _check(load().rsvd_plan_set_profiling(self._h, 1 if on else 0))

    def stage_ms(self) -> dict:
        """Per-stage device times (ms) of the last profiled run, plus the A-pass count."""
        arr = (C.c_double * len(_lib.STAGES))()
        calls = C.c_int32()
        _check(load().rsvd_plan_stage_ms(self._h, arr, C.byref(calls)))
        out = {name: arr[i] for i, name in enumerate(_lib.STAGES)}
        out["apass_calls"] = calls.value
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().rsvd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rsvd_function():
    torch = _torch()

    class RSVDFunction(torch.autograd.Function):
        """U, S, V = rsvd(A); backward through the truncated-SVD adjoint (rsvd_backward).

        The range finder is not differentiated: the gradient is that of the
        truncated SVD evaluated at the returned factors.
        """

        @staticmethod
        def forward(ctx, A, plan):
            U, S, V = plan.run(A.detach())
            ctx.plan = plan
            ctx.save_for_backward(U, S, V)
            return U, S, V

        @staticmethod
        def backward(ctx, dU, dS, dV):
            U, S, V = ctx.saved_tensors
            return ctx.plan.backward(U, S, V, dU, dS, dV), None

    return RSVDFunction


def rsvd(A, k, p=10, q=2, seed=0, mem_cap=0, prec=None, mb=0, nb=0, refine=True, At=None, fused=False):
    """Rank-k randomized SVD of a dense float64/float32 matrix, or of one stored
    as bfloat16/float16 (FP32 outputs, BF16-precision plan) (CUDA or pinned
    host tensor), of a float32 torch sparse CSR tensor (CUDA or host; `At`
    optionally its transpose in CSR form, else built by the library), or of a
    float32 torch sparse COO tensor (converted to the CSR of A and of A^T on
    the host by the library; repeated entries add up).

    If a dense A requires grad, the result is differentiable through the
    truncated-SVD adjoint (rsvd_backward)."""
    torch = _torch()
    if _is_coo(A):
        A, At = _coo_pair(A)
    if _is_csr(A):
        plan = Plan(A.shape[0], A.shape[1], k, p, q, seed, mem_cap, prec or "fp32", "f32", mb, nb, refine,
                    kind="csr")
        try:
            return plan.run(A, At=At)
        finally:
            plan.close()
    dtype = "f64" if A.dtype == torch.float64 else "f32"
    if A.dtype in (torch.bfloat16, torch.float16):  # 16-bit storage: FP32 outputs, tensor-core passes
        if A.requires_grad:
            raise TypeError("a bfloat16 or float16 A has no backward pass")
        prec = prec or "bf16"
    plan = Plan(A.shape[0], A.shape[1], k, p, q, seed, mem_cap, prec, dtype, mb, nb, refine, fused=fused)
    if A.requires_grad:
        return _rsvd_function().apply(A, plan)
    try:
        return plan.run(A)
    finally:
        plan.close()


def kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(load().rsvd_kernel_launches())


def full_svd(A):
    """Exact thin SVD (U, S, V) of a dense CUDA matrix, min(m, n) <= 512."""
    torch = _torch()
    m, n = A.shape
    t = min(m, n)
    U = torch.empty(m, t, dtype=A.dtype, device=A.device)
    S = torch.empty(t, dtype=A.dtype, device=A.device)
    V = torch.empty(n, t, dtype=A.dtype, device=A.device)
    d = _dense_desc(A)
    _check(load().rsvd_full(C.byref(d), C.c_void_p(U.data_ptr()), C.c_void_p(S.data_ptr()),
                            C.c_void_p(V.data_ptr()), _stream_ptr()))
    return U, S, V


def gaussian(n, r, seed, dtype="f32", layout=0, out=None, device="cuda"):
    """The n x r Gaussian test matrix (layout 0) or its transpose (layout 1)."""
    torch = _torch()
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    if out is None:
        out = torch.empty((n, r) if layout == 0 else (r, n), dtype=tdt, device=device)
    ld = out.stride(0)
    _check(load().rsvd_gaussian(seed, n, r, _lib.DTYPE[dtype], layout, C.c_void_p(out.data_ptr()), ld,
                                _stream_ptr()))
    return out


def tile_map(m, n, mb, nb, n_slots=2):
    """Block-cyclic tile map as a list of (t, I, J, row0, row1, col0, col1, slot)."""
    lib = load()
    cnt = C.c_int64()
    _check(lib.rsvd_tile_map(m, n, mb, nb, n_slots, None, 0, C.byref(cnt)))
    arr = (_lib.RsvdTile * max(cnt.value, 1))()
    _check(lib.rsvd_tile_map(m, n, mb, nb, n_slots, arr, cnt.value, C.byref(cnt)))
    return [(x.t, x.I, x.J, x.row0, x.row1, x.col0, x.col1, x.slot) for x in arr[:cnt.value]]


def apass(A, X, trans=False, prec=None, mb=0, nb=0, out=None, At=None, split_long_rows=True):
    """One A-pass: A @ X (trans=False) or A.T @ X (trans=True), on the library's kernels.

    A sparse CSR A (CUDA, float32) needs `At`, the CSR of A^T, for trans=True;
    `split_long_rows` gives the call the workspace that splits long rows (the
    compact panels of prec "bf16" / "bf16x3" always have it)."""
    torch = _torch()
    if _is_csr(A):
        m, n = A.shape
        r = X.shape[1]
        prec = prec or "fp32"
        if out is None:
            out = torch.empty(n if trans else m, (r + 3) // 4 * 4, dtype=torch.float32, device=A.device)[:, :r]
        d, keep = _csr_desc(A, At)
        lib = load()
        if prec == "fp32":
            wsb = lib.rsvd_spmm_workspace(d.nnz, r) if split_long_rows else 0
        else:
            wsb = lib.rsvd_csr_apass_workspace(d.nnz, m if trans else n, r, _lib.PREC[prec])
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=A.device)
        _check(lib.rsvd_apass(C.byref(d), int(trans), _lib.PREC[prec], r, C.c_void_p(X.data_ptr()),
                              X.stride(0), C.c_void_p(out.data_ptr()), out.stride(0), 0, 0,
                              C.c_void_p(ws.data_ptr() if wsb else None), wsb, _stream_ptr()))
        del keep
        return out
    a16 = A.dtype in (torch.bfloat16, torch.float16)  # stored in 16 bits: FP32 panels and output
    if prec is None:
        prec = "fp64" if A.dtype == torch.float64 else ("bf16" if a16 else "fp32")
    m, n = A.shape
    r = X.shape[1]
    M = n if trans else m
    if out is None:
        out = torch.empty(M, r, dtype=torch.float32 if a16 else A.dtype, device=A.device)
    lib = load()
    wsb = lib.rsvd_apass_workspace(m, n, r, int(trans), _lib.PREC[prec], mb, nb)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=A.device)
    d = _dense_desc(A)
    _check(lib.rsvd_apass(C.byref(d), int(trans), _lib.PREC[prec], r, C.c_void_p(X.data_ptr()), X.stride(0),
                          C.c_void_p(out.data_ptr()), out.stride(0), mb, nb, C.c_void_p(ws.data_ptr()), wsb,
                          _stream_ptr()))
    return out


def csr_transpose(A):
    """CSR of A^T for a host torch sparse CSR tensor A (float32), computed by the
    library's host transpose (stable: entries of each row in increasing row of A)."""
    torch = _torch()
    if A.is_cuda:
        raise ValueError("csr_transpose takes a host tensor")
    rp, ci, v = _csr_arrays(A)
    m, n = A.shape
    nnz = v.numel()
    trp = torch.empty(n + 1, dtype=torch.int32)
    tci = torch.empty(nnz, dtype=torch.int32)
    tv = torch.empty(nnz, dtype=torch.float32)
    _check(load().rsvd_csr_transpose(m, n, C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()),
                                     C.c_void_p(v.data_ptr()), C.c_void_p(trp.data_ptr()),
                                     C.c_void_p(tci.data_ptr()), C.c_void_p(tv.data_ptr())))
    return torch.sparse_csr_tensor(trp, tci, tv, size=(n, m))


def csr_tile(A, row0, row1, col0, col1):
    """Entries of a host torch sparse CSR tensor A (float32) inside rows
    [row0, row1) x columns [col0, col1), as a host sparse CSR tensor of shape
    (row1 - row0, col1 - col0) with local indices (the block of Section 3.1),
    cut by the library's host tile builder."""
    torch = _torch()
    if A.is_cuda:
        raise ValueError("csr_tile takes a host tensor")
    rp, ci, v = _csr_arrays(A)
    m, n = A.shape
    lib = load()
    cnt = C.c_int64()
    args = (m, n, C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()), C.c_void_p(v.data_ptr()),
            row0, row1, col0, col1)
    _check(lib.rsvd_csr_tile(*args, None, None, None, 0, C.byref(cnt)))
    trp = torch.empty(row1 - row0 + 1, dtype=torch.int32)
    tci = torch.empty(max(cnt.value, 1), dtype=torch.int32)
    tv = torch.empty(max(cnt.value, 1), dtype=torch.float32)
    _check(lib.rsvd_csr_tile(*args, C.c_void_p(trp.data_ptr()), C.c_void_p(tci.data_ptr()),
                             C.c_void_p(tv.data_ptr()), cnt.value, C.byref(cnt)))
    return torch.sparse_csr_tensor(trp, tci[:cnt.value], tv[:cnt.value], size=(row1 - row0, col1 - col0))


def coo_to_csr(A, transpose=False):
    """Host CSR (torch sparse CSR tensor) of a torch sparse COO matrix A with
    float32 values, or of A^T with transpose=True, by the library's stable
    counting sort (rsvd_coo_to_csr): entries keep their COO order within each
    row, repeated entries stay separate.  A may be uncoalesced; CUDA tensors
    are copied to the host first."""
    torch = _torch()
    if A.dim() != 2:
        raise ValueError("A must be a 2-D sparse COO tensor")
    A = A.cpu()
    idx = A._indices()
    ri = idx[1 if transpose else 0].to(torch.int64).contiguous()
    ci = idx[0 if transpose else 1].to(torch.int64).contiguous()
    v = A._values()
    if v.dtype != torch.float32:
        raise TypeError(f"COO values must be float32, got {v.dtype}")
    v = v.contiguous()
    m, n = A.shape
    if transpose:
        m, n = n, m
    nnz = v.numel()
    rp = torch.empty(m + 1, dtype=torch.int32)
    oci = torch.empty(nnz, dtype=torch.int32)
    ov = torch.empty(nnz, dtype=torch.float32)
    _check(load().rsvd_coo_to_csr(m, n, nnz, 64, C.c_void_p(ri.data_ptr()), C.c_void_p(ci.data_ptr()),
                                  C.c_void_p(v.data_ptr()), C.c_void_p(rp.data_ptr()),
                                  C.c_void_p(oci.data_ptr()), C.c_void_p(ov.data_ptr())))
    return torch.sparse_csr_tensor(rp, oci, ov, size=(m, n))


def fp8_quantize(A, qm=0, qn=0):
    """E4M3 codes (uint8, m x n) and per-tile power-of-two scales of a dense
    float32 CUDA matrix (rsvd_fp8_quantize); qm / qn = 0 means one tile."""
    torch = _torch()
    m, n = A.shape
    qm = qm or m
    qn = qn or n
    ldc = (n + 15) // 16 * 16
    codes = torch.empty(m, ldc, dtype=torch.uint8, device=A.device)
    scales = torch.empty(-(-m // min(qm, m)), -(-n // min(qn, n)), dtype=torch.float32, device=A.device)
    d = _dense_desc(A)
    _check(load().rsvd_fp8_quantize(C.byref(d), qm, qn, C.c_void_p(codes.data_ptr()), ldc,
                                    C.c_void_p(scales.data_ptr()), _stream_ptr()))
    return codes[:, :n], scales


def checkpoint_info(path) -> dict:
    """Header of a checkpoint file written by a plan with set_checkpoint."""
    info = _lib.RsvdCheckpointInfo()
    _check(load().rsvd_checkpoint_info(str(path).encode(), C.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def orth(Y, want_R=False):
    """CholeskyQR2 of a device panel: returns Q (and the FP64 factor R when asked)."""
    torch = _torch()
    M, r = Y.shape
    Q = torch.empty_like(Y)
    R = torch.empty(r, r, dtype=torch.float64, device=Y.device) if want_R else None
    lib = load()
    wsb = lib.rsvd_orth_workspace(M, r)
    ws = torch.empty(wsb, dtype=torch.uint8, device=Y.device)
    _check(lib.rsvd_orth(_dtype_code(Y), M, r, C.c_void_p(Y.data_ptr()), Y.stride(0), C.c_void_p(Q.data_ptr()),
                         Q.stride(0), C.c_void_p(R.data_ptr() if R is not None else None),
                         C.c_void_p(ws.data_ptr()), wsb, _stream_ptr()))
    return (Q, R) if want_R else Q


def small_svd(Mc):
    """One-sided Jacobi SVD of a square FP64 device matrix given column-major (i.e. pass M^T row-major)."""
    torch = _torch()
    r = Mc.shape[0]
    sigma = torch.empty(r, dtype=torch.float64, device=Mc.device)
    U = torch.empty(r, r, dtype=torch.float64, device=Mc.device)
    W = torch.empty(r, r, dtype=torch.float64, device=Mc.device)
    lib = load()
    wsb = lib.rsvd_small_svd_workspace(r)
    ws = torch.empty(wsb, dtype=torch.uint8, device=Mc.device)
    Mc = Mc.contiguous()
    _check(lib.rsvd_small_svd(r, C.c_void_p(Mc.data_ptr()), C.c_void_p(sigma.data_ptr()),
                              C.c_void_p(U.data_ptr()), C.c_void_p(W.data_ptr()), C.c_void_p(ws.data_ptr()),
                              wsb, _stream_ptr()))
    return sigma, U, W


def small_svd_noalloc(Mc, sigma=None, U=None, W=None):
    """small_svd without a workspace: for callers that cannot allocate device
    memory (the library uses its own static scratch; calls must not overlap on
    the GPU).  Outputs may be passed in preallocated."""
    torch = _torch()
    r = Mc.shape[0]
    if sigma is None:
        sigma = torch.empty(r, dtype=torch.float64, device=Mc.device)
    if U is None:
        U = torch.empty(r, r, dtype=torch.float64, device=Mc.device)
    if W is None:
        W = torch.empty(r, r, dtype=torch.float64, device=Mc.device)
    _check(load().rsvd_small_svd_noalloc(r, C.c_void_p(Mc.data_ptr()), C.c_void_p(sigma.data_ptr()),
                                         C.c_void_p(U.data_ptr()), C.c_void_p(W.data_ptr()), _stream_ptr()))
    return sigma, U, W
