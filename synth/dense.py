"""Dense synthetic matrices A = U diag(s) V^T with a prescribed spectrum."""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def spectrum_geometric(t: int, ratio: float, scale: float = 1.0) -> np.ndarray:
    """s_i = scale * ratio^(i-1), i = 1..t."""
    return scale * ratio ** np.arange(t, dtype=np.float64)


def spectrum_harmonic_noisy(t: int, noise: float, seed: int) -> np.ndarray:
    """s_i = |1/i + noise*g_i| with g_i ~ N(0,1) seeded, re-sorted descending.

    The noise sits on the spectrum, not on the entries: a dense noise matrix
    of that size would have a norm far above s_100.
    """
    g = np.random.Generator(np.random.PCG64(seed)).standard_normal(t)
    s = np.abs(1.0 / np.arange(1, t + 1, dtype=np.float64) + noise * g)
    return np.sort(s)[::-1].copy()


def spectrum_exp_floor(t: int, decay: float, floor: float) -> np.ndarray:
    """s_i = exp(-(i-1)/decay) + floor."""
    return np.exp(-np.arange(t, dtype=np.float64) / decay) + floor


def _orthonormal(rows: int, cols: int, rng) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((rows, cols)))
    return q * np.sign(np.where(np.diag(r) == 0, 1.0, np.diag(r)))


def prescribed_dense(m: int, n: int, s, seed: int, dtype=np.float64):
    """Host A = U diag(s) V^T, U (m x t) and V (n x t) orthonormal, t = len(s) <= min(m, n).

    Returns (A, U, V) with A rounded to ``dtype``.
    """
    s = np.asarray(s, dtype=np.float64)
    t = len(s)
    rng = np.random.Generator(np.random.PCG64(seed))
    U = _orthonormal(m, t, rng)
    V = _orthonormal(n, t, rng)
    A = (U * s) @ V.T
    return A.astype(dtype), U, V


def prescribed_dense_torch(m: int, n: int, s, seed: int, device="cuda", dtype=None):
    """Device A = U diag(s) V^T built with torch (for sizes the host cannot build quickly).

    U and V come from a library QR of seeded Gaussians in FP32 on the device;
    A is returned in ``dtype`` (default FP32).  The same seed gives the same A
    on the same device type and library version, not bit-identical across them.
    """
    import torch
    dtype = dtype or torch.float32
    s = torch.as_tensor(np.asarray(s, dtype=np.float64), device=device, dtype=torch.float32)
    t = s.numel()
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        G = torch.randn(m, t, generator=gen, device=device, dtype=torch.float32)
        U, _ = torch.linalg.qr(G)
        del G
        H = torch.randn(n, t, generator=gen, device=device, dtype=torch.float32)
        V, _ = torch.linalg.qr(H)
        del H
        A = (U * s) @ V.T
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return A.to(dtype).contiguous()


def lowrank_plus_noise_torch(m: int, n: int, rank: int, decay: float, floor: float,
                             seed: int, noise_seed: int, device="cuda", row0: int = 0,
                             rows: int | None = None):
    """Rows [row0, row0+rows) of A = U_R diag(exp(-i/decay)) V_R^T + floor*G/sqrt(m).

    U_R (m x rank), V_R (n x rank) orthonormal; G an i.i.d. Gaussian drawn per
    row block from (noise_seed, row0) so a block can be built on its own.
    The singular values of the floor lie near floor*[1-sqrt(n/m), 1+sqrt(n/m)];
    the spectrum is therefore approximate by construction.
    """
    import torch
    rows = m - row0 if rows is None else rows
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    UR, _ = torch.linalg.qr(torch.randn(m, rank, generator=gen, device=device))
    VR, _ = torch.linalg.qr(torch.randn(n, rank, generator=gen, device=device))
    s = torch.exp(-torch.arange(rank, device=device, dtype=torch.float32) / decay)
    gn = torch.Generator(device=device)
    gn.manual_seed(noise_seed * 1_000_003 + row0)
    G = torch.randn(rows, n, generator=gn, device=device)
    return ((UR[row0:row0 + rows] * s) @ VR.T + (floor / float(np.sqrt(m))) * G).contiguous()


class LowRankPlusNoise:
    """Row blocks of A = U_R diag(exp(-i/decay)) V_R^T + floor * G / sqrt(m), built on a GPU.

    The factors are drawn once (QR of seeded Gaussians); each row block adds its
    own seeded Gaussian noise, so blocks can be produced one at a time and
    copied out (for matrices larger than device memory).
    """

    def __init__(self, m, n, rank, decay, floor, seed, noise_seed, device="cuda"):
        import torch
        self.m, self.n, self.floor, self.noise_seed, self.device = m, n, floor, noise_seed, device
        gen = torch.Generator(device=device)
        gen.manual_seed(seed)
        self.UR, _ = torch.linalg.qr(torch.randn(m, rank, generator=gen, device=device))
        self.VRt = torch.linalg.qr(torch.randn(n, rank, generator=gen, device=device))[0].T.contiguous()
        self.s = torch.exp(-torch.arange(rank, device=device, dtype=torch.float32) / decay)

    def rows(self, row0, nrows):
        import torch
        gn = torch.Generator(device=self.device)
        gn.manual_seed(self.noise_seed * 1_000_003 + row0)
        G = torch.randn(nrows, self.n, generator=gn, device=self.device)
        return (self.UR[row0:row0 + nrows] * self.s) @ self.VRt + (self.floor / float(np.sqrt(self.m))) * G


@dataclass(frozen=True)
class Workload:
    name: str
    m: int
    n: int
    k: int
    p: int
    q: int
    seed: int         # seed of the Gaussian test matrix
    data_seed: int
    noise_seed: int
    tile: int         # square tile edge of the block-cyclic map
    description: str


WORKLOADS = {
    "dense_fp64_2000x1000": Workload(
        "dense_fp64_2000x1000", 2000, 1000, 20, 10, 2, 2001, 1001, 3001, 1024,
        "dense FP64 2000x1000, s_i = 0.9^(i-1), k=20 p=10 q=2"),
    "dense_fp32_100000x20000": Workload(
        "dense_fp32_100000x20000", 100000, 20000, 100, 20, 2, 2002, 1002, 3002, 4096,
        "dense FP32 100000x20000 (8 GB), s_i = |1/i + 1e-4 g_i|, k=100 p=20 q=2, 4096^2 tiles"),
    "dense_fp32_600000x100000_ooc": Workload(
        "dense_fp32_600000x100000_ooc", 600000, 100000, 200, 40, 2, 2003, 1003, 3003, 8192,
        "dense FP32 600000x100000 (240 GB) in pinned host memory, s_i = exp(-i/50) + 1e-3 floor, "
        "k=200 p=40 q=2, 8192^2 tiles streamed under a 64 GB device cap"),
    "csr_fp32_5000000x1000000": Workload(
        "csr_fp32_5000000x1000000", 5_000_000, 1_000_000, 300, 50, 3, 2004, 1004, 3004, 0,
        "CSR 5e6 x 1e6, 5e8 entries: rank-size row lengths min(20000, C rho^-1.1), Zipf(1.0) "
        "columns, values log(1 + Poisson(3 | >= 1)) * idf; k=300 p=50 q=3"),
    "dense_fp32_20000x10000_diff": Workload(
        "dense_fp32_20000x10000_diff", 20000, 10000, 64, 16, 2, 2005, 1005, 3005, 4096,
        "dense FP32 20000x10000, s_i = 10*0.95^(i-1), k=64 p=16 q=2 (differentiable)"),
}
