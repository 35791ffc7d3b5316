"""Seeded synthetic inputs shaped like the paper's workloads.

This module serves both the oracle and the CUDA path and holds none of the
method's arithmetic: it only draws seeded random matrices with a prescribed
singular spectrum (or sparsity pattern) and the loss weights of the
differentiable workload.  Orthonormal factors for the prescribed spectra come
from a library QR (numpy on the host, torch on a GPU) of seeded Gaussians.

Seeds: data = 1000 + c, test-matrix seed = 2000 + c, noise = 3000 + c for
workload c (c = 1..5); the differentiable workload also uses 4005 (X) and
5005 (w).
"""

from .dense import (  # noqa: F401
    spectrum_geometric, spectrum_harmonic_noisy, spectrum_exp_floor,
    prescribed_dense, prescribed_dense_torch, lowrank_plus_noise_torch, LowRankPlusNoise,
    WORKLOADS, Workload,
)
from .sparse import zipf_csr, zipf_csr_torch  # noqa: F401
