"""Plain, slow FP64 CPU oracle for the randomized SVD hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or call it.  It shares no code with the CUDA library
(``paper_1907_06470_gb300``): every routine here is written from the paper
(Demchik, Bacak, Bordag, "Out-of-core singular value decomposition",
arXiv:1907.06470) and from the published methods it names (Halko,
Martinsson & Tropp 2011; Salmon et al. 2011 for Philox; Demmel & Veselic
1992 for one-sided Jacobi), and it is pinned against mathematics by the
``-m "not gpu"`` tests.

Modules
-------
gaussian  Section 2.1 step 1: the Gaussian test matrix, drawn from a
          counter-based Philox4x32-10 stream through Box-Muller with
          self-written FP64 ln / sin / cos.
linalg    Householder QR (Section 2.1 steps 3-4), one-sided Jacobi SVD
          (Section 2.1 step 6), FP64 products with exact upcast.
tiles     Block-cyclic tile map (Section 1, Section 3.1) and CSR tiles.
rsvd      The randomized SVD with power iterations (Section 2.1 steps 1-7,
          Section 2.2 Eq. (2)/(3)) and the exact full SVD.
adjoint   Truncated-SVD adjoint (not in the paper; Townsend 2016).
panel     FP32 panels rounded to BF16 or to 24-bit floats (Section 3.2's
          choice of number precision, applied to the gathered panel of the
          sparse products of Section 3.3).

Parity pins: every function above is pinned by a test in ``tests/`` except
where its docstring says "parity unpinned".
"""
