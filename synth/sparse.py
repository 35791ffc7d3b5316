"""Sparse synthetic matrices shaped like the paper's sparse workloads.

Recipe (rank-size reading of the sparse workload): row rho (1-based, before a
seeded row permutation) has L(rho) = min(cap, max(1, floor(C rho^-1.1)))
entries, C chosen so the total is the target nnz; column ids follow Zipf(1.0)
over 1..n, drawn without replacement inside a row and sorted; values are
log(1 + P) * idf_j with P ~ Poisson(3) conditioned on P >= 1 and
idf_j = log(1 + m / (1 + df_j)), df_j the column's entry count.
"""

from __future__ import annotations

import numpy as np


def _row_lengths(m, nnz_target, cap, n):
    rho = np.arange(1, m + 1, dtype=np.float64)
    cap = min(cap, n)
    if not m <= nnz_target <= m * cap:
        raise ValueError(f"nnz target {nnz_target} outside [m, m*cap] = [{m}, {m * cap}]")

    w = rho ** -1.1

    def total(C):
        return np.minimum(cap, np.maximum(1, np.floor(C * w))).sum()

    lo, hi = 0.0, 1.0
    while total(hi) < nnz_target:
        hi *= 2
    for _ in range(64):          # hi - lo shrinks to below one unit in the last place
        mid = 0.5 * (lo + hi)
        if total(mid) < nnz_target:
            lo = mid
        else:
            hi = mid
    return np.minimum(cap, np.maximum(1, np.floor(hi * w))).astype(np.int64)


def zipf_csr(m, n, nnz_target, seed, cap=20000):
    """Returns (rowptr int32, colidx int32, val float32) of an m x n CSR matrix.

    The row-length cap is also held to n/50, so that sampling a row's columns
    without replacement from the Zipf law stays quick on scaled-down sizes.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cap = max(1, min(cap, n // 50))
    L = _row_lengths(m, nnz_target, cap, n)[rng.permutation(m)]
    w = 1.0 / np.arange(1, n + 1, dtype=np.float64)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    done = []                                # keys of rows that reached their length
    pend = np.empty(0, dtype=np.int64)        # keys of rows still short
    need = L.copy()
    for _ in range(200):
        short = np.nonzero(need > 0)[0]
        if short.size == 0:
            break
        rows = np.repeat(short, 2 * need[short] + 4)
        cols = np.searchsorted(cdf, rng.random(rows.size))
        pend = np.unique(np.concatenate([pend, rows * n + cols]))
        prow = pend // n
        cnt = np.bincount(prow, minlength=m)
        need = np.where(need > 0, np.maximum(0, L - cnt), 0)
        complete = (need == 0)[prow]
        done.append(pend[complete])
        pend = pend[~complete]
    keys = np.concatenate(done) if done else np.empty(0, dtype=np.int64)
    have_rows, have_cols = keys // n, keys % n
    # rows with more distinct columns than their length keep a random subset
    cnt = np.bincount(have_rows, minlength=m)
    prio = rng.random(have_rows.size)
    order = np.lexsort((prio, have_rows))
    have_rows, have_cols = have_rows[order], have_cols[order]
    start = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    rank = np.arange(have_rows.size) - start[have_rows]
    keep = rank < L[have_rows]
    have_rows, have_cols = have_rows[keep], have_cols[keep]
    order = np.lexsort((have_cols, have_rows))
    rows, cols = have_rows[order], have_cols[order]
    rowptr = np.zeros(m + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(np.bincount(rows, minlength=m))
    df = np.bincount(cols, minlength=n)
    idf = np.log1p(m / (1.0 + df))
    P = rng.poisson(3.0, size=cols.size)
    while np.any(P == 0):
        z = P == 0
        P[z] = rng.poisson(3.0, size=int(z.sum()))
    val = (np.log1p(P) * idf[cols]).astype(np.float32)
    return rowptr.astype(np.int32), cols.astype(np.int32), val


def zipf_csr_torch(m, n, nnz_target, seed, cap=20000, device="cuda"):
    """The same recipe drawn with torch on a device, for sizes the host draws
    too slowly (the full sparse workload has 5e8 entries).

    Returns (rowptr int32, colidx int32, val float32) as device tensors.  Row
    lengths and their permutation are those of ``zipf_csr`` for the same seed;
    column and value draws come from a torch generator seeded with ``seed``, so
    the matrix is the same recipe but not the same matrix as ``zipf_csr``.
    """
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    cap = max(1, min(cap, n // 50))
    L_np = _row_lengths(m, nnz_target, cap, n)[rng.permutation(m)]
    L = torch.as_tensor(L_np, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    w = 1.0 / torch.arange(1, n + 1, dtype=torch.float64, device=device)
    cdf = torch.cumsum(w, 0)
    cdf /= cdf[-1].clone()
    done = []
    pend = torch.empty(0, dtype=torch.int64, device=device)
    need = L.clone()
    for _ in range(200):
        short = torch.nonzero(need > 0).flatten()
        if short.numel() == 0:
            break
        rows = torch.repeat_interleave(short, 2 * need[short] + 4)
        u = torch.rand(rows.numel(), generator=gen, dtype=torch.float64, device=device)
        cols = torch.searchsorted(cdf, u).clamp_(max=n - 1)
        del u
        pend = torch.unique(torch.cat([pend, rows * n + cols]))
        del rows, cols
        prow = pend // n
        cnt = torch.bincount(prow, minlength=m)
        need = torch.where(need > 0, (L - cnt).clamp(min=0), torch.zeros_like(need))
        complete = (need == 0)[prow]
        done.append(pend[complete])
        pend = pend[~complete]
        del prow, cnt, complete
    keys = torch.cat(done)
    del done, pend
    rows = keys // n
    # rows with more distinct columns than their length keep a random subset:
    # order by (row, random priority), keep the first L[row]
    prio = torch.randint(0, 1 << 30, (keys.numel(),), generator=gen, device=device)
    order = torch.argsort(rows * (1 << 30) + prio)
    del prio
    keys = keys[order]
    rows = rows[order]
    del order
    cnt = torch.bincount(rows, minlength=m)
    start = torch.cumsum(cnt, 0) - cnt
    rank = torch.arange(keys.numel(), device=device) - start[rows]
    keep = rank < L[rows]
    del rank, start
    keys = torch.sort(keys[keep]).values
    del keep, rows
    rows = keys // n
    cols = keys % n
    del keys
    rowptr = torch.zeros(m + 1, dtype=torch.int64, device=device)
    rowptr[1:] = torch.cumsum(torch.bincount(rows, minlength=m), 0)
    del rows
    df = torch.bincount(cols, minlength=n).to(torch.float64)
    idf = torch.log1p(m / (1.0 + df))
    P = torch.poisson(torch.full((cols.numel(),), 3.0, device=device), generator=gen)
    while True:
        z = P == 0
        nz = int(z.sum())
        if nz == 0:
            break
        P[z] = torch.poisson(torch.full((nz,), 3.0, device=device), generator=gen)
    val = (torch.log1p(P.to(torch.float64)) * idf[cols]).to(torch.float32)
    return rowptr.to(torch.int32), cols.to(torch.int32), val
