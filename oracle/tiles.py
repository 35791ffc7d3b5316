"""Block-cyclic tile map (Section 1 and Section 3.1) and CSR row tiles.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 3.1 specifies blocks as ranges of row and column indices of the
source matrix, sized from the memory limits; the block-cyclic distribution
of Dongarra & Walker assigns blocks to workers cyclically.  Reading used
here: tile (I, J) covers rows [I*mb, min(m, (I+1)*mb)) and columns
[J*nb, min(n, (J+1)*nb)); tiles are numbered t = I*Tn + J (row-major over the
tile grid, Tn = ceil(n/nb)) and tile t goes to slot t mod S.
"""

from __future__ import annotations

import numpy as np


def tile_map(m: int, n: int, mb: int, nb: int, slots: int):
    """List of tuples (t, I, J, row0, row1, col0, col1, slot) in visit order."""
    if m < 0 or n < 0 or mb <= 0 or nb <= 0 or slots <= 0:
        raise ValueError("bad tile map arguments")
    Tm = -(-m // mb)
    Tn = -(-n // nb)
    out = []
    for I in range(Tm):
        for J in range(Tn):
            t = I * Tn + J
            out.append((t, I, J, I * mb, min(m, (I + 1) * mb),
                        J * nb, min(n, (J + 1) * nb), t % slots))
    return out


def csr_tile(rowptr, colidx, vals, row0: int, row1: int, col0: int, col1: int):
    """Entries of a CSR matrix inside rows [row0,row1) x cols [col0,col1).

    Returns (local_rowptr, local_colidx, local_vals) with row and column
    indices relative to the tile origin; within each row the column order of
    the source is kept.  Each source row is scanned entry by entry.
    """
    lrp = [0]
    lci = []
    lv = []
    for i in range(row0, row1):
        for e in range(int(rowptr[i]), int(rowptr[i + 1])):
            c = int(colidx[e])
            if col0 <= c < col1:
                lci.append(c - col0)
                lv.append(vals[e])
        lrp.append(len(lci))
    return (np.array(lrp, dtype=np.int64), np.array(lci, dtype=np.int64),
            np.array(lv, dtype=np.asarray(vals).dtype))


def csr_transpose(m: int, n: int, rowptr, colidx, vals):
    """CSR of A^T from CSR of A (an m x n matrix) by scattering every entry.

    Rows of the result are the columns of A; inside each, entries appear in
    increasing row index of A.
    """
    rows_of = [[] for _ in range(n)]
    for i in range(m):
        for e in range(int(rowptr[i]), int(rowptr[i + 1])):
            rows_of[int(colidx[e])].append((i, vals[e]))
    trp = [0]
    tci = []
    tv = []
    for j in range(n):
        for i, v in rows_of[j]:
            tci.append(i)
            tv.append(v)
        trp.append(len(tci))
    return (np.array(trp, dtype=np.int64), np.array(tci, dtype=np.int64),
            np.array(tv, dtype=np.asarray(vals).dtype))


def coo_to_csr(m: int, n: int, rowidx, colidx, vals):
    """CSR of an m x n matrix given in coordinate format (Section 3.3).

    Every entry e = (rowidx[e], colidx[e], vals[e]) goes to the list of its
    row, in the order the entries are given; repeated positions stay separate
    entries (the matrix is their sum).  Raises ValueError for an index outside
    [0, m) x [0, n).
    """
    rows_of = [[] for _ in range(m)]
    for e in range(len(vals)):
        i, j = int(rowidx[e]), int(colidx[e])
        if not (0 <= i < m and 0 <= j < n):
            raise ValueError("COO index out of range")
        rows_of[i].append((j, vals[e]))
    rp = [0]
    ci = []
    v = []
    for i in range(m):
        for j, x in rows_of[i]:
            ci.append(j)
            v.append(x)
        rp.append(len(ci))
    return (np.array(rp, dtype=np.int64), np.array(ci, dtype=np.int64),
            np.array(v, dtype=np.asarray(vals).dtype))
