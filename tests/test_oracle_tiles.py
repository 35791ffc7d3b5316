"""Pins for the oracle's block-cyclic tile map and CSR tiles (brute force)."""

import numpy as np
import pytest

from oracle import tiles as T


@pytest.mark.parametrize("m,n,mb,nb,S", [(10, 7, 3, 2, 2), (100000, 20000, 4096, 4096, 2),
                                         (1, 1, 5, 5, 3), (8, 8, 8, 8, 1), (0, 5, 2, 2, 2)])
def test_tile_map_partitions_the_matrix(m, n, mb, nb, S):
    tiles = T.tile_map(m, n, mb, nb, S)
    Tm, Tn = -(-m // mb), -(-n // nb)
    assert len(tiles) == Tm * Tn
    assert [t[0] for t in tiles] == list(range(len(tiles)))
    if m * n <= 10000:
        cover = np.zeros((m, n), dtype=np.int64)
        for t, I, J, r0, r1, c0, c1, slot in tiles:
            cover[r0:r1, c0:c1] += 1
            assert slot == t % S and t == I * Tn + J
        assert np.all(cover == 1)
    else:
        area = sum((r1 - r0) * (c1 - c0) for _, _, _, r0, r1, c0, c1, _ in tiles)
        assert area == m * n


def test_c2_tile_edges():
    tiles = T.tile_map(100000, 20000, 4096, 4096, 2)
    assert len(tiles) == 25 * 5
    last = tiles[-1]
    assert last[3:7] == (24 * 4096, 100000, 4 * 4096, 20000)
    assert 100000 - 24 * 4096 == 1696 and 20000 - 4 * 4096 == 3616


def _random_csr(m, n, density, seed):
    rng = np.random.default_rng(seed)
    D = (rng.random((m, n)) < density) * rng.integers(1, 9, size=(m, n)).astype(np.float32)
    rp = [0]
    ci = []
    v = []
    for i in range(m):
        nz = np.nonzero(D[i])[0]
        ci += list(nz)
        v += list(D[i, nz])
        rp.append(len(ci))
    return D, np.array(rp), np.array(ci), np.array(v, dtype=np.float32)


def test_csr_tiles_match_dense_slices():
    D, rp, ci, v = _random_csr(23, 17, 0.2, 1)
    for (_, _, _, r0, r1, c0, c1, _) in T.tile_map(23, 17, 5, 6, 2):
        lrp, lci, lv = T.csr_tile(rp, ci, v, r0, r1, c0, c1)
        sub = np.zeros((r1 - r0, c1 - c0), dtype=np.float32)
        for i in range(r1 - r0):
            for e in range(lrp[i], lrp[i + 1]):
                sub[i, lci[e]] = lv[e]
        assert np.array_equal(sub, D[r0:r1, c0:c1])
    total = sum(T.csr_tile(rp, ci, v, r0, r1, c0, c1)[0][-1]
                for (_, _, _, r0, r1, c0, c1, _) in T.tile_map(23, 17, 5, 6, 2))
    assert total == len(v)


def test_csr_transpose_is_exact():
    D, rp, ci, v = _random_csr(19, 11, 0.3, 2)
    trp, tci, tv = T.csr_transpose(19, 11, rp, ci, v)
    Dt = np.zeros((11, 19), dtype=np.float32)
    for j in range(11):
        assert np.all(np.diff(tci[trp[j]:trp[j + 1]]) > 0)
        for e in range(trp[j], trp[j + 1]):
            Dt[j, tci[e]] = tv[e]
    assert np.array_equal(Dt, D.T)


def test_coo_to_csr_hand_example():
    # a 3 x 4 matrix given out of order, with (2, 1) stored twice; rows keep
    # the given order of their entries
    ri = [2, 0, 2, 1, 2, 0]
    ci = [1, 3, 0, 2, 1, 0]
    v = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0], dtype=np.float32)
    rp, oci, ov = T.coo_to_csr(3, 4, ri, ci, v)
    assert rp.tolist() == [0, 2, 3, 6]
    assert oci.tolist() == [3, 0, 2, 1, 0, 1]
    assert ov.tolist() == [2.0, 6.0, 4.0, 1.0, 3.0, 5.0]
    with pytest.raises(ValueError):
        T.coo_to_csr(3, 4, [3], [0], np.ones(1, np.float32))
    with pytest.raises(ValueError):
        T.coo_to_csr(3, 4, [0], [-1], np.ones(1, np.float32))
    rp, oci, ov = T.coo_to_csr(2, 2, [], [], np.zeros(0, np.float32))
    assert rp.tolist() == [0, 0, 0] and oci.size == 0


def test_coo_to_csr_gives_the_same_matrix():
    # the dense matrix summed from the COO entries equals the one read back
    # from the CSR, on shuffled entries with repeats
    rng = np.random.default_rng(5)
    m, n, nnz = 17, 13, 120
    ri = rng.integers(0, m, nnz)
    ci = rng.integers(0, n, nnz)
    v = rng.standard_normal(nnz)
    D = np.zeros((m, n))
    np.add.at(D, (ri, ci), v)
    rp, oci, ov = T.coo_to_csr(m, n, ri, ci, v)
    Dc = np.zeros((m, n))
    for i in range(m):
        for e in range(rp[i], rp[i + 1]):
            Dc[i, oci[e]] += ov[e]
    assert np.allclose(Dc, D, rtol=0, atol=1e-12)
    assert np.all(np.diff(rp) == np.bincount(ri, minlength=m))


def test_coo_of_the_swapped_indices_is_the_csr_transpose():
    # the COO of A in row order, read with rows and columns swapped, gives the
    # CSR of A^T that the entry-by-entry transpose builds
    D, rp, ci, v = _random_csr(19, 11, 0.3, 4)
    rows = np.repeat(np.arange(19), np.diff(rp))
    trp, tci, tv = T.coo_to_csr(11, 19, ci, rows, v)
    erp, eci, ev = T.csr_transpose(19, 11, rp, ci, v)
    assert np.array_equal(trp, erp) and np.array_equal(tci, eci) and np.array_equal(tv, ev)


@pytest.mark.parametrize("m,n,nnz,seed", [(50, 40, 300, 1), (7, 300, 900, 2), (200, 3, 150, 3)])
def test_library_csr_tile_is_bit_exact_with_oracle(m, n, nnz, seed):
    """The library's host block cutter (the tiles the out-of-core sparse
    passes stream) against the oracle's csr_tile on every block of a ragged
    grid, including empty blocks and zero-width ranges."""
    torch = pytest.importorskip("torch")
    import paper_1907_06470_gb300 as g
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.integers(0, m, nnz))
    cols = rng.integers(0, n, nnz)
    vals = rng.standard_normal(nnz).astype(np.float32)
    rp = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    A = torch.sparse_csr_tensor(torch.as_tensor(rp, dtype=torch.int32), torch.as_tensor(cols, dtype=torch.int32),
                                torch.as_tensor(vals), size=(m, n))
    for (r0, r1, c0, c1) in [(0, m, 0, n), (3, m - 2, 1, n - 1), (m // 2, m // 2, 0, n), (1, 4, n - 1, n),
                             (0, m, n // 3, n // 3)]:
        lrp, lci, lv = T.csr_tile(rp, cols, vals, r0, r1, c0, c1)
        t = g.csr_tile(A, r0, r1, c0, c1)
        assert np.array_equal(t.crow_indices().numpy(), lrp)
        assert np.array_equal(t.col_indices().numpy(), lci)
        assert np.array_equal(t.values().numpy(), lv)
