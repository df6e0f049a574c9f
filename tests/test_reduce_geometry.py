"""Launch geometry of the split-form reduction's stacked products (host logic,
no GPU): the contraction kernel's tile order is replayed for the shapes
hs_reduce launches, and every tensor-map row block, every store and the block
of the product that is needed are checked.

A full product A^H B (A: K x m, B: K x nc, both K-major) comes from the lower
triangle of M^H M for the stacked operand M = [B | 0 | A]: B's columns first,
zeros up to nc_pad = roundup(nc, 128), then A's.  The launch covers only the row
blocks of A's part (first row block nc_pad / 128); the block below the split is
(A^H B) and is written through an output base shifted back by nc_pad rows into an
m x (nc_pad + m) buffer.  The same launch shape serves the transform's H L^-H
(A = H, B = L^-H, nc = m = N_G) and the inverse's trailing updates.
"""
import numpy as np
import pytest

BM, BNC, ROWS_ALIGN = 128, 64, 128  # tile rows, complex tile columns, slice row alignment


def rows_pad(n):
    return (n + ROWS_ALIGN - 1) // ROWS_ALIGN * ROWS_ALIGN


def contraction_tiles(bi0, nbi, nbj, band=8):
    """(row origin, column origin) of every CTA of a lower-triangle contraction:
    consecutive CTAs 2p, 2p + 1 take column blocks 2c, 2c + 1 of one row block, pairs
    c <= row block, row blocks in bands, column-major inside a band."""
    npr = (nbj + 1) >> 1
    out = []
    for b0 in range(bi0, nbi, band):
        b1 = min(b0 + band, nbi)
        for c in range(npr):
            for bi in range(max(b0, c), b1):
                out += [(bi * BM, (2 * c + half) * BNC) for half in (0, 1)]
    return out


def check_stacked(m, nc):
    nc_pad = rows_pad(nc)
    NM = nc_pad + m
    rpM = rows_pad(NM)
    nbj = (NM + BNC - 1) // BNC
    bi0, nbi = nc_pad // BM, (NM + BM - 1) // BM
    tiles = contraction_tiles(bi0, nbi, nbj)
    # the library's tile count
    assert len(tiles) == sum(2 * min(b + 1, (nbj + 1) // 2) for b in range(bi0, nbi))
    covered = set()
    for i0, j0 in tiles:
        assert i0 >= nc_pad                      # only A's rows: the shifted base is safe
        assert i0 + BM <= rpM and j0 + BNC <= rpM  # tensor-map row blocks inside M's slices
        rows = [i for i in range(i0, i0 + BM) if i < NM]
        cols = [j for j in range(j0, j0 + BNC) if j < NM]
        for i in rows:                           # stores: (i - nc_pad) + j m < m (nc_pad + m)
            assert 0 <= i - nc_pad < m
        if rows and cols:
            assert (rows[-1] - nc_pad) + cols[-1] * m < m * NM
            covered.add((i0 // BM, j0 // BNC))
    need = {(bi, bj) for bi in range(bi0, nbi) for bj in range((nc + BNC - 1) // BNC)}
    assert need <= covered


@pytest.mark.parametrize("n", [1, 37, 64, 65, 128, 129, 257, 520, 777, 4000, 12000])
def test_transform_product_geometry(n):
    check_stacked(n, n)  # H L^-H: A = H, B = L^-H


@pytest.mark.parametrize("n", [300, 777, 4000])
def test_inverse_update_geometry(n):
    # trailing update of block row i: m = n - (i + 1) 128 rows, nc = (i + 1) 128 columns
    for i0 in range(0, n - 128, 128):
        check_stacked(n - i0 - 128, i0 + 128)


def test_stacked_block_is_the_product():
    # the algebra the launches rely on, with exact products standing in for the slices
    rng = np.random.default_rng(0)
    K, m, nc = 40, 70, 50
    A = rng.standard_normal((K, m)) + 1j * rng.standard_normal((K, m))
    B = rng.standard_normal((K, nc)) + 1j * rng.standard_normal((K, nc))
    nc_pad = rows_pad(nc)
    M = np.zeros((K, nc_pad + m), complex)
    M[:, :nc], M[:, nc_pad:] = B, A
    G = M.conj().T @ M
    assert np.allclose(G[nc_pad:, :nc], A.conj().T @ B, rtol=0, atol=1e-12)
