"""Launch geometry of the split contractions' lower-triangle tiles (host logic, no
GPU), for the S and H launches of the assembly and the row ranges [bi0, bi1) of the
chunked S contraction of the host call, in the complex and the real form.

A contraction CTA takes one tile: 128 rows x 64 complex columns (128 real columns in
the real form).  Consecutive tiles 2p, 2p + 1 are the two column blocks of column
pair c of one row block; row block r needs the pairs c <= r (c <= r / 2 in the real
form, whose pairs span 256 columns); row blocks are numbered band by band, column
pairs column-major inside a band.  This file replays the kernel's decode (the same
loop, written here again) and checks that
* the decode enumerates every tile once, and the tile count is the library's;
* every 128-row x column-block block of the lower triangle of rows [128 bi0,
  min(N_G, 128 bi1)) is stored by exactly one CTA, and chunked launches together
  store each block once;
* every row and column exponent a CTA reads lies inside the slice arrays
  (roundup(N_G, 128) rows, roundup(N_G, 256) in the real form);
* a tile's column pair reaches the lower triangle of its rows (in the real form the
  second block of a pair can lie wholly above it: computed, stored into the upper
  triangle, and overwritten by the mirror).
"""
import pytest

BM, BNC, BN = 128, 64, 128


def rows_pad(n, real):
    al = 256 if real else 128
    return (n + al - 1) // al * al


def nbj_of(N_G, real):
    w = BN if real else BNC
    return (N_G + w - 1) // w


def tile_count(bi0, nbi, nbj, real):
    """The host's tile count (split_plan.cu)."""
    npr = (nbj + 1) // 2
    return sum(2 * min((b // 2 if real else b) + 1, npr) for b in range(bi0, nbi))


def decode_tile(tile, bi0, nbi, nbj, band, real):
    """The kernel's decode of contraction tile `tile`: (row origin, column origin)."""
    npr = (nbj + 1) >> 1
    p, bi, c = tile >> 1, 0, 0
    for b0 in range(bi0, nbi, band):
        b1 = min(b0 + band, nbi)
        n = sum(min((r // 2 if real else r) + 1, npr) for r in range(b0, b1))
        if p < n:
            for c in range(npr):
                lo = max(b0, 2 * c if real else c)
                cnt = b1 - lo
                if p < cnt:
                    bi = lo + p
                    break
                p -= cnt
            break
        p -= n
    return bi * BM, (2 * c + (tile & 1)) * (BN if real else BNC)


def stored_blocks(N_G, bi0, bi1, band, real):
    nbj = nbj_of(N_G, real)
    w = BN if real else BNC
    rp = rows_pad(N_G, real)
    ntiles = tile_count(bi0, bi1, nbj, real)
    seen, stored = set(), {}
    for t in range(ntiles):
        i0, j0 = decode_tile(t, bi0, bi1, nbj, band, real)
        assert bi0 * BM <= i0 < bi1 * BM
        assert (i0, j0) not in seen
        seen.add((i0, j0))
        assert i0 + BM <= rp and j0 + w <= rp   # row and column exponents, map rows
        assert j0 - (t & 1) * w <= i0 + BM - 1  # its column pair reaches the lower triangle
        if i0 < N_G and j0 < N_G:
            key = (i0 // BM, j0 // w)
            assert key not in stored
            stored[key] = t
    return stored


@pytest.mark.parametrize("real", [False, True])
@pytest.mark.parametrize("N_G", [1, 7, 64, 65, 128, 129, 255, 256, 257, 300, 777, 1000, 4000,
                                 8000, 12000])
@pytest.mark.parametrize("band", [1, 2, 4, 8, 16, 32])
def test_tiles_cover_the_lower_triangle_once(real, N_G, band):
    nbi = (N_G + BM - 1) // BM
    w = BN if real else BNC
    stored = stored_blocks(N_G, 0, nbi, band, real)
    need = {(r, jb) for r in range(nbi) for jb in range(nbj_of(N_G, real))
            if jb * w < min((r + 1) * BM, N_G)}
    assert need <= set(stored)


@pytest.mark.parametrize("real", [False, True])
@pytest.mark.parametrize("N_G,cuts", [(4000, (0, 8, 16, 24, 32)), (1000, (0, 3, 5, 8)),
                                      (12000, (0, 24, 47, 71, 94)), (777, (0, 1, 2, 7))])
def test_chunked_row_ranges_store_each_block_once(real, N_G, cuts):
    """The host call contracts S chunk by chunk, rows [128 bi0, 128 bi1) per chunk as
    the columns below 128 bi1 arrive; the chunks together store each block once."""
    w = BN if real else BNC
    total = set()
    for bi0, bi1 in zip(cuts[:-1], cuts[1:]):
        blocks = set(stored_blocks(N_G, bi0, bi1, 8, real))
        assert not (blocks & total)
        total |= blocks
    nbi = (N_G + BM - 1) // BM
    assert {(r, jb) for r in range(nbi) for jb in range(nbj_of(N_G, real))
            if jb * w < min((r + 1) * BM, N_G)} <= total


def test_tile_count_at_the_bench_shape():
    # large_12000: 94 row blocks, 188 complex column blocks -> 8930 CTAs per launch (the
    # grid the ncu capture of the S and H launches shows)
    assert tile_count(0, 94, 188, False) == 8930
