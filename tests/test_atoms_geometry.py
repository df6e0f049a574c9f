"""Packed-K geometry of the split per-atom products (host logic, no GPU).

The per-atom products Z_a = [T^BA_a | 1/2 T^BB_a][A_a; B_a] and W2 = M2_a A_a run on
the tensor cores as D[g][n] = sum_x X'[g][16 kbL + x] Op_a[n][sg P + x] over whole
16-wide K blocks: the coefficient slices pack atom a's complex rows at real positions
2 (a N_L + l) + {0, 1} (one position per row in the real form), so its rows start
inside K block kbL = floor(2 a N_L / 16); the operator slices put column l of each part
at the same offset inside the part (complex position oc + l, oc = (2 a N_L mod 16) / 2;
real position (a N_L mod 16) + l), zeros elsewhere.  This file replays those index
rules and checks, for every atom, that
* the K blocks the product reads fit the operator part (16 kblocks <= P, with P the
  library's op_part_k) and the coefficient slices (kbL + kblocks <= kpad / 16);
* each operator position is nonzero exactly where the paired coefficient position
  belongs to atom a, and then holds column l = (row) - a N_L of the same part, the
  real/imaginary parity included: neighbouring atoms' rows in a shared K block meet
  zeros, and no row of atom a is left out.
"""
import pytest

KB = 16


def kpad_of(nblk, N_L, real):
    return ((1 if real else 2) * nblk * N_L + KB - 1) // KB * KB


def op_part_k(N_A, N_L, real):
    pr = 1 if real else 2
    return KB * max((pr * (a + 1) * N_L + KB - 1) // KB - (pr * a * N_L) // KB
                    for a in range(N_A))


def check(N_A, N_L, real):
    pr = 1 if real else 2
    P = op_part_k(N_A, N_L, real)
    kpad = kpad_of(N_A, N_L, real)
    for a in range(N_A):
        kbL = (pr * a * N_L) // KB
        kblocks = (pr * (a + 1) * N_L + KB - 1) // KB - kbL
        assert KB * kblocks <= P
        assert kbL + kblocks <= kpad // KB
        covered = set()
        for x in range(KB * kblocks):
            pos = KB * kbL + x                 # coefficient position
            row = pos // pr                    # coefficient row (complex or real)
            if real:                           # operator column of position x of a part
                l = x - ((a * N_L) & (KB - 1))
            else:
                oc = ((2 * a * N_L) & (KB - 1)) >> 1
                l = x // 2 - oc
            nonzero = 0 <= l < N_L
            assert nonzero == (a * N_L <= row < (a + 1) * N_L), (a, x)
            if nonzero:
                assert l == row - a * N_L
                covered.add(row)
        assert covered == set(range(a * N_L, (a + 1) * N_L))


@pytest.mark.parametrize("real", [False, True])
@pytest.mark.parametrize("N_A,N_L", [(1, 1), (4, 16), (3, 9), (5, 16), (2, 5), (3, 33),
                                     (2, 121), (100, 121), (256, 144), (64, 81), (7, 49),
                                     (13, 25)])
def test_per_atom_k_ranges_pair_coefficients_with_operator_columns(real, N_A, N_L):
    check(N_A, N_L, real)


def test_operator_part_width_at_the_bench_shape():
    # N_L = 144: 2 N_L = 288 real positions = 18 whole K blocks for every atom
    assert op_part_k(256, 144, False) == 288
    # N_L = 121: 242 positions per atom, starting at offsets 0, 2, ..., 14 inside a
    # block; 14 + 242 = 256 positions = 16 whole blocks
    assert op_part_k(100, 121, False) == 16 * KB
