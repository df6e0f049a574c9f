"""The launch count bench.py --reduce reports (``gpu_launches``) follows the
library's launch sequence for hs_reduce; the numbers are the ones the committed
ncu launch list of auag_like_4000 shows (317 launches per FP64 call, 539 per
split call) and the structure of the blocked algorithms for other sizes."""
import bench


def test_reduce_launch_counts_match_the_launch_list():
    assert bench._reduce_launches(4000, split=False) == 317
    assert bench._reduce_launches(4000, split=True) == 539


def test_reduce_launch_counts_structure():
    # FP64: per 64-column block a diagonal factorisation, a panel solve and an update
    # (none below the last block), per block row a solve and an update (none after the
    # last), plus zeroing, identity, P, G and G + G^H
    for n in (1, 64, 65, 300):
        nblk = (n + 63) // 64
        assert bench._reduce_launches(n, split=False) == 5 * nblk + 2
    # split, one 128-wide panel: the same FP64 launches and the 8 of the two-sided
    # products; a second panel adds the tensor-core updates of both chains
    assert bench._reduce_launches(128, split=True) == bench._reduce_launches(128, False) - 3 + 8
    assert bench._reduce_launches(129, split=True) > bench._reduce_launches(129, False) - 3 + 8
