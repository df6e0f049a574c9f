"""K-split of one k-point over atoms (the multi-GPU form), host logic on CPU with gloo.

Eqs. (h) and (s) are sums over atoms, so partials over disjoint atom ranges add up to
the whole.  Each rank computes its range's partial with the ORACLE (no GPU here), the
package's collective sum adds them over a gloo process group, and every rank must
then hold the oracle's full H and S.  This pins the partition (``atom_range``) and the
reduction (``sum_over_ranks``) that the GPU path uses around ``hs_assemble_partial``.
World sizes 2 and 3, 127.0.0.1 rendezvous.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

from paper_1611_00606_gb300.ksplit import atom_range  # noqa: E402


def test_atom_range_is_an_even_partition():
    for N_A in range(1, 24):
        for world in range(1, min(N_A, 9) + 1):
            rs = [atom_range(N_A, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == N_A
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        atom_range(3, 0, 4)
    with pytest.raises(ValueError):
        atom_range(8, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, root, case, q):
    import sys
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import assemble, fail_flags, rel_frobenius
    from paper_1611_00606_gb300 import synth
    from paper_1611_00606_gb300.ksplit import atom_range, sum_over_ranks
    N_A, N_L, N_G, indef = case
    d = synth.make_inputs(synth.Workload("k", N_A, N_L, N_G, indef, seed=31))
    a0, a1 = atom_range(N_A, rank, world)
    r = slice(a0 * N_L, a1 * N_L)
    Hr, Sr = assemble(d["A"][r], d["B"][r], d["T_AA"][a0:a1], d["T_AB"][a0:a1],
                      d["T_BB"][a0:a1], d["U"][a0:a1], a1 - a0, N_L)
    # the GPU path's buffer layout: column-major (N_G, N_G) views of contiguous storage
    H = torch.empty((N_G, N_G), dtype=torch.complex128).T
    S = torch.empty((N_G, N_G), dtype=torch.complex128).T
    H.copy_(torch.from_numpy(Hr))
    S.copy_(torch.from_numpy(Sr))
    sum_over_ranks(H, S)
    Hf, Sf = assemble(d["A"], d["B"], d["T_AA"], d["T_AB"], d["T_BB"], d["U"], N_A, N_L)
    nf = int(fail_flags(d["T_AA"][a0:a1]).sum())
    q.put((rank, a0, a1, nf, rel_frobenius(H.numpy(), Hf), rel_frobenius(S.numpy(), Sf)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,case", [
    (2, (4, 16, 64, (3,))),        # the tiny shape's atoms; the failing atom on rank 1
    (3, (5, 9, 40, (0, 4))),       # uneven split (2, 2, 1); failing atoms on ranks 0 and 2
])
def test_partials_of_atom_ranges_sum_to_the_whole_gloo(root, world, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, root, case, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    N_A, indef = case[0], case[3]
    assert [o[1:3] for o in out] == [atom_range(N_A, r, world) for r in range(world)]
    # each rank counts the failing atoms it owns
    assert [o[3] for o in out] == [sum(1 for a in indef if o[1] <= a < o[2]) for o in out]
    for o in out:
        assert o[4] < 1e-14 and o[5] < 1e-14
