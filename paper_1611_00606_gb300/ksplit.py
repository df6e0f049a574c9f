"""K-split of one k-point over atoms, across the ranks of a process group.

The paper's multi-GPU experiments (Sec. 4, Tabs. 2-5) spread the five large BLAS
calls of one k-point over 1, 2 or 4 GPUs.  Here the natural cut of Eqs. (h) and (s)
is used instead: both are sums over atoms, so with the atoms split into disjoint
ranges r,

    H = sum_r H_r,   S = sum_r S_r,   H_r, S_r = the terms of the atoms of range r.

Rank r assembles H_r and S_r with ``hs_assemble_partial`` (its own Cholesky of its
atoms' T^AA, its own fallback atoms, its own per-atom products and stacked
contractions, lower triangles only), the ranks add the partials with one collective
sum of the two N_G x N_G buffers, and every rank fills the upper triangles of the
sums with ``hs_finalize``.  That collective is the only exchange; the inputs of a
rank are the rows of A and B and the T, U blocks of its atoms.

Partition: ``atom_range`` gives rank r the atoms [a0, a1) of an even split (the
first N_A mod W ranks take one atom more).  Atoms whose Cholesky fails are found
and counted by the rank that owns them.

This module does argument marshalling and the collective only; every step of the
assembly runs in libhs's kernels.  It imports the binding lazily, so the partition
and the reduction can be used (and tested) without a GPU.
"""
from __future__ import annotations


def atom_range(N_A: int, rank: int, world: int) -> tuple:
    """(a0, a1): the atoms of ``rank`` in an even split of N_A atoms over ``world`` ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("atom_range: need 0 <= rank < world")
    if N_A < world:
        raise ValueError(f"atom_range: {N_A} atoms cannot give each of {world} ranks one")
    base, extra = divmod(N_A, world)
    a0 = rank * base + min(rank, extra)
    return a0, a0 + base + (1 if rank < extra else 0)


def sum_over_ranks(H, S, group=None) -> None:
    """Add H and S (N_G x N_G, column-major views of contiguous buffers) over the ranks
    of ``group``, in place: one all-reduce per matrix on the contiguous storage."""
    import torch
    import torch.distributed as dist
    for X in (H, S):
        buf = X.T if not X.is_contiguous() else X  # the (contiguous) storage order
        if not buf.is_contiguous():
            raise ValueError("sum_over_ranks: H and S must be views of contiguous buffers")
        # complex values as (re, im) float64 pairs: a plain elementwise sum for any backend
        dist.all_reduce(torch.view_as_real(buf), op=dist.ReduceOp.SUM, group=group)


class KSplitPlan:
    """One rank's share of a K-split assembly: a plan for its atom range.

    ``assemble`` takes the FULL stacked inputs (A, B: (N_A*N_L, N_G) column-major with
    leading dimension N_A*N_L; T_*: (N_A, N_L, N_L); U: (N_A, N_L)) on this rank's
    device, assembles the partial of this rank's atoms, sums over the group and
    finalises, so every rank ends with the full H and S.
    """

    def __init__(self, N_A: int, N_L: int, N_G_max: int, precision: str = "split_bf16",
                 slices: int = 0, rank: int = 0, world: int = 1, stream=None):
        from . import hs
        self.N_A, self.N_L = N_A, N_L
        self.a0, self.a1 = atom_range(N_A, rank, world)
        self.plan = hs.Plan(self.a1 - self.a0, N_L, N_G_max, precision, slices, 0, stream)

    def partial(self, A, B, T_AA, T_AB, T_BB, U, N_G: int, H, S) -> dict:
        """H_r, S_r of this rank's atoms (lower triangles) into H, S."""
        from . import hs
        a0, a1, N_L = self.a0, self.a1, self.N_L
        r = slice(a0 * N_L, a1 * N_L)
        return hs.hs_assemble_partial(self.plan.h, A[r], B[r], T_AA[a0:a1], T_AB[a0:a1],
                                      T_BB[a0:a1], U[a0:a1], a1 - a0, N_L, N_G, H, S)

    def set_t(self, T_AA, T_AB, T_BB) -> None:
        """Re-factorise this rank's T^AA blocks (after T changed in place)."""
        from . import hs
        a0, a1 = self.a0, self.a1
        hs.hs_set_t(self.plan.h, T_AA[a0:a1], T_AB[a0:a1], T_BB[a0:a1])

    def assemble(self, A, B, T_AA, T_AB, T_BB, U, N_G: int, H, S, group=None) -> dict:
        from . import hs
        info = self.partial(A, B, T_AA, T_AB, T_BB, U, N_G, H, S)
        if self.a1 - self.a0 < self.N_A:  # more than one range: add the partials up
            sum_over_ranks(H, S, group)
        hs.hs_finalize(self.plan.h, H, S, N_G)
        return info

    def close(self):
        self.plan.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
