"""Row-sharded products across processes (one GPU per process, torch.distributed).

The rows of P = A ⊗ B are independent (Section 2 product formula), so a product over N
ranks splits A and C by row blocks (sr_shard_rows: whole 128-row tile groups, balanced)
and replicates B; each rank computes its rows with the library's own product call and
no reduction follows.  Only moving the operands is collective: B is broadcast from the
rank that holds it, and the row blocks of C can be gathered where the whole result is
wanted.  The local product is the caller's (the C-ABI antidist_mul / bool_mul on this
rank's GPU), passed in as `local_mul(A_rows, B, C_rows)`.
"""

from __future__ import annotations

from . import _capi


def my_rows(R: int, rank: int, world: int, align: int = 128):
    """This rank's row range [r0, r1)."""
    return _capi.sr_shard_rows(R, world, rank, align)


def sharded_mul(local_mul, A, B, rank: int, world: int, group=None, src: int = 0, gather: bool = True,
                align: int = 128):
    """C = A ⊗ B with rows split over the ranks of `group`.

    A: the full R x K operand on every rank, or None where only the rows are needed
    (each rank then passes its own rows via A, shaped (r1 - r0) x K).  B: K x N, held by
    rank `src` (other ranks pass a tensor of the same shape and dtype to receive it).
    Returns this rank's C rows, or with gather=True the full C on every rank."""
    import torch
    import torch.distributed as dist
    dist.broadcast(B, src=src, group=group)
    R = A.shape[0] if A is not None else None
    if R is None:
        raise ValueError("A is needed to know R")
    r0, r1 = my_rows(R, rank, world, align)
    C_rows = torch.zeros((r1 - r0, B.shape[1]), dtype=B.dtype, device=B.device)
    if r1 > r0:
        local_mul(A[r0:r1], B, C_rows)
    if not gather:
        return C_rows
    parts = []
    for r in range(world):
        a0, a1 = my_rows(R, r, world, align)
        parts.append(torch.empty((a1 - a0, B.shape[1]), dtype=B.dtype, device=B.device))
    if world == 1:
        return C_rows
    # uneven blocks: pad every block to the largest, gather, trim
    m = max(p.shape[0] for p in parts)
    padded = torch.zeros((m, B.shape[1]), dtype=B.dtype, device=B.device)
    padded[:C_rows.shape[0]] = C_rows
    outs = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(outs, padded, group=group)
    return torch.cat([o[:p.shape[0]] for o, p in zip(outs, parts)], dim=0)
