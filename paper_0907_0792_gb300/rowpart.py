"""Row partition of the generalized inner product over the ranks of a
process group (one process per GPU).

The psi-flattening (Fig. 1) makes row i of the result D depend on row i of
the left operand A and on all of B, and on nothing else, so the M result
rows split into contiguous blocks, one per rank, with no reduction between
ranks for any (reduce, combine) pair: this is the paper's distribution of
result rows over threads (Sec. II, one row per thread; the appendix deals
rows to threads), with ranks in place of threads and a block of rows in
place of one.  The only exchange is one broadcast of B from the rank that
holds it; each rank then computes its block with ``moa_inner`` on its own
device.  ``gather_rows`` reassembles D where a caller wants it whole.

Host logic only: the collectives are torch.distributed calls (NCCL between
GPUs, gloo on CPU), the arithmetic is the library's (or, in tests without a
GPU, whatever ``compute`` is given).
"""
from __future__ import annotations

import math


def row_block(M: int, world: int, rank: int):
    """Rows [r0, r1) of rank ``rank``: contiguous blocks whose sizes differ
    by at most one, the first M % world ranks one row longer."""
    if world < 1 or not 0 <= rank < world or M < 0:
        raise ValueError("bad partition")
    base, extra = divmod(M, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def flat_extents(shapeA, shapeB):
    """(M, K, N) of Eq. (2) for rho A = <..., p> and rho B = <p, ...>."""
    if len(shapeA) < 1 or len(shapeB) < 1 or shapeA[-1] != shapeB[0]:
        raise ValueError("the last axis of A must match the first axis of B")
    return math.prod(shapeA[:-1]), shapeA[-1], math.prod(shapeB[1:])


def broadcast_operand(B, src: int = 0, group=None):
    """B (a tensor of the same shape and type on every rank) from rank ``src``
    to all ranks, in place."""
    import torch.distributed as dist
    dist.broadcast(B, src=src, group=group)
    return B


def sharded_inner(reduce, combine, dtype, form, A_rows, B, out_rows, out_dtype, compute=None, stream=None):
    """This rank's block of D = reduce_p(A combine B): A_rows is the rank's
    block of the flattened A (rows x K), out_rows its block of D (rows x N),
    B the whole right operand (K x N, after ``broadcast_operand``).  By
    default the block runs through the library's moa_inner on the rank's
    device; ``compute(A_rows, B, out_rows)`` replaces it (CPU tests)."""
    rows, K = A_rows.shape
    if B.shape[0] != K or tuple(out_rows.shape) != (rows, B.shape[1]):
        raise ValueError("block shapes do not match")
    if compute is not None:
        compute(A_rows, B, out_rows)
        return out_rows
    from . import moa_inner
    moa_inner(reduce, combine, dtype, form, (rows, K), A_rows, (K, B.shape[1]), B, out_rows, out_dtype, stream)
    return out_rows


def gather_rows(out_rows, M: int, group=None):
    """The whole M x N result on every rank from the ranks' row blocks
    (blocks padded to the longest one for the collective, then trimmed)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    longest = row_block(M, world, 0)[1]
    N = out_rows.shape[1]
    pad = torch.zeros((longest, N), dtype=out_rows.dtype, device=out_rows.device)
    pad[: out_rows.shape[0]] = out_rows
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    blocks = []
    for r in range(world):
        r0, r1 = row_block(M, world, r)
        blocks.append(parts[r][: r1 - r0])
    return torch.cat(blocks, dim=0)
