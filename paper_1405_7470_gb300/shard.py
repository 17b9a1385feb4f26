"""Element-range sharding across ranks (replicas with independent work).

Elements are independent in the contraction (the unordered semantics of Section 2.3:
any traversal order, or partition, of the e loop gives the same result), so a batch
splits into contiguous element ranges, one per rank, with the operators D replicated
and no exchange on the data path.  The only collective is a max of timings (and,
optionally, a sum of error-norm partials) at the end.
"""

from __future__ import annotations


def element_range(E: int, world: int, rank: int) -> tuple[int, int]:
    """[e0, e1) of rank `rank`: contiguous, sizes differing by at most one element."""
    if world < 1 or not 0 <= rank < world or E < 0:
        raise ValueError("bad sharding arguments")
    base, extra = divmod(E, world)
    e0 = rank * base + min(rank, extra)
    return e0, e0 + base + (1 if rank < extra else 0)


def shard_u(u, layout: str, e0: int, e1: int):
    """The rank's slice of u: rows e0..e1 (element-major) or columns (node-major)."""
    return u[e0:e1] if layout == "elem" else u[:, e0:e1]
