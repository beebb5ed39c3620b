"""Static sharding of independent Krylov bases over ranks.

The forward and adjoint solves of different right-hand sides (sources,
receivers) are independent (Sec. 5.3: the systems per source, receiver and
time are solved separately), so a multi-GPU run assigns whole right-hand
sides to ranks and needs no exchange inside a solve.
"""
from __future__ import annotations

from typing import List


def partition(n: int, rank: int, world: int) -> List[int]:
    """Contiguous block of item indices for `rank` (sizes differ by at most 1)."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad partition arguments")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return list(range(lo, hi))
