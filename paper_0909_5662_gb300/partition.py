"""Operator partition across ranks.

Uniform-matrix distribution (Sec. 3.2): with p ranks, each owns floor(L/p)
contiguous operators and the first L mod p ranks own one more.  On one GPU the
whole batch goes into one launch; across GPUs each rank rotates its own
contiguous slice with no data-path collective (U is replicated, as R is on
every node in the paper).
"""
from __future__ import annotations

from typing import Tuple


def umd_partition(L: int, p: int, rank: int) -> Tuple[int, int]:
    if p < 1 or not (0 <= rank < p) or L < 0:
        raise ValueError("need p >= 1, 0 <= rank < p and L >= 0")
    base, extra = divmod(L, p)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)
