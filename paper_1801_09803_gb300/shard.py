"""Host-side partition of one cross-section problem over ranks.

The path shards along the wavenumber grid without any reduction: rank r owns
the contiguous grid range [k0, k1) and needs only the lines whose cut can
reach it, i.e. wavenumbers in [nu_k0 - cut, nu_(k1-1) + cut] -- a contiguous
range of the sorted list (a halo of one cutoff on each side).  Each rank's
result is the exact slice of the full cross section (every grid point sums the
same lines), so concatenating the slices reproduces the single-GPU result.

Independent problems (different line lists or condition sets per rank) need
no partition at all; the benchmark uses that form (weak scaling).
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def grid_shard(n_pts: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous, balanced grid range [k0, k1) of rank `rank` out of `world`."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, extra = divmod(int(n_pts), world)
    k0 = rank * base + min(rank, extra)
    k1 = k0 + base + (1 if rank < extra else 0)
    return k0, k1


def halo_line_range(nu_sorted: np.ndarray, nu_A: float, step: float, k0: int, k1: int,
                    cutoff: float) -> Tuple[int, int]:
    """Index range [l0, l1) of the sorted lines whose cut can reach points k0..k1-1."""
    if k1 <= k0:
        return 0, 0
    x0 = nu_A + k0 * step
    x1 = nu_A + (k1 - 1) * step
    margin = cutoff * (1.0 + 1e-12) + 1e-12 * (abs(x0) + abs(x1))
    l0 = int(np.searchsorted(nu_sorted, x0 - margin, side="left"))
    l1 = int(np.searchsorted(nu_sorted, x1 + margin, side="right"))
    return l0, l1
