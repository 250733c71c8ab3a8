"""Host-side bookkeeping of a z-slab decomposition of one lattice across ranks.

Each rank owns a contiguous range of z planes. One time step needs, from each
neighbour, the populations that cross the shared face: with the pull scheme of
the GPU kernel these are the 5 post-collision populations with e_z = +1
(Z_PLUS, Eq. A1 order) of the plane below the face and the 5 with e_z = -1
(Z_MINUS) of the plane above it. A solver that stores the post-streaming state
(as the FP64 oracle does) exchanges whole boundary planes instead and steps a
slab extended by one ghost plane on each side. Holds no method arithmetic.
"""
from __future__ import annotations

from typing import List, Tuple

import torch

Z_PLUS = (5, 11, 12, 15, 16)
Z_MINUS = (6, 13, 14, 17, 18)


def partition(nz: int, world: int) -> List[Tuple[int, int]]:
    """Balanced [z0, z1) ranges, one per rank (earlier ranks take the remainder)."""
    if world < 1 or nz < world:
        raise ValueError("need 1 <= world <= nz")
    base, rem = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < rem else 0)
        out.append((z, z + n))
        z += n
    return out


def neighbours(rank: int, world: int) -> Tuple[int, int]:
    """(lower, upper) neighbour ranks along a periodic z axis."""
    return (rank - 1) % world, (rank + 1) % world


def exchange_planes(local: torch.Tensor, rank: int, world: int, dist) -> Tuple[torch.Tensor, torch.Tensor]:
    """Send the bottom plane down and the top plane up; return (ghost_below,
    ghost_above): the upper plane of the lower neighbour and the lower plane of
    the upper neighbour. local: (Q, nz_local, ny, nx), contiguous."""
    lo, hi = neighbours(rank, world)
    bottom = local[:, 0].contiguous()
    top = local[:, -1].contiguous()
    ghost_below = torch.empty_like(bottom)
    ghost_above = torch.empty_like(top)
    if world == 1:
        return top.clone(), bottom.clone()
    reqs = [dist.isend(top, hi), dist.isend(bottom, lo), dist.irecv(ghost_below, lo), dist.irecv(ghost_above, hi)]
    for r in reqs:
        r.wait()
    return ghost_below, ghost_above
