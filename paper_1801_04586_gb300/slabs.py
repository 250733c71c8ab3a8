"""Host-side driver of a z-slab decomposition of one lattice across ranks.

Each rank owns a contiguous range of z planes. One time step needs, from each
neighbour, the populations that cross the shared face (Eq. 8): with the pull
scheme of the GPU kernel these are the 5 post-collision populations with
e_z = +1 (Z_PLUS, Eq. A1 order) of the plane below the face and the 5 with
e_z = -1 (Z_MINUS) of the plane above it. A slab lattice of the library
(Lattice(..., slab=..., z0=...)) writes its outgoing faces into send planes
and pulls the incoming ones from receive planes; exchange_faces moves them
between ranks after every step, over torch.distributed point-to-point calls
(NCCL on device memory, or staged through host memory for gloo), or within
one rank for a single slab that is its own neighbour.

A solver that stores the post-streaming state (as the FP64 oracle does)
exchanges whole boundary planes instead and steps a slab extended by one
ghost plane on each side (exchange_planes). Holds no method arithmetic.
"""
from __future__ import annotations

from typing import List, Tuple

import torch

SLAB_LO, SLAB_HI = 1, 2
TAG_UP, TAG_DOWN = 11, 12  # faces travelling to the upper / lower neighbour

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


def _sum_over_ranks(v: torch.Tensor, dist) -> torch.Tensor:
    """In-place sum of an FP64 tensor over the ranks of the default group (the
    device tensor itself with NCCL, a host copy with gloo); unchanged with one
    rank or dist None."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return v
    if dist.get_backend() == "nccl":
        dist.all_reduce(v)
        return v
    h = v.cpu()
    dist.all_reduce(h)
    v.copy_(h)
    return v


def global_moments(lat, dist=None) -> torch.Tensor:
    """FP64 [total mass, total momentum x, y, z] (Eq. 9) of the whole lattice:
    this slab's sums (reduce_moments, exact fixed-point totals) added over the
    ranks by an FP64 all-reduce."""
    return _sum_over_ranks(lat.reduce_moments(), dist)


def global_pair(lat, a: torch.Tensor, b: torch.Tensor = None, dist=None) -> torch.Tensor:
    """FP64 [sum (a-b)^2, sum b^2, sum a b] over the whole lattice, for fields
    split across the slabs like the populations (L2 error norms, the dot
    products of a finite-difference check): reduce_pair on this slab's part,
    added over the ranks by an FP64 all-reduce."""
    return _sum_over_ranks(lat.reduce_pair(a, b), dist)


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


def slab_of(nz: int, rank: int, world: int, periodic_z: bool = True) -> Tuple[int, int, int]:
    """(z0, nz_local, slab bits) of rank's slab of an nz-plane lattice. A
    periodic z axis gives every slab both halo faces (one rank: its own
    neighbour); with z walls the first slab's z- face and the last slab's z+
    face are walls instead."""
    z0, z1 = partition(nz, world)[rank]
    if periodic_z:
        bits = SLAB_LO | SLAB_HI
    else:
        bits = (SLAB_LO if rank > 0 else 0) | (SLAB_HI if rank < world - 1 else 0)
    return z0, z1 - z0, bits


_SIDE_STREAMS = {}


def _side_stream(device) -> torch.cuda.Stream:
    """One stream per device for the face copies of self-neighbouring slabs."""
    key = torch.device(device).index
    if key not in _SIDE_STREAMS:
        _SIDE_STREAMS[key] = torch.cuda.Stream(device=device)
    return _SIDE_STREAMS[key]


def _self_copies(send, recv, half, has_lo, has_hi):
    """A slab's own outgoing faces into its receive planes (on the current stream)."""
    if has_hi:
        recv[:half].copy_(send[half:])
    if has_lo:
        recv[half:].copy_(send[:half])


class _StreamJoin:
    """An unwaited transfer on another stream: wait() makes the current stream wait for it."""

    def __init__(self, done: torch.cuda.Event):
        self.done = done

    def wait(self):
        torch.cuda.current_stream().wait_event(self.done)


def exchange_faces(lat, rank: int, world: int, dist=None, host: bool = False, wait: bool = True) -> list:
    """After a step (or after its SLAB_FACES part): send this slab's outgoing
    faces to its z neighbours and receive theirs into the newest state's
    receive planes. The first half of `send` (the first plane's e_z = -1
    populations) goes down, into the lower neighbour's second receive half;
    the second half (the last plane's e_z = +1 populations) goes up, into the
    upper neighbour's first receive half. Messages going up are issued before
    those going down, so that with NCCL (which matches a pair's messages in
    order) two ranks that are each other's upper and lower neighbour pair
    them correctly. host=True stages the faces through host memory (gloo).
    With wait=False (device path) the transfers are returned unwaited, so
    that the caller can enqueue the interior part of the step before waiting:
    their wait() makes the current stream wait for them. For a slab that is
    its own neighbour they are device copies on a side stream, which start
    once the lattice's stream has passed the faces part."""
    send, recv = lat.faces()
    return exchange_views(send, recv, lat.slab, lat.stream, getattr(lat, "device", None), rank, world, dist, host,
                          wait)


def state_faces(lat, state: torch.Tensor) -> Tuple[torch.Tensor, torch.Tensor]:
    """(send, recv) byte views of the halo planes of a raw state buffer of
    `lat` (clbm_export_state layout: the population arrays, then 10 receive
    planes, then 10 send planes), as faces() gives them for the context's own
    state. For the recomputation of states by step_raw."""
    info = lat.info()
    elem = 4 if info["storage"] == 0 else 2
    plane = lat.nx * lat.ny
    base = info["q"] * info["pop_stride"] * elem
    b = state.view(torch.uint8)
    return b[base + 10 * plane * elem: base + 20 * plane * elem], b[base: base + 10 * plane * elem]


def lam_faces(lat, lam: torch.Tensor) -> Tuple[torch.Tensor, torch.Tensor]:
    """(send, recv) byte views of the halo planes of an adjoint array of a
    z-slab (Lattice.lam_numel floats: 19 x N, 10 receive planes, 10 send
    planes). The adjoint gathers lambda from the node each population streams
    into, so across a halo face it needs the upper neighbour's first plane
    (e_z = +1) and the lower neighbour's last plane (e_z = -1); adjoint_seed and
    adjoint_step write this slab's matching faces into the send planes."""
    plane = lat.nx * lat.ny
    base = 19 * lat.nz * plane * 4
    b = lam.view(torch.uint8)
    return b[base + 10 * plane * 4: base + 20 * plane * 4], b[base: base + 10 * plane * 4]


def exchange_adjoint_faces(lat, lam: torch.Tensor, rank: int, world: int, dist=None, host: bool = False,
                           wait: bool = True) -> list:
    """After adjoint_seed or adjoint_step wrote lam: its faces to the z
    neighbours and theirs into lam's receive planes, as exchange_faces does
    for the populations (the reverse-direction halo of the adjoint)."""
    send, recv = lam_faces(lat, lam)
    return exchange_views(send, recv, lat.slab, lat.stream, lat.device, rank, world, dist, host, wait)


def exchange_state_faces(lat, state: torch.Tensor, rank: int, world: int, dist=None, host: bool = False,
                         wait: bool = True) -> list:
    """After step_raw wrote the raw state `state`: its faces to the z
    neighbours and theirs into its receive planes."""
    send, recv = state_faces(lat, state)
    return exchange_views(send, recv, lat.slab, lat.stream, lat.device, rank, world, dist, host, wait)


def exchange_views(send: torch.Tensor, recv: torch.Tensor, slab: int, stream, device, rank: int, world: int,
                   dist=None, host: bool = False, wait: bool = True) -> list:
    """The exchange behind exchange_faces, on byte views: the first half of
    `send` goes down into the lower neighbour's second receive half, the
    second half up into the upper neighbour's first (see exchange_faces)."""
    half = send.numel() // 2
    has_lo, has_hi = bool(slab & SLAB_LO), bool(slab & SLAB_HI)
    with torch.cuda.stream(stream):
        if world == 1 or dist is None:
            # its own neighbour on both sides (a periodic z axis on one slab)
            if wait:
                _self_copies(send, recv, half, has_lo, has_hi)
                return []
            ready = torch.cuda.Event()
            ready.record(stream)
            side = _side_stream(device)
            side.wait_event(ready)
            with torch.cuda.stream(side):
                _self_copies(send, recv, half, has_lo, has_hi)
            done = torch.cuda.Event()
            done.record(side)
            return [_StreamJoin(done)]
        lo, hi = neighbours(rank, world)
        if host:
            send_h = send.cpu()
            recv_h = torch.empty(recv.numel(), dtype=torch.uint8)
            s_up, s_dn, r_lo, r_hi = send_h[half:], send_h[:half], recv_h[:half], recv_h[half:]
        else:
            s_up, s_dn, r_lo, r_hi = send[half:], send[:half], recv[:half], recv[half:]
        ops = []
        if has_hi:
            ops.append(("send", s_up, hi, TAG_UP))
        if has_lo:
            ops.append(("recv", r_lo, lo, TAG_UP))
        if has_lo:
            ops.append(("send", s_dn, lo, TAG_DOWN))
        if has_hi:
            ops.append(("recv", r_hi, hi, TAG_DOWN))
        if host:
            reqs = [dist.isend(t, p, tag=tag) if kind == "send" else dist.irecv(t, p, tag=tag)
                    for kind, t, p, tag in ops]
            for r in reqs:
                r.wait()
            if has_lo:
                recv[:half].copy_(recv_h[:half])
            if has_hi:
                recv[half:].copy_(recv_h[half:])
            return []
        if not ops:
            return []
        p2p = [dist.P2POp(dist.isend if kind == "send" else dist.irecv, t, p, tag=tag) for kind, t, p, tag in ops]
        reqs = dist.batch_isend_irecv(p2p)
        if wait:
            for r in reqs:
                r.wait()
            return []
        return reqs
