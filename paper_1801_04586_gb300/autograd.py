"""Differentiable unroll: the final Eq. 9 velocity as a function of a body-force
field, with gradients from the hand-written adjoint kernel.

Forward runs `nsteps` lattice steps from a fixed initial raw state, keeping a
checkpoint of the raw state every `every` steps. Backward walks the segments
from last to first with one clbm_adjoint_segment call each: the segment's
states are recomputed from its checkpoint straight into a tape (no extra
copies), then the adjoint step kernel runs back to front, accumulating dL/dF. Memory: one checkpoint per
segment plus one tape of `every` states.
"""
from __future__ import annotations

import torch

from .lattice import Lattice


class ForceToVelocity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F: torch.Tensor, lattice: Lattice, init_state: torch.Tensor, nsteps: int, every: int):
        if lattice.storage != "f32":
            raise ValueError("the adjoint supports FP32 storage only")
        F = F.detach().contiguous()
        lattice.set_force_field(F)
        lattice.import_state(init_state, set_steps=0)
        ckpts = []
        t = 0
        while t < nsteps:
            k = min(every, nsteps - t)
            ckpts.append((k, lattice.export_state()))
            lattice.step(k)
            t += k
        _, u = lattice.macros()
        ctx.lattice = lattice
        ctx.ckpts = ckpts
        ctx.final = lattice.export_state()
        ctx.F = F
        ctx.every = every
        return u

    @staticmethod
    def backward(ctx, gu: torch.Tensor):
        lat: Lattice = ctx.lattice
        lat.set_force_field(ctx.F)
        gu = gu.detach().to(torch.float32).contiguous()
        lam = lat.empty(19, *lat.shape)
        lam2 = lat.empty(19, *lat.shape)
        gF = lat.empty(3, *lat.shape)
        lat.adjoint_seed(gu, lam, gF, state=ctx.final)
        nb = lat.state_bytes()
        tape = torch.empty(max(ctx.every - 1, 1) * nb, dtype=torch.uint8, device=lat.device)
        for k, ck in reversed(ctx.ckpts):
            lat.adjoint_segment(ck, tape, k, lam, lam2, gF)
        ctx.ckpts = None
        return gF, None, None, None, None


def final_velocity(F: torch.Tensor, lattice: Lattice, init_state: torch.Tensor, nsteps: int,
                   every: int = 20) -> torch.Tensor:
    """u(x, nsteps) (3, nz, ny, nx) after nsteps steps from init_state under the
    force field F (3, nz, ny, nx); differentiable with respect to F."""
    return ForceToVelocity.apply(F, lattice, init_state, int(nsteps), int(every))
