"""Differentiable BTO flow map: a torch.autograd.Function over libbto's tape.

``FlowMap.apply(seeds, fields, tape, dt)`` advances particles from ``seeds``
(P x 3, physical) through ``fields`` (L x (nz+1) x (ny+1) x (nx+1) x 3, one
F3 node field per cycle) with one RK4 step per cycle and closed-box
termination (Sec. 3.1), and returns the end positions (the basis flows,
Sec. 2.3), the valid flags and the exit cycles. Its backward pass runs the
checkpointed discrete adjoint kernels of libbto and returns the gradients
with respect to the seeds and to every cycle's node velocities. Only
argument marshalling happens here; all arithmetic runs in libbto.

``ftle(tape, seeds, fields, dt)`` returns the flow-map Jacobian (three
reverse sweeps) and the finite-time Lyapunov exponent of every particle that
stays in its block for the interval.
"""
from __future__ import annotations

import torch

from . import bto


class Tape:
    """Owning handle of a libbto tape (one block, P particles, L cycles,
    positions kept every ``checkpoint_every`` cycles)."""

    def __init__(self, extent, origin, spacing, num_particles, cycles, checkpoint_every=16):
        self.handle = bto.bto_tape_create(extent, origin, spacing, num_particles, cycles, checkpoint_every)
        self.extent = tuple(int(v) for v in extent)
        self.P = int(num_particles)
        self.L = int(cycles)
        self.generation = 0        # forwards run; a backward must belong to the last one

    def close(self):
        if self.handle:
            bto.bto_tape_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _field_table(fields):
    return torch.tensor([fields[c].data_ptr() for c in range(fields.shape[0])], dtype=torch.int64,
                        device=fields.device)


def _check_inputs(seeds, fields, tape):
    if seeds.dtype != torch.float32 or fields.dtype != torch.float32:
        raise TypeError("seeds and fields must be float32")
    if not (seeds.is_cuda and fields.is_cuda):
        raise ValueError("seeds and fields must be CUDA tensors")
    n = tape.extent
    want = (tape.L, n[2] + 1, n[1] + 1, n[0] + 1, 3)
    if tuple(fields.shape) != want:
        raise ValueError(f"fields shape {tuple(fields.shape)} != {want}")
    if tuple(seeds.shape) != (tape.P, 3):
        raise ValueError(f"seeds shape {tuple(seeds.shape)} != {(tape.P, 3)}")


class FlowMap(torch.autograd.Function):
    @staticmethod
    def forward(ctx, seeds, fields, tape, dt):
        _check_inputs(seeds, fields, tape)
        seeds_c = seeds.detach().contiguous()
        fields_c = fields.detach().contiguous()
        table = _field_table(fields_c)
        P = tape.P
        ends = torch.empty((P, 3), dtype=torch.float32, device=seeds.device)
        valid = torch.empty((P,), dtype=torch.uint8, device=seeds.device)
        exit_cycle = torch.empty((P,), dtype=torch.int32, device=seeds.device)
        bto.bto_tape_forward(tape.handle, seeds_c, table, dt, ends, valid, exit_cycle)
        tape.generation += 1
        ctx.tape = tape
        ctx.generation = tape.generation
        ctx.keep = (seeds_c, fields_c, table)     # the tape reads them in backward
        ctx.mark_non_differentiable(valid, exit_cycle)
        return ends, valid, exit_cycle

    @staticmethod
    def backward(ctx, g_ends, g_valid, g_exit):
        tape = ctx.tape
        if tape.generation != ctx.generation:
            raise RuntimeError("the tape ran another forward since this one; backward would be wrong")
        seeds_c, fields_c, _ = ctx.keep
        grad_seeds = torch.empty_like(seeds_c)
        grad_fields = None
        gtable = None
        if ctx.needs_input_grad[1]:
            grad_fields = torch.zeros_like(fields_c)
            gtable = _field_table(grad_fields)
        bto.bto_tape_backward(tape.handle, g_ends.contiguous(), grad_seeds, gtable)
        return (grad_seeds if ctx.needs_input_grad[0] else None), grad_fields, None, None


def flow_map(seeds, fields, tape, dt):
    """(ends, valid, exit_cycle) with gradients through ``ends``."""
    return FlowMap.apply(seeds, fields, tape, dt)


def ftle(tape, seeds, fields, dt):
    """Forward, flow-map Jacobian (P x 3 x 3, d end / d seed) and FTLE (NaN
    for particles that leave the block)."""
    _check_inputs(seeds, fields, tape)
    seeds_c = seeds.detach().contiguous()
    fields_c = fields.detach().contiguous()
    table = _field_table(fields_c)         # must outlive the Jacobian sweeps below
    P = tape.P
    dev = seeds.device
    ends = torch.empty((P, 3), dtype=torch.float32, device=dev)
    valid = torch.empty((P,), dtype=torch.uint8, device=dev)
    bto.bto_tape_forward(tape.handle, seeds_c, table, dt, ends, valid, None)
    tape.generation += 1
    jac = torch.empty((P, 9), dtype=torch.float32, device=dev)
    bto.bto_tape_jacobian(tape.handle, jac)
    out = torch.empty((P,), dtype=torch.float32, device=dev)
    bto.bto_tape_ftle(tape.handle, jac, out)
    torch.cuda.current_stream().synchronize()
    return ends, valid, jac.view(P, 3, 3), out
