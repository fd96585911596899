"""Differentiable typed pack (halo gathers inside differentiable solvers).

`typed_pack(x, dtype, count, offset)` packs `count` elements of a float32
layout whose displacement 0 is element `offset` of the flat tensor `x`, and
returns the packed float32 vector.  Its backward is the adjoint of the pack,
computed by the library's `dte_pack_adjoint_f32_enqueue` kernels: a
scatter-add that is bit-exact for layouts without repeated entries and a
deterministic FP64 segmented sum for layouts that repeat entries.  Both
directions run on the current CUDA stream; this module only marshals
pointers.
"""
from __future__ import annotations

import torch

from . import Datatype, _check_span, dte_pack_adjoint_f32_enqueue, dte_pack_enqueue


class TypedPack(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, dtype: Datatype, count: int, offset: int):
        if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
            raise TypeError("typed_pack expects a contiguous float32 CUDA tensor")
        _check_span("typed_pack input", 4 * x.numel(), 4 * offset, count, dtype)
        n = count * dtype.size // 4
        out = torch.empty(n, dtype=torch.float32, device=x.device)
        stream = torch.cuda.current_stream(x.device).cuda_stream
        dte_pack_enqueue(x.data_ptr() + 4 * offset, count, dtype.h, out.data_ptr(), 4 * n, 0, stream)
        ctx.dtype, ctx.count, ctx.offset = dtype, count, offset
        ctx.shape = x.shape
        return out

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        gy = gy.contiguous()
        if gy.dtype != torch.float32:
            gy = gy.float()
        gx = torch.zeros(ctx.shape, dtype=torch.float32, device=gy.device)
        stream = torch.cuda.current_stream(gy.device).cuda_stream
        dte_pack_adjoint_f32_enqueue(gy.data_ptr(), ctx.count, ctx.dtype.h, gx.data_ptr() + 4 * ctx.offset, stream)
        return gx, None, None, None


def typed_pack(x: torch.Tensor, dtype: Datatype, count: int = 1, offset: int = 0) -> torch.Tensor:
    """Pack a float32 layout out of `x` (differentiable in `x`)."""
    return TypedPack.apply(x, dtype, count, offset)
