"""Differentiable stress: torch.autograd functions over the C ABI.

``stress(X, layout)`` is f(X) of Eq. (1) with the hand-written force kernel
as its backward: d f / d X = -2 F with F = (L^X - L^W) X (``fd_forces``).

``stress_lengths(X, edge_len, row_ptr, col_idx)`` is f(X; l) for a weighted
graph whose ideal distances are shortest-path lengths in the edge lengths l
(Sec. 2, Sec. 5.4).  Its backward gives d f / d X (forces) and d f / d l
(``fd_energy_length_grad``: the pair derivatives summed along every pair's
shortest path).  ``edge_len`` holds each edge's length in both of its CSR
entries; the function reads an edge's length as the mean of its two entries,
so each entry receives half of the edge's derivative (a per-edge parameter
scattered to both entries gets the whole derivative back).  Each forward
call rebuilds the distances for the current lengths (``fd_layout_create``).

Argument marshalling only: every value comes from the CUDA library.
"""
from __future__ import annotations

import torch

from . import api


class _Stress(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, layout):
        Xc = X.detach().contiguous()
        ctx.layout = layout
        ctx.save_for_backward(Xc)
        return torch.tensor(layout.energy(Xc), dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(ctx, g):
        (Xc,) = ctx.saved_tensors
        F = ctx.layout.forces(Xc)
        return (-2.0 * g).to(F.dtype) * F, None


def stress(X: torch.Tensor, layout: api.Layout) -> torch.Tensor:
    """f(X) (FP64 scalar tensor); differentiable in X."""
    return _Stress.apply(X, layout)


class _StressLengths(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, edge_len, row_ptr, col_idx):
        Xc = X.detach().contiguous()
        lc = edge_len.detach().contiguous()
        L = api.Layout(row_ptr, col_idx, dim=int(X.shape[1]), edge_len=lc, stream=None)
        f, gl = L.length_grad(Xc)
        F = L.forces(Xc)
        L.close()
        ctx.save_for_backward(F, gl)
        return torch.tensor(f, dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(ctx, g):
        F, gl = ctx.saved_tensors
        gx = (-2.0 * g).to(F.dtype) * F if ctx.needs_input_grad[0] else None
        gw = (0.5 * g).to(gl.dtype) * gl if ctx.needs_input_grad[1] else None
        return gx, gw, None, None


def stress_lengths(X: torch.Tensor, edge_len: torch.Tensor, row_ptr, col_idx) -> torch.Tensor:
    """f(X; l) for a weighted graph; differentiable in X and in the edge
    lengths l (float32, one per CSR entry, equal for an edge's two entries)."""
    return _StressLengths.apply(X, edge_len, row_ptr, col_idx)
