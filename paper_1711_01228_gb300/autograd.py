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

``unrolled_layout(X0, l, row_ptr, col_idx, K, omega, every)`` is X^K after K
iterations of Algorithm 2, differentiable in X0 and l through the adjoint of
each iteration (checkpoints every ``every`` iterations).

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


class _Unrolled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X0, edge_len, row_ptr, col_idx, K, omega, every, cg_tol, cg_max, omega_vertex, solver):
        lens = edge_len.detach().contiguous()
        L = api.Layout(row_ptr, col_idx, dim=int(X0.shape[1]), edge_len=lens, stream=None)
        if omega_vertex is not None:
            L.set_vertex_omega(omega_vertex)
        if solver == api.SOLVER_DIRECT:
            L.factor()  # one factorisation serves every forward, recomputed and adjoint solve
        opts = dict(omega=float(omega), strategy=api.OMEGA_FIXED, cg_tol=cg_tol, cg_max=cg_max, solver=int(solver))
        X = X0.detach().contiguous().clone()
        ckpt = {0: X.clone()}
        # one launch per checkpoint segment: tol = 0 runs exactly the
        # segment's iterations (the backward pass recomputes them one by one)
        for s0 in range(0, K, every):
            L.run(X, max_iter=min(every, K - s0), tol=0.0, **opts)
            if s0 + every < K:
                ckpt[s0 + every] = X.clone()
        ctx.L, ctx.ckpt, ctx.K, ctx.every, ctx.opts = L, ckpt, K, every, opts
        ctx.lens_dtype = edge_len.dtype
        return X

    @staticmethod
    def backward(ctx, gXK):
        L, K, every, opts = ctx.L, ctx.K, ctx.every, ctx.opts
        L.adjoint_reset()
        xbar = gXK.detach().contiguous().clone()
        for s in reversed(range(0, K, every)):
            # recompute the layouts of this segment from its checkpoint
            X = ctx.ckpt[s].clone()
            traj, accs = [X.clone()], []
            for k in range(s, min(s + every, K)):
                _, acc, _ = L.sor_step(X, k=k, **opts)
                traj.append(X.clone())
                accs.append(acc)
            for k in reversed(range(len(accs))):
                xbar, _ = L.sor_step_adjoint(traj[k], traj[k + 1], accs[k], opts["omega"], xbar,
                                             cg_tol=opts["cg_tol"], cg_max=opts["cg_max"], solver=opts["solver"])
        g_full = torch.empty(L._nnz, dtype=torch.float32, device=gXK.device)
        L.adjoint_length_grad(out=g_full)
        L.close()
        ctx.L = None
        return xbar, (0.5 * g_full).to(ctx.lens_dtype), None, None, None, None, None, None, None, None, None


def unrolled_layout(X0: torch.Tensor, edge_len: torch.Tensor, row_ptr, col_idx, K: int = 32, omega: float = 0.5,
                    every: int = 8, cg_tol: float = 1e-6, cg_max: int = 500, omega_vertex=None,
                    solver: int = api.SOLVER_CG) -> torch.Tensor:
    """X^K after K iterations of Algorithm 2 (fixed omega) from X0 on a
    weighted graph; differentiable in X0 and in the edge lengths.  The
    backward pass recomputes the layouts from checkpoints taken every
    ``every`` iterations and runs the adjoint of each iteration
    (``fd_sor_step_adjoint``; the acceptance of line 6 held at its forward
    outcome), then pushes the summed pair sensitivities through the shortest
    paths (``fd_adjoint_length_grad``).  As in ``stress_lengths``, each CSR
    entry of an edge receives half of the edge's derivative.  ``omega_vertex``:
    per-vertex factors m (omega_i = omega m_i, Sec. 6; not differentiated).
    ``solver=api.SOLVER_DIRECT`` factors L^W once (``fd_factor``) and uses the
    inverse in every solve, the adjoint ones included: they all share L^W."""
    return _Unrolled.apply(X0, edge_len, row_ptr, col_idx, int(K), float(omega), int(every), float(cg_tol),
                           int(cg_max), omega_vertex, int(solver))
