"""torch.autograd face of the discrete adjoint (fv_adjoint_vjp).

``RKStage`` runs one Runge-Kutta stage through the C ABI in forward and its
vector-Jacobian product in backward.  Each stage keeps its input state as the
checkpoint the adjoint kernels linearise around (stage checkpointing), so a
chain of stages can be differentiated end to end by torch.  The tensors are
packed ghosted states (float64, on the GPU); gradients flow through interior
cells only - fixed ghost values are constants of the problem.

Memory: a plain chain keeps one state per stage (the stage inputs, which
the chain holds anyway; nothing is copied), O(stages).  With ``segment`` =
k steps, ``run_stages`` keeps only the input of every k-th step and
recomputes a segment's stages (deterministically, so the gradient is the
same bit for bit) when its backward runs: about (stages / (k M) + k M)
states.

Everything numerical runs in the library's kernels; this module copies
states in and out of the library's buffers and maps between the packed
ghosted layout and the packed interior field (index gathers).
"""
from __future__ import annotations

import torch


def _interior_index(solver) -> torch.Tensor:
    """Positions, in the packed ghosted state, of the interior cells in
    packed-interior-field order (per block: variable, k, j, i)."""
    idx = getattr(solver, "_interior_idx", None)
    if idx is not None:
        return idx
    parts, off = [], 0
    for b in solver.block_dims:
        ni, nj, nk = b
        gi, gj, gk = ni + 4, nj + 4, nk + 4
        v = torch.arange(5, dtype=torch.int64).view(5, 1, 1, 1)
        k = torch.arange(2, nk + 2, dtype=torch.int64).view(1, nk, 1, 1)
        j = torch.arange(2, nj + 2, dtype=torch.int64).view(1, 1, nj, 1)
        i = torch.arange(2, ni + 2, dtype=torch.int64).view(1, 1, 1, ni)
        parts.append((off + ((v * gk + k) * gj + j) * gi + i).reshape(-1))
        off += 5 * gi * gj * gk
    idx = torch.cat(parts).cuda()
    solver._interior_idx = idx
    return idx


def interior(solver, q: torch.Tensor) -> torch.Tensor:
    return q.index_select(0, _interior_index(solver))


def scatter_interior(solver, field: torch.Tensor) -> torch.Tensor:
    out = torch.zeros(solver.state_size, dtype=torch.float64, device=field.device)
    out.index_copy_(0, _interior_index(solver), field)
    return out


class RKStage(torch.autograd.Function):
    """Q^(m) = Q^(0) - alpha_m dt / Omega R(X(Q^(m-1))) for stage m."""

    @staticmethod
    def forward(ctx, q0, qin, solver, m: int, dt: float):
        src, dst = solver.stage_buffers(m)
        solver.set_buffer(0, q0.detach().contiguous())
        if m > 1:
            solver.set_buffer(src, qin.detach().contiguous())
        solver.rk_stage(m, dt)
        out = solver.get_state(dst)
        # stage checkpoint: the input itself (stage outputs are fresh tensors
        # nobody writes in place, so no copy is needed)
        ctx.save_for_backward(qin)
        ctx.solver, ctx.m, ctx.dt = solver, m, dt
        return out

    @staticmethod
    def backward(ctx, gout):
        (qin,) = ctx.saved_tensors
        s = ctx.solver
        lam_out = interior(s, gout.contiguous())
        lam_in = torch.empty_like(lam_out)
        lam_q0 = torch.zeros_like(lam_out)
        s.adjoint_vjp(ctx.m, ctx.dt, qin, lam_out, lam_in, lam_q0)
        return scatter_interior(s, lam_q0), scatter_interior(s, lam_in), None, None, None


def _chain(solver, q: torch.Tensor, dt: float, first: int, count: int) -> torch.Tensor:
    """Stages first .. first+count-1 of the global stage sequence from q,
    the input of stage index ``first`` (a step boundary)."""
    M = solver.n_stages
    q0 = q
    cur = q
    for st in range(first, first + count):
        m = st % M + 1
        if m == 1:
            q0 = cur
        cur = RKStage.apply(q0, cur, solver, m, dt)
    return cur


def run_stages(solver, q: torch.Tensor, dt: float, nstages: int, segment: int = 0) -> torch.Tensor:
    """Differentiable chain of ``nstages`` RK stages (whole steps of M stages,
    the last possibly partial) starting from packed ghosted state ``q``.
    ``segment`` > 0: recompute each run of ``segment`` steps in backward
    instead of keeping its stage checkpoints (torch.utils.checkpoint)."""
    if segment <= 0 or not q.requires_grad:
        return _chain(solver, q, dt, 0, nstages)
    from torch.utils.checkpoint import checkpoint
    span = segment * solver.n_stages
    cur = q
    for first in range(0, nstages, span):
        count = min(span, nstages - first)
        cur = checkpoint(_chain, solver, cur, dt, first, count, use_reentrant=False)
    return cur
