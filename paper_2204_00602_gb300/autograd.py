"""Differentiable mesh simulation: phases -> U(phi) -> output distribution -> KL.

torch.autograd.Function wrappers whose forward and backward passes are the
library's kernels (mesh forward/backward, factorised distribution, adjoint,
KL gradient); torch only holds the tensors and runs the autograd graph.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _abi as abi
from . import _host_occ, _stream, distribution_batched, num_outputs, workspace


def mesh_unitary(phases: torch.Tensor, m: int) -> torch.Tensor:
    """U(phi) [B, m, m] of the Clements mesh for phases [B, m(m-1)] (float64 CUDA)."""
    if not (phases.is_cuda and phases.dtype == torch.float64 and phases.dim() == 2 and phases.shape[1] == m * (m - 1)):
        raise TypeError(f"phases must be float64 CUDA [B, {m * (m - 1)}]")
    phases = phases.contiguous()
    B = phases.shape[0]
    U = torch.empty(B, m, m, dtype=torch.complex128, device=phases.device)
    abi.pcv_mesh_unitary(phases, B, m, U, _stream(phases.device))
    return U


def distribution_backward(U: torch.Tensor, input_occ, grad_amp: torch.Tensor) -> torch.Tensor:
    """dL/dU [B, m, m] from dL/da [B, N] (dL/dRe + i dL/dIm) over every output."""
    B, m = U.shape[0], U.shape[1]
    t = _host_occ(input_occ, m)
    gU = torch.empty_like(U)
    ws = workspace(abi.pcv_distribution_backward_workspace(B, m, int(t.sum())), U.device)
    abi.pcv_distribution_backward(U, B, m, t, grad_amp.contiguous(), gU, ws, 0 if ws is None else ws.numel(),
                                  _stream(U.device))
    return gU


def mesh_backward(phases: torch.Tensor, U: torch.Tensor, grad_U: torch.Tensor) -> torch.Tensor:
    B, m = U.shape[0], U.shape[1]
    g = torch.empty_like(phases)
    abi.pcv_mesh_backward(phases.contiguous(), B, m, U, grad_U.contiguous(), g, _stream(U.device))
    return g


def dist_stats(p: torch.Tensor, q: torch.Tensor | None = None) -> torch.Tensor:
    """[B, 3]: sum p, TVD(p, q), KL(q || p) per row of p [B, N] (q [N] or [B, N])."""
    p2 = p.reshape(-1, p.shape[-1]).contiguous()
    B, N = p2.shape
    out = torch.empty(B, 3, dtype=torch.float64, device=p.device)
    ws = workspace(abi.pcv_dist_stats_workspace(B), p.device)
    qb = 0
    if q is not None:
        q = q.contiguous()
        qb = 1 if q.dim() == 2 else 0
    abi.pcv_dist_stats(p2, q, N, B, qb, out, ws, ws.numel(), _stream(p.device))
    return out


class MeshDistribution(torch.autograd.Function):
    """phases [B, m(m-1)] -> probabilities [B, C(m+n-1, n)] of every output."""

    @staticmethod
    def forward(ctx, phases, m, input_occ):
        U = mesh_unitary(phases, m)
        prob, amp = distribution_batched(U, input_occ)
        ctx.save_for_backward(phases, U, amp)
        ctx.input_occ = np.asarray(input_occ, dtype=np.uint8)
        return prob

    @staticmethod
    def backward(ctx, gprob):
        phases, U, amp = ctx.saved_tensors
        gprob = gprob.contiguous()
        gamp = torch.empty_like(amp)
        abi.pcv_prob_grad_to_amp(gprob, amp, amp.numel(), gamp, _stream(amp.device))
        gU = distribution_backward(U, ctx.input_occ, gamp)
        return mesh_backward(phases, U, gU), None, None


class MeshKL(torch.autograd.Function):
    """phases [B, m(m-1)], target q [N] -> KL(q || p_b) [B], p_b the mesh's
    output distribution (Sec. 4.4's circuit-learning loss, here KL)."""

    @staticmethod
    def forward(ctx, phases, m, input_occ, q):
        U = mesh_unitary(phases, m)
        prob, amp = distribution_batched(U, input_occ)
        kl = dist_stats(prob, q)[:, 2].clone()
        ctx.save_for_backward(phases, U, amp, prob, q)
        ctx.input_occ = np.asarray(input_occ, dtype=np.uint8)
        return kl

    @staticmethod
    def backward(ctx, gkl):
        phases, U, amp, prob, q = ctx.saved_tensors
        B, N = prob.shape
        gamp = torch.empty_like(amp)
        abi.pcv_kl_grad(prob, q.contiguous(), amp, N, B, 1 if q.dim() == 2 else 0, gkl.contiguous(), 1.0, gamp,
                        _stream(amp.device))
        gU = distribution_backward(U, ctx.input_occ, gamp)
        return mesh_backward(phases, U, gU), None, None, None


def mesh_distribution(phases, m, input_occ):
    return MeshDistribution.apply(phases, m, input_occ)


def mesh_kl(phases, m, input_occ, q):
    return MeshKL.apply(phases, m, input_occ, q)
