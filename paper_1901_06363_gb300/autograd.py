"""torch.autograd.Function wrappers of the differentiable trilinear score.

Forward and backward both run in the library's CUDA kernels (the trilinear
form of Eq. 1 and its hand-written adjoint); these classes only hand tensors
to the C calls.

  o = TrilinearScore.apply(xyz, docker, batch_id, pocket_id, clip)
      o per ligand from coordinates (CUDA float32, atom_off layout, Å)
  z = PoseDofs.apply(q, x, docker, batch_id)
      coordinates of the poses x moved by q = (t, omega, theta_1..theta_T)
  pose_score(docker, batch_id, pocket_id, x, q)  =  o(z(q)), differentiable in q
"""
from __future__ import annotations

import torch


class TrilinearScore(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xyz, docker, batch_id, pocket_id, clip=1):
        ctx.docker, ctx.bid, ctx.pid, ctx.clip = docker, batch_id, pocket_id, clip
        ctx.save_for_backward(xyz)
        return docker.score_trilinear(batch_id, pocket_id, xyz.detach(), clip)

    @staticmethod
    def backward(ctx, grad_o):
        (xyz,) = ctx.saved_tensors
        g = ctx.docker.score_trilinear_grad(ctx.bid, ctx.pid, xyz.detach(), grad_o.float(), ctx.clip)
        return g, None, None, None, None


class PoseDofs(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, x, docker, batch_id):
        if x.requires_grad:
            raise ValueError("PoseDofs differentiates with respect to q only")
        ctx.docker, ctx.bid = docker, batch_id
        ctx.save_for_backward(q, x)
        return docker.dof_apply(batch_id, x.detach(), q.detach())

    @staticmethod
    def backward(ctx, grad_z):
        q, x = ctx.saved_tensors
        return ctx.docker.dof_grad(ctx.bid, x, q.detach(), grad_z.float()), None, None, None


def pose_score(docker, batch_id, pocket_id, x, q, clip=1):
    """Trilinear o per ligand of the poses x moved by q; differentiable with respect to q."""
    return TrilinearScore.apply(PoseDofs.apply(q, x, docker, batch_id), docker, batch_id, pocket_id, clip)
