"""torch.autograd.Function wrappers of P2M and M2P (positions and values differentiable).

The backward passes call the hand-written adjoint kernels through the C ABI.  P2M offers two
modes: "recompute" rebuilds the shape functions in the backward pass; "checkpoint" stores the
explicit per-node weights in the forward pass and uses them for the value gradient (the
position gradient always recomputes the geometry).  Topology (Delaunay triangles, stencils)
is held fixed, i.e. these are the derivatives of the piecewise-smooth maps between topology
changes.
"""
from __future__ import annotations

import torch

from . import api as A


class ProjectP2M(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, pos, n, shape, solve, checkpoint, nb):
        N, C = vals.shape
        proj = A.Projector(n, N, C=C, nb=nb, pos_dtype=pos.dtype, device=vals.device)
        proj.build(pos.detach().contiguous())
        v = vals.detach().contiguous()
        weights = None
        if checkpoint:
            weights = proj.shape_weights(shape=shape, solve=solve, K=32, w_dtype=vals.dtype)
            mesh = proj.p2m(v, weights=weights)
        else:
            mesh = proj.p2m(v, shape=shape, solve=solve)
        ctx.proj, ctx.weights, ctx.shape, ctx.solve = proj, weights, shape, solve
        ctx.save_for_backward(v)
        return mesh

    @staticmethod
    def backward(ctx, grad_mesh):
        (v,) = ctx.saved_tensors
        want_pos = ctx.needs_input_grad[1]
        gv, gp = ctx.proj.backward(v, grad_mesh.contiguous(), shape=ctx.shape, solve=ctx.solve,
                                   weights=ctx.weights, want_pos=want_pos)
        return gv, gp, None, None, None, None, None


class InterpM2P(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, pos, n, nb):
        N = pos.shape[0]
        proj = A.Projector(n, N, C=mesh.shape[-1], nb=nb, pos_dtype=pos.dtype, device=mesh.device)
        p = pos.detach().contiguous()
        proj.build(p)
        m = mesh.detach().contiguous()
        out = proj.m2p(p, m)
        ctx.proj = proj
        ctx.save_for_backward(m, p)
        return out

    @staticmethod
    def backward(ctx, grad_vals):
        m, p = ctx.saved_tensors
        gm, gp = ctx.proj.m2p_backward(p, m, grad_vals.contiguous(),
                                       want_pos=ctx.needs_input_grad[1])
        return gm, gp, None, None


def p2m(vals, pos, n, shape=A.PFEM_SHAPE_QUADRATIC, solve=None, checkpoint=False, nb=None):
    """Differentiable P2M: mesh [n,n,C] from particle values [N,C] at positions [N,2]."""
    if solve is None:
        solve = A.PFEM_SOLVE_F64 if vals.dtype == torch.float64 else A.PFEM_SOLVE_F32
    return ProjectP2M.apply(vals, pos, n, shape, solve, checkpoint, nb)


def m2p(mesh, pos, n, nb=None):
    """Differentiable M2P: particle values [N,C] from mesh [n,n,C] at positions [N,2]."""
    return InterpM2P.apply(mesh, pos, n, nb)
