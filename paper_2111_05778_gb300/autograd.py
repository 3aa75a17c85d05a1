"""torch.autograd binding of the implicit-surface adjoint.

``polygonize_mlp(params, ...)`` returns the deduplicated mesh vertices of the
neural SDB with parameters ``params`` (a float32 tensor packed like the MLP
blob) and its faces; gradients of any loss on the vertices flow back to
``params`` through gh_backward: for a vertex on the level set f = 0,
dv/dtheta = -grad_x f (df/dtheta) / |grad_x f|^2.
"""
from __future__ import annotations

import torch

from . import gh


class _ImplicitPolygonize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, width, n_mid, N, lo, hi, r0, alpha, beta, lam, precision):
        sdb = gh.MlpSdb(params.detach().cpu().numpy(), width, n_mid, r0, alpha, beta, lam)
        eps = sdb.calibrate(N, lo, hi) if precision == "bf16" else None
        mesh = gh.polygonize(sdb, N, lo=lo, hi=hi, precision=precision, eps=eps, indexed=True)
        verts, faces = mesh.verts, mesh.faces.long()
        ctx.sdb = sdb
        ctx.save_for_backward(verts)
        ctx.mark_non_differentiable(faces)
        return verts, faces

    @staticmethod
    def backward(ctx, dverts, dfaces):
        (verts,) = ctx.saved_tensors
        grad = gh.backward(ctx.sdb, verts, dverts)
        return (grad.to(dverts.device),) + (None,) * 10


class _ImplicitPolygonizeCsg(torch.autograd.Function):
    @staticmethod
    def forward(ctx, prims, N, lo, hi):
        sdb = gh.CsgSdb(prims.detach().cpu().double().numpy())
        mesh = gh.polygonize(sdb, N, lo=lo, hi=hi, indexed=True)
        verts, faces = mesh.verts, mesh.faces.long()
        ctx.sdb = sdb
        ctx.shape = prims.shape
        ctx.dtype = prims.dtype
        ctx.save_for_backward(verts)
        ctx.mark_non_differentiable(faces)
        return verts, faces

    @staticmethod
    def backward(ctx, dverts, dfaces):
        (verts,) = ctx.saved_tensors
        g = gh.backward(ctx.sdb, verts, dverts)  # [n, 20] like the device records
        out = torch.zeros(ctx.shape, dtype=ctx.dtype, device=dverts.device)
        out[:, 2:8] = g[:, 2:8].to(ctx.dtype)  # centre and size parameters
        return out, None, None, None


def polygonize_csg(prims, N=128, lo=-1.0, hi=1.0):
    """(verts [V,3], faces [T,3]) of an analytic scene given as primitive rows
    [n,17] (type, op, centre, params, rotation); differentiable in the centres
    and size parameters."""
    return _ImplicitPolygonizeCsg.apply(prims, N, lo, hi)


def polygonize_mlp(params, width, n_mid=5, N=256, lo=-1.0, hi=1.0, r0=0.6, alpha=0.1, beta=1.1, lam=1.0,
                   precision="fp32"):
    """(verts [V,3], faces [T,3]) of the neural SDB; differentiable in params."""
    return _ImplicitPolygonize.apply(params, width, n_mid, N, lo, hi, r0, alpha, beta, lam, precision)
