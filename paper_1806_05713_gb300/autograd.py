"""torch.autograd.Function over the library's force map and its adjoint.

``lj_forces(q4, eps, sigma, plist, r_cut, box, precision)`` returns the
forces F (n x 4, pad column zero): the impulse of ``lj_force`` with dt = 1
and zero momenta (Algorithm 1 inside Algorithm 3, Eq. (1) with parameters
eps, sigma).  Its backward is the hand-written adjoint kernel
``lj_force_vjp``: gradients with respect to the positions and to the two
scalar tensors eps and sigma.  The pair list is a constant of the map (it
is rebuilt by the caller when positions move by more than the margin).
"""
from __future__ import annotations

import torch

from . import lj


class LJForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q4, eps, sigma, plist, r_cut, box, precision):
        e, s = float(eps), float(sigma)
        F = torch.zeros_like(q4)
        lj.lj_force(q4, F, plist, 1.0, r_cut, box, e, s, precision)
        ctx.save_for_backward(q4)
        ctx.meta = (plist, r_cut, box, e, s, precision, eps.shape, sigma.shape)
        return F

    @staticmethod
    def backward(ctx, gF):
        (q4,) = ctx.saved_tensors
        plist, r_cut, box, e, s, precision, es_shape, ss_shape = ctx.meta
        gq, ges = lj.lj_force_vjp(q4, gF.contiguous(), plist, r_cut, box, e, s, precision)
        return (gq, ges[0].reshape(es_shape), ges[1].reshape(ss_shape), None, None, None, None)


def lj_forces(q4: torch.Tensor, eps: torch.Tensor, sigma: torch.Tensor, plist: lj.PairList,
              r_cut: float, box, precision: int = lj.LJ_FP64) -> torch.Tensor:
    """Differentiable forces F(q; eps, sigma) (n x 4)."""
    return LJForces.apply(q4, eps, sigma, plist, r_cut, box, precision)
