"""torch.autograd wrapper of the navigator step.

GeoDist.apply(vol, p, d, trans, params, mode) returns the step of every track
(p, d: (3, n) float64 CUDA tensors, SoA rows x, y, z); its backward runs the
adjoint kernel of the library (geo_dist_to_boundary_adjoint) and returns
gradients for p, d and for the geometry tensors trans (nd, 3) and params
(nd + 1, 5) (daughters' shape parameters, the mother's last).  The geometry
tensors only carry gradients: the volume `vol` must have been built from the
same values.
"""
from __future__ import annotations

import torch

from . import geonav


class GeoDist(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vol, p, d, trans, params, mode=geonav.GEO_FP32_REFINE):
        p = p.contiguous()
        d = d.contiguous()
        step, hit = geonav.geo_dist_to_boundary(vol, p[0], p[1], p[2], d[0], d[1], d[2], mode=mode)
        ctx.vol = vol
        ctx.save_for_backward(p, d, hit)
        ctx.mark_non_differentiable(hit)
        return step, hit

    @staticmethod
    def backward(ctx, grad_step, grad_hit):
        p, d, hit = ctx.saved_tensors
        need_geo = ctx.needs_input_grad[3] or ctx.needs_input_grad[4]
        out = geonav.geo_dist_to_boundary_adjoint(ctx.vol, p[0], p[1], p[2], d[0], d[1], d[2], hit,
                                                  grad_step.contiguous(), want_geometry=need_geo)
        gp, gd = out[0], out[1]
        gt = out[2] if need_geo else None
        gprm = out[3] if need_geo else None
        return None, gp, gd, gt, gprm, None


def dist_to_boundary(vol, p, d, trans=None, params=None, mode=geonav.GEO_FP32_REFINE):
    """Differentiable step; returns (step, hit)."""
    nd = vol.n_daughters
    dev = p.device
    if trans is None:
        trans = torch.zeros((nd, 3), dtype=torch.float64, device=dev)
    if params is None:
        params = torch.zeros((nd + 1, 5), dtype=torch.float64, device=dev)
    return GeoDist.apply(vol, p, d, trans, params, mode)
