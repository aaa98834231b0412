"""Differentiable hinge clearance through the CAPT (torch.autograd.Function).

Forward: per sphere d = min(||c - p*||, r_max), exact whenever the nearest cloud point
p* is within r_max (every such point is in the leaf's affordance set, Lemma 1 case 1);
cost_t = sum over a trajectory's spheres of max(0, r + margin - d)^2.
Backward: d cost_t / d c = g_t * (-2 h) * (c - p*) / d where h > 0 and d < r_max, else 0.
Both directions run in libcapt.so (capt_clearance_fwd / capt_clearance_bwd).
"""
from __future__ import annotations

import torch


class CaptClearance(torch.autograd.Function):
    """cost = CaptClearance.apply(tree, centers [T,W,S,3], radii [S], margin) -> [T]."""

    @staticmethod
    def forward(ctx, tree, centers, radii, margin):
        from . import capt_clearance_fwd
        centers = centers.contiguous()
        radii = radii.contiguous()
        cost, dist, argmin = capt_clearance_fwd(tree, centers, radii, margin)
        ctx.tree = tree
        ctx.margin = float(margin)
        ctx.save_for_backward(centers, radii, dist, argmin)
        ctx.mark_non_differentiable(dist, argmin)
        return cost, dist, argmin

    @staticmethod
    def backward(ctx, grad_cost, grad_dist, grad_argmin):
        from . import capt_clearance_bwd
        centers, radii, dist, argmin = ctx.saved_tensors
        if grad_cost is None:
            return None, None, None, None
        g = capt_clearance_bwd(ctx.tree, centers, radii, dist, argmin, grad_cost.contiguous().float(), ctx.margin)
        return None, g, None, None
