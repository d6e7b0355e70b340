"""``torch.autograd`` interface of the contact manifold.

``contacts(batch, pose_a, pose_b, twist_a, twist_b)`` returns the group
outputs y [G, 8] of ``ccm_contacts`` and is differentiable with respect to the
twists (w_X, v_X) of the two bodies of every pair, in the chart
R_X <- Exp([w_X]x) R_X, t_X <- t_X + v_X.  The twists must be zero: they are a
local chart at the given poses.  The backward pass is the hand-written adjoint
kernel (``ccm_contacts_backward_saved``, given the record the forward kept
with ``ccm_contacts_save``); its own backward -- double backward -- calls the
same kernel with a direction and returns the Hessian-vector product and the
output tangents, so ``torch.autograd.grad(..., create_graph=True)`` followed
by a second ``grad`` gives H u.
"""
from __future__ import annotations

import torch

from .api import Batch


class _ContactsGrad(torch.autograd.Function):
    """grad(ybar) = d<ybar, y>/d(twist) at the current poses."""

    @staticmethod
    def forward(ctx, ybar, twist_a, twist_b, batch, pose_a, pose_b, params, saved):
        grad, _, _ = batch.backward(pose_a, pose_b, ybar, None, params, saved=saved)
        ctx.batch, ctx.params = batch, params
        ctx.save_for_backward(ybar, pose_a, pose_b, saved)
        return grad

    @staticmethod
    def backward(ctx, gbar):
        ybar, pose_a, pose_b, saved = ctx.saved_tensors
        u = gbar.contiguous()
        _, hvp, jvp = ctx.batch.backward(pose_a, pose_b, ybar, u, ctx.params, want_jvp=True,
                                         saved=saved)
        # d<gbar, grad>/d ybar = J gbar ;  d<gbar, grad>/d twist = H gbar
        return jvp, hvp[:, :6], hvp[:, 6:], None, None, None, None, None


class _Contacts(torch.autograd.Function):
    @staticmethod
    def forward(ctx, twist_a, twist_b, batch, pose_a, pose_b, params):
        saved = batch.saved_buffer(pose_a.device)
        y = batch.contacts(pose_a, pose_b, params, saved=saved)
        ctx.batch, ctx.params = batch, params
        ctx.save_for_backward(twist_a, twist_b, pose_a, pose_b, saved)
        return y

    @staticmethod
    def backward(ctx, ybar):
        twist_a, twist_b, pose_a, pose_b, saved = ctx.saved_tensors
        g = _ContactsGrad.apply(ybar.contiguous(), twist_a, twist_b, ctx.batch, pose_a, pose_b,
                                ctx.params, saved)
        return g[:, :6], g[:, 6:], None, None, None, None


def contacts(batch: Batch, pose_a, pose_b, twist_a=None, twist_b=None, params=None):
    """Differentiable group outputs [G, 8] (d, a, p, n); see module docstring."""
    n = batch.n_pairs
    if twist_a is None:
        twist_a = torch.zeros((n, 6), device=pose_a.device, dtype=torch.float32)
    if twist_b is None:
        twist_b = torch.zeros((n, 6), device=pose_a.device, dtype=torch.float32)
    return _Contacts.apply(twist_a, twist_b, batch, pose_a, pose_b, params)
