"""The node bound as a differentiable PyTorch op (Sec. 3.1).

``NodeBound.apply(alpha, beta, gamma, context, nodes)`` returns the lower bound
of each BaB node at the given parameters: the back-substitution sweep of the
objective row with slopes alpha, split multipliers beta and multi-neuron
multipliers gamma, concretised over the input box.  Its backward is the
library's adjoint back-substitution (the relaxed network evaluated forward at
the minimiser x*), which returns d lb / d (alpha, beta, gamma) exactly; the
bound is piecewise linear in each parameter, with D-case switches treated as
fixed, as in projected gradient ascent.

Every number is computed by the library's kernels; this module only moves the
parameters and results between torch tensors and the C ABI.  A bound is sound
only for 0 <= alpha <= 1 and beta, gamma >= 0: callers that step the
parameters project them (the library's own optimiser does).
"""
from __future__ import annotations

import numpy as np
import torch

__all__ = ["NodeBound", "node_bound"]


class NodeBound(torch.autograd.Function):
    """lb = NodeBound.apply(alpha [n, SD], beta [n, SD], gamma [n, E], context, nodes).

    The nodes (ids of one network and one property, so that they share E) take
    the given parameters and keep them; their bounds l, u and splits are used
    as they are (re-bound split nodes first, e.g. with ``Context.bound_batch``).
    Tensors may live on any device; lb comes back on alpha's device.
    """

    @staticmethod
    def forward(fctx, alpha, beta, gamma, context, nodes):
        n = len(nodes)
        SD = alpha.shape[1]
        E = gamma.shape[1] if gamma is not None and gamma.numel() else 0
        flat = torch.cat([alpha.detach().float().reshape(n, SD), beta.detach().float().reshape(n, SD)]
                         + ([gamma.detach().float().reshape(n, E)] if E else []), dim=1)
        context.set_params(nodes, flat.cpu().numpy())
        lb, ga, gb, gg = context.bound_grad(nodes, SD, E)
        dev = alpha.device
        fctx.save_for_backward(torch.from_numpy(np.ascontiguousarray(ga)).to(dev),
                               torch.from_numpy(np.ascontiguousarray(gb)).to(dev),
                               torch.from_numpy(np.ascontiguousarray(gg)).to(dev))
        fctx.has_gamma = gamma is not None
        return torch.from_numpy(lb).to(dev)

    @staticmethod
    def backward(fctx, grad_lb):
        ga, gb, gg = fctx.saved_tensors
        w = grad_lb.reshape(-1, 1).to(ga.dtype)
        g_gamma = w * gg if fctx.has_gamma else None
        return w * ga, w * gb, g_gamma, None, None


def node_bound(context, nodes, alpha, beta, gamma=None):
    """Convenience wrapper: NodeBound with an empty gamma when the property has
    no multi-neuron constraints."""
    if gamma is None:
        gamma = torch.zeros(len(nodes), 0, device=alpha.device)
    return NodeBound.apply(alpha, beta, gamma, context, nodes)
