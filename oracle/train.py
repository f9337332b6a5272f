"""The training objective of one step, FP64 (Sec. 6.1 Eq. 7; Supp. C).

For each system b of a batch: probes Z_b from the SplitMix64 stream keyed by
(step_seed, b) -- Rademacher (the benchmark configuration) or, with
probes="gaussian", Gaussian draws smoothed by two damped-Jacobi sweeps with
omega = 0.6 (Sec. 6.2 Eq. 8; Supp. C) -- the fixed operand W_b = A_b Z_b (no gradient through A), the
learned factors from the network forward, Y_b = M_b W_b by the structured apply,
and L_b = 1 - <Z_b, Y_b>_F / (||Z_b||_F ||Y_b||_F).  The batch loss is the mean
of the L_b.  Gradients with respect to the flat weight vector come from torch
autograd on this FP64 forward.
"""
from __future__ import annotations

import numpy as np
import torch

from . import grid, loss, network


def sai_scale(sys):
    """||A|| of the SAI loss: the Gershgorin bound 2 max_i A_ii, which bounds lambda_max(A) from
    above for these diagonally dominant operators (the off-diagonal magnitudes of a row sum to at
    most A_ii) and meets it up to a few per cent where the coefficient is locally constant."""
    return 2.0 * float(np.max(sys["diag"]))


def batch_loss(blob, layout, cfg, systems, step_seed, n_probes, geoms=None, grad=True, probes="rademacher",
               omega=0.6, smooth_steps=2, loss_kind="cosine", highway=True):
    """Mean loss of a batch and (optionally) its gradient w.r.t. the weights.

    loss_kind "cosine" is Eq. 7; "sai" is the SAI ablation of Sec. 6.1 on the same operand,
    || Y / ||A|| - Z ||_F^2 / ||Z||_F^2 with Y = M A Z.  The paper writes A M Z; for symmetric A
    and M both orders have the same probe expectation ||M A / ||A|| - I||_F^2 (the two matrices
    are transposes of each other), and the division by ||Z||_F^2 makes the value a mean per
    probe entry.  ``highway=False`` runs the network with its highway channels held at zero
    (the ablation of Sec. 7.3)."""
    flat = torch.as_tensor(np.asarray(blob, dtype=np.float64)).clone().requires_grad_(grad)
    p = {}
    off = 0
    for name, shape in layout:
        k = int(np.prod(shape))
        p[name] = flat[off:off + k].reshape(shape)
        off += k
    total = 0.0
    losses = []
    for b, sys in enumerate(systems):
        a = grid.sparse_matrix(sys)
        if probes == "gaussian":
            z = loss.smoothed_gaussian_probes(step_seed, b, sys["n"], n_probes, lambda v: a @ v, sys["diag"],
                                              omega, smooth_steps)
        else:
            z = loss.rademacher_probes(step_seed, b, sys["n"], n_probes)
        w = torch.as_tensor(a @ z)
        geom = geoms[b] if geoms is not None else None
        f = network.forward(p, sys, cfg, geom=geom, highway=highway)
        y = network.apply_torch(f, w)
        zt = torch.as_tensor(z)
        if loss_kind == "sai":
            c = sai_scale(sys)
            lb = ((y / c - zt) ** 2).sum() / (zt * zt).sum()
        else:
            lb = 1.0 - (zt * y).sum() / (zt.norm() * y.norm())
        losses.append(float(lb))
        total = total + lb
    total = total / len(systems)
    g = None
    if grad:
        (g,) = torch.autograd.grad(total, flat)
        g = g.numpy()
    return float(total), g, losses
