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


def batch_loss(blob, layout, cfg, systems, step_seed, n_probes, geoms=None, grad=True, probes="rademacher",
               omega=0.6, smooth_steps=2):
    """Mean cosine loss of a batch and (optionally) its gradient w.r.t. the weights."""
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
        f = network.forward(p, sys, cfg, geom=geom)
        y = network.apply_torch(f, w)
        zt = torch.as_tensor(z)
        lb = 1.0 - (zt * y).sum() / (zt.norm() * y.norm())
        losses.append(float(lb))
        total = total + lb
    total = total / len(systems)
    g = None
    if grad:
        (g,) = torch.autograd.grad(total, flat)
        g = g.numpy()
    return float(total), g, losses
