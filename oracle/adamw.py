"""AdamW with global-norm gradient clipping, FP64 (Supp. C "Optimizer and schedule").

Decoupled weight decay (p <- p - lr wd p), bias-corrected first and second
moments, beta = (0.9, 0.999), eps = 1e-8 (PyTorch defaults, as Supp. C states),
weight decay 1e-4, gradients clipped to global l2 norm 1 with the usual
max_norm / (norm + 1e-6) factor applied only when the norm exceeds max_norm.
"""
from __future__ import annotations

import numpy as np


def clip_global(g, max_norm=1.0):
    g = np.asarray(g, dtype=np.float64)
    nrm = float(np.sqrt(g @ g))
    if nrm > max_norm:
        return g * (max_norm / (nrm + 1e-6))
    return g.copy()


def adamw_step(p, g, m, v, step, lr, wd=1e-4, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW update; returns (p, m, v).  ``step`` counts from 1."""
    p = np.asarray(p, dtype=np.float64) * (1.0 - lr * wd)
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    p = p - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v
