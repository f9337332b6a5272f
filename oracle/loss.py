"""Cosine-Hutchinson probe loss and probes (Sec. 6.1 Eq. 7; Sec. 6.2 Eq. 8).

L_cos = 1 - <Z, M A Z>_F / (||Z||_F ||M A Z||_F): one global cosine over all
N * K_z entries of a system (Eq. 7).  A Z is a fixed input (no gradient flows
through A).  A batch of systems reduces by the mean of the per-system losses
(reading: the paper pads a mini-batch to a common size and does not say how it
reduces).
"""
from __future__ import annotations

import numpy as np

from . import rng


def cosine_loss(z, y):
    """1 - <Z, Y>_F / (||Z||_F ||Y||_F) for Y = M A Z (Eq. 7)."""
    z = np.asarray(z, dtype=np.float64).ravel()
    y = np.asarray(y, dtype=np.float64).ravel()
    return 1.0 - float(z @ y) / (float(np.sqrt(z @ z)) * float(np.sqrt(y @ y)))


def sai_loss(z, amz, anorm):
    """|| (1/||A||) A M Z - Z ||_F^2, the vector-distance loss of Sec. 6.1."""
    d = np.asarray(amz, dtype=np.float64) / anorm - np.asarray(z, dtype=np.float64)
    return float(np.sum(d * d))


def projector_distance(u, v):
    """1/2 || Pi_u - Pi_v ||_F^2 for the rank-one projectors onto the lines
    through u and v (Prop. 1, Eq. 7's subspace reading), formed explicitly."""
    u = np.asarray(u, dtype=np.float64).ravel()
    v = np.asarray(v, dtype=np.float64).ravel()
    pu = np.outer(u, u) / (u @ u)
    pv = np.outer(v, v) / (v @ v)
    d = pu - pv
    return 0.5 * float(np.sum(d * d))


def rademacher_probes(step_seed, system, n, kz):
    """The Rademacher probes drawn from the counter-based SplitMix64 stream."""
    return np.array(rng.rademacher(step_seed, system, n, kz), dtype=np.float64)


def gaussian_probes(step_seed, system, n, kz):
    """Gaussian probes drawn from the counter-based SplitMix64 stream (Box-Muller)."""
    return np.array(rng.gaussian(step_seed, system, n, kz), dtype=np.float64)


def smoothed_gaussian_probes(step_seed, system, n, kz, matvec, diag, omega=0.6, steps=2):
    """The paper's training probes: Gaussian, then `steps` damped-Jacobi sweeps (Eq. 8)."""
    return jacobi_smooth(gaussian_probes(step_seed, system, n, kz), matvec, diag, omega, steps)


def jacobi_smooth(z, matvec, diag, omega=0.6, steps=2):
    """Damped-Jacobi low-pass on probes, z <- z - omega D^-1 A z (Eq. 8)."""
    z = np.array(z, dtype=np.float64, copy=True)
    for _ in range(steps):
        z = z - omega * (matvec(z) / diag[:, None])
    return z


def probe_count(n):
    """K_z = max(64, ceil(sqrt(N))) (Sec. 6.3, Supp. C)."""
    import math
    return max(64, int(math.ceil(math.sqrt(n))))
