"""Diagnostics of the preconditioner: the spectrum of M A (Fig. 1) and the off-diagonal rank
audit (Fig. 3).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.  Plain FP64 dense linear algebra
(LAPACK through numpy), for systems of a few thousand unknowns.
"""
from __future__ import annotations

import numpy as np

from . import hmatrix


def spectrum_ma(a, m):
    """Eigenvalues of M A, ascending, for SPD A and symmetric M (Fig. 1).

    M A = A^-1/2 (A^1/2 M A^1/2) A^1/2 is similar to the symmetric A^1/2 M A^1/2, so the
    spectrum is real; it is computed on that form with a symmetric eigensolver (syevd),
    A^1/2 from A's own eigendecomposition.
    """
    w, v = np.linalg.eigh(a)
    half = (v * np.sqrt(w)) @ v.T
    s = half @ m @ half
    return np.linalg.eigvalsh(0.5 * (s + s.T))


def condition_number(ev):
    """lambda_max / lambda_min of a positive spectrum (inf when it is not positive)."""
    lo, hi = float(np.min(ev)), float(np.max(ev))
    return hi / lo if lo > 0.0 else float("inf")


def eps_rank(sv, eps):
    """Smallest r with ||X - X_r||_F <= eps ||X||_F, X_r the rank-r truncated SVD.

    By Eckart-Young ||X - X_r||_F^2 is the sum of the squared singular values from index r
    on; ``sv`` holds them in descending order.
    """
    sq = np.asarray(sv, dtype=np.float64) ** 2
    total = sq.sum()
    if total == 0.0:
        return 0
    tail = np.concatenate([np.cumsum(sq[::-1])[::-1], [0.0]])   # tail[r] = sum_{i >= r}
    return int(np.argmax(tail <= (eps * eps) * total))


def rank_audit(ainv, leaf, rank, eps_list=(1e-3, 1e-6, 1e-9)):
    """Required vs provided off-diagonal rank by distance class (Fig. 3).

    For every tile X = A^-1[R, C] of the weak-admissibility partition, with S leaves per
    side, the required rank fraction is eps_rank(X, eps) / (S L); the provided one is
    rank / (S L).  Returns {S: dict(tiles, provided, ranks[tile][eps], mean[eps], std[eps])},
    mean and std taken over the tiles of one class.
    """
    n = ainv.shape[0]
    out = {}
    for (_, _, (r0, r1), (c0, c1)) in hmatrix.partition(n, leaf):
        s = r1 - r0
        x = ainv[r0 * leaf:r1 * leaf, c0 * leaf:c1 * leaf]
        sv = np.linalg.svd(x, compute_uv=False)
        cls = out.setdefault(s, dict(tiles=0, provided=rank / (s * leaf), ranks=[]))
        cls["tiles"] += 1
        cls["ranks"].append([eps_rank(sv, e) for e in eps_list])
    for s, cls in out.items():
        frac = np.asarray(cls["ranks"], dtype=np.float64) / (s * leaf)
        cls["mean"] = frac.mean(axis=0)
        cls["std"] = frac.std(axis=0)
    return out
