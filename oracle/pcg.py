"""Preconditioned conjugate gradients in FP64 (Sec. 5; Sec. 6.3; Supp. A, G).

The iteration is the textbook PCG (Saad, Iterative Methods, Alg. 9.1):

    x0 = 0, r0 = b, z0 = M r0, p0 = z0
    repeat:  q = A p;  alpha = (r.z) / (p.q);  x += alpha p;  r -= alpha q
             stop when ||r||_2 / ||r0||_2 <= rtol          (Supp. A stop test)
             z = M r;  beta = (r.z)_new / (r.z)_old;  p = z + beta p

Readings: every ``recompute_every``-th iteration the recursive residual is
replaced by the true residual b - A x (the periodic true-residual recompute; the
paper keeps only the scalars in FP64, Supp. G); the iteration count is the
number of A p products; breakdown is declared when p.q <= 0 or r.z <= 0, which
for SPD A and M cannot happen in exact arithmetic.
"""
from __future__ import annotations

import numpy as np

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, -4


def pcg(matvec, precond, b, rtol=1e-6, max_iter=None, recompute_every=10,
        keep_history=False):
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    if max_iter is None:
        max_iter = 10 * n
    x = np.zeros(n)
    r = b.copy()
    bnorm = float(np.sqrt(b @ b))
    hist = dict(res=[1.0], x=[x.copy()], r=[r.copy()], z=[])
    if bnorm == 0.0:
        return dict(x=x, iters=0, status=OK, rel_res=0.0, hist=hist)
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    if keep_history:
        hist["z"].append(z.copy())
    status = NOT_CONVERGED
    it = 0
    if rz <= 0.0:
        status = BREAKDOWN
        max_iter = 0
    while it < max_iter:
        q = matvec(p)
        it += 1
        pq = float(p @ q)
        if not pq > 0.0:
            status = BREAKDOWN
            break
        alpha = rz / pq
        x = x + alpha * p
        if recompute_every and it % recompute_every == 0:
            r = b - matvec(x)
        else:
            r = r - alpha * q
        rel = float(np.sqrt(r @ r)) / bnorm
        if keep_history:
            hist["res"].append(rel)
            hist["x"].append(x.copy())
            hist["r"].append(r.copy())
        if rel <= rtol:
            status = OK
            break
        z = precond(r)
        rz_new = float(r @ z)
        if keep_history:
            hist["z"].append(z.copy())
        if not rz_new > 0.0:
            status = BREAKDOWN
            break
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    true_rel = float(np.linalg.norm(b - matvec(x))) / bnorm
    return dict(x=x, iters=it, status=status, rel_res=true_rel, hist=hist)
