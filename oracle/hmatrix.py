"""Weak-admissibility H-matrix preconditioner, FP64 (Sec. 4, Sec. 5, Supp. B).

Partition (Sec. 4 "Notation"; Supp. B "Apply-path tensor layout"; eta = 1):
K = N / L leaves of L contiguous indices.  Level l = 1 .. log2 K splits the
cluster tree: tile t of level l (S = K / 2^l leaves per side) has row leaves
R = [2tS, (2t+1)S) and column leaves C = [(2t+1)S, (2t+2)S).  The lower block
(C, R) reuses the tile through its transpose, so there are M_H = K - 1 unique
tiles.  Tiles are numbered in heap order m = 2^(l-1) - 1 + t.

Packed layouts (one flat vector each):

* learned (Sec. 4.4, P = K L^2 + M_H L_s^2 + 2 N L_s + N):
  [F_k (K x L x L, row-major)] [B_m (M_H x L_s x L_s)] [U~ (N x L_s)]
  [V~ (N x L_s)] [g (N)], where row i of U~ / V~ is node i's bridge row and
  g_i = lambda_i / diag(A)_i is the Jacobi-gate coefficient (the gate term
  diag(lambda) diag(A)^-1 of Sec. 4.4 with the division folded in).
  M_kk = F_k F_k^T + diag(g_k);  M[R_m, C_m] = U~_{R_m} B_m V~_{C_m}^T.
* svdh (the plain method): [G_k (K x L x L)] [Sigma_m (M_H x r x r, diagonal
  stored dense)] [W (levels x N x r)], where W[l] row i is row i of U_r (if
  leaf(i) lies in the row cluster of its level-l tile) or of V_r (column cluster).
  M_kk = G_k;  M[R_m, C_m] = U_r Sigma_r V_r^T.

Both layouts are applied by the same four-stage chain of Sec. 5 (restriction,
strip aggregation, coupling, prolongation); in the learned layout the bridge of
leaf k is U~_k when k is in a tile's row cluster and V~_k in its column cluster,
at every level; in the svdh layout the bridge is W[l] at level l.
"""
from __future__ import annotations

import math
import numpy as np


# ----------------------------------------------------------------- partition
def partition(n, leaf):
    """List of tiles (m, level, R=(r0, r1), C=(c0, c1)) in leaf units, heap order."""
    assert n % leaf == 0
    k = n // leaf
    levels = int(round(math.log2(k)))
    assert 1 << levels == k, "K must be a power of two"
    tiles = []
    for lev in range(1, levels + 1):
        s = k >> lev
        for t in range(1 << (lev - 1)):
            m = (1 << (lev - 1)) - 1 + t
            tiles.append((m, lev, (2 * t * s, (2 * t + 1) * s),
                          ((2 * t + 1) * s, (2 * t + 2) * s)))
    return tiles


def packed_width(n, leaf, rank, layout="learned"):
    """Number of elements of the packed factor vector (Sec. 4.4, Supp. B)."""
    k = n // leaf
    mh = k - 1
    if layout == "learned":
        return k * leaf * leaf + mh * rank * rank + 2 * n * rank + n
    levels = int(round(math.log2(k)))
    return k * leaf * leaf + mh * rank * rank + levels * n * rank


def offsets(n, leaf, rank, layout="learned"):
    k = n // leaf
    mh = k - 1
    o = {"leaf": 0, "core": k * leaf * leaf}
    o["bridge"] = o["core"] + mh * rank * rank
    if layout == "learned":
        o["U"] = o["bridge"]
        o["V"] = o["U"] + n * rank
        o["g"] = o["V"] + n * rank
    return o


# ----------------------------------------------------------------- unpacking
def unpack(packed, n, leaf, rank, layout):
    """Split a packed vector into named float64 arrays."""
    k = n // leaf
    mh = k - 1
    p = np.asarray(packed, dtype=np.float64)
    o = offsets(n, leaf, rank, layout)
    f = dict(layout=layout, n=n, leaf=leaf, rank=rank, K=k)
    f["leafblk"] = p[o["leaf"]:o["core"]].reshape(k, leaf, leaf)
    f["core"] = p[o["core"]:o["bridge"]].reshape(mh, rank, rank)
    if layout == "learned":
        f["U"] = p[o["U"]:o["V"]].reshape(n, rank)
        f["V"] = p[o["V"]:o["g"]].reshape(n, rank)
        f["g"] = p[o["g"]:o["g"] + n]
    else:
        levels = int(round(math.log2(k)))
        f["W"] = p[o["bridge"]:].reshape(levels, n, rank)
    return f


def pack(f):
    parts = [f["leafblk"].ravel(), f["core"].ravel()]
    if f["layout"] == "learned":
        parts += [f["U"].ravel(), f["V"].ravel(), f["g"].ravel()]
    else:
        parts += [f["W"].ravel()]
    return np.concatenate(parts)


def bridge(f, lev, k, side):
    """L x r bridge of leaf k at level ``lev``; side 0 = row cluster, 1 = column."""
    leaf = f["leaf"]
    rows = slice(k * leaf, (k + 1) * leaf)
    if f["layout"] == "learned":
        return (f["U"] if side == 0 else f["V"])[rows]
    return f["W"][lev - 1][rows]


# ----------------------------------------------------------------- dense M
def dense_m(f):
    """Assemble M densely from its factors (test use only: M is never formed
    on the apply path, Sec. 5)."""
    n, leaf, k = f["n"], f["leaf"], f["K"]
    m = np.zeros((n, n))
    for b in range(k):
        s = slice(b * leaf, (b + 1) * leaf)
        blk = f["leafblk"][b]
        if f["layout"] == "learned":
            m[s, s] = blk @ blk.T + np.diag(f["g"][s])
        else:
            m[s, s] = blk
    for (t, lev, (r0, r1), (c0, c1)) in partition(n, leaf):
        ur = np.vstack([bridge(f, lev, kk, 0) for kk in range(r0, r1)])
        vc = np.vstack([bridge(f, lev, kk, 1) for kk in range(c0, c1)])
        blk = ur @ f["core"][t] @ vc.T
        m[r0 * leaf:r1 * leaf, c0 * leaf:c1 * leaf] = blk
        m[c0 * leaf:c1 * leaf, r0 * leaf:r1 * leaf] = blk.T
    return m


# ----------------------------------------------------------------- structured apply
def apply(f, r):
    """z = M r by the stages of Sec. 5, without forming M.

    (i) diagonal stage: z_k = F_k (F_k^T r_k) + g_k * r_k (learned) or G_k r_k;
    (ii) off-diagonal chain: restriction u^_k = U~_k^T r_k, v^_k = V~_k^T r_k;
    strip aggregation s^r_m = sum_{k in R_m} u^_k, s^c_m = sum_{k in C_m} v^_k;
    coupling t^c_m = B_m^T s^r_m, t^r_m = B_m s^c_m; prolongation
    dz_k = U~_k sum_{m: k in R_m} t^r_m + V~_k sum_{m: k in C_m} t^c_m.
    ``r`` may be a vector (N) or a matrix (N x nrhs).
    """
    r = np.asarray(r, dtype=np.float64)
    vec = r.ndim == 1
    if vec:
        r = r[:, None]
    n, leaf, k = f["n"], f["leaf"], f["K"]
    z = np.zeros_like(r)
    # (i) diagonal stage
    for b in range(k):
        s = slice(b * leaf, (b + 1) * leaf)
        blk = f["leafblk"][b]
        if f["layout"] == "learned":
            z[s] = blk @ (blk.T @ r[s]) + f["g"][s][:, None] * r[s]
        else:
            z[s] = blk @ r[s]
    # (ii) off-diagonal chain, tile by tile
    tiles = partition(n, leaf)
    t_row = {}
    t_col = {}
    for (m, lev, (r0, r1), (c0, c1)) in tiles:
        s_r = sum(bridge(f, lev, kk, 0).T @ r[kk * leaf:(kk + 1) * leaf] for kk in range(r0, r1))
        s_c = sum(bridge(f, lev, kk, 1).T @ r[kk * leaf:(kk + 1) * leaf] for kk in range(c0, c1))
        t_col[m] = f["core"][m].T @ s_r
        t_row[m] = f["core"][m] @ s_c
    for (m, lev, (r0, r1), (c0, c1)) in tiles:
        for kk in range(r0, r1):
            z[kk * leaf:(kk + 1) * leaf] += bridge(f, lev, kk, 0) @ t_row[m]
        for kk in range(c0, c1):
            z[kk * leaf:(kk + 1) * leaf] += bridge(f, lev, kk, 1) @ t_col[m]
    return z[:, 0] if vec else z


# ----------------------------------------------------------------- SVD-H (plain method)
def pseudo_inverse(a_dense, rel_tol=1e-12):
    """Moore-Penrose pseudo-inverse of a symmetric positive semi-definite matrix from its
    eigendecomposition (LAPACK syevd): eigenvalues at or below rel_tol * lambda_max count as
    the null space.  With zero-flux boundaries A 1 = 0 (Supp. D, "Operator assembly"), so A
    has no inverse; A^+ is the inverse on the complement of the constants, where CG works for
    a consistent right-hand side."""
    w, v = np.linalg.eigh(a_dense)
    keep = w > rel_tol * w.max()
    p = (v[:, keep] / w[keep]) @ v[:, keep].T
    return 0.5 * (p + p.T)


def svdh_factors(a_dense, leaf, rank, leaves="block_inverse", inverse="cholesky"):
    """The plain H-matrix preconditioner built from the exact inverse.

    Leaves: ``"block_inverse"`` stores (A_kk)^-1, the exact inverse of A's
    diagonal block; ``"inverse_block"`` stores (A^-1)_kk.  Tiles: the rank-r
    truncated SVD X_r = U_r Sigma_r V_r^T of the exact block X = A^-1[R, C]
    (LAPACK gesdd), with r = min(rank, S L).  A^-1 comes from a Cholesky
    factorisation (LAPACK potrf/potrs), or, with ``inverse="pseudo"`` for a singular
    zero-flux operator, is the pseudo-inverse A^+ (``pseudo_inverse``).
    """
    import scipy.linalg as sl
    n = a_dense.shape[0]
    k = n // leaf
    levels = int(round(math.log2(k)))
    if inverse == "pseudo":
        ainv = pseudo_inverse(a_dense)
    else:
        cf = sl.cho_factor(a_dense, lower=True)
        ainv = sl.cho_solve(cf, np.eye(n))
        ainv = 0.5 * (ainv + ainv.T)
    f = dict(layout="svdh", n=n, leaf=leaf, rank=rank, K=k)
    f["leafblk"] = np.zeros((k, leaf, leaf))
    for b in range(k):
        s = slice(b * leaf, (b + 1) * leaf)
        if leaves == "block_inverse":
            g = np.linalg.inv(a_dense[s, s])
            f["leafblk"][b] = 0.5 * (g + g.T)
        else:
            f["leafblk"][b] = ainv[s, s]
    f["core"] = np.zeros((k - 1, rank, rank))
    f["W"] = np.zeros((levels, n, rank))
    f["sigma"] = {}
    for (m, lev, (r0, r1), (c0, c1)) in partition(n, leaf):
        x = ainv[r0 * leaf:r1 * leaf, c0 * leaf:c1 * leaf]
        u, s, vt = sl.svd(x, lapack_driver="gesdd")
        rr = min(rank, x.shape[0])
        f["core"][m][:rr, :rr] = np.diag(s[:rr])
        f["W"][lev - 1][r0 * leaf:r1 * leaf, :rr] = u[:, :rr]
        f["W"][lev - 1][c0 * leaf:c1 * leaf, :rr] = vt[:rr].T
        f["sigma"][m] = s
    f["ainv"] = ainv
    return f
