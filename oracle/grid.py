"""Morton ordering and multiphase Poisson assembly, FP64 (Supp. D; Sec. 7.1).

Readings (the paper is silent or ambiguous; each is stated once here):

* Morton code (Supp. D "Grid and ordering"): bits are interleaved from the
  least significant end, x first (x0 y0 [z0] x1 y1 ...).  When an axis runs out
  of bits the remaining axes keep interleaving, so a 32x16x16 grid puts x4 on
  top.  All extents are powers of two, so the codes are exactly 0..N-1 and the
  Morton code of a cell is its solver index.
* Face conductance: w_ij = 2 / (rho_i + rho_j), the harmonic mean of 1/rho, the
  pressure-Poisson coefficient.  The paper prints the harmonic mean of rho,
  2 rho_i rho_j / (rho_i + rho_j) (Sec. 7.1, Supp. D); it is kept behind
  ``face="rho"``.
* Boundary: Dirichlet through a ghost cell at distance h with p = 0 and the same
  density, so a boundary face adds 1 / rho_i to the diagonal (``bc="dirichlet"``);
  ``bc="neumann"`` adds nothing (Supp. D's zero-flux form).
* diag(A)_i = sum of the cell's face weights, accumulated in the fixed order
  -x, +x, -y, +y, -z, +z with boundary faces in their slot.
"""
from __future__ import annotations

import numpy as np


def morton_bit_order(dims):
    """List of (axis, bit) from the least significant code bit upward."""
    nbits = []
    for n in dims:
        b = int(n).bit_length() - 1
        assert 1 << b == n, "extents must be powers of two"
        nbits.append(b)
    order = []
    level = 0
    while any(level < nb for nb in nbits):
        for ax, nb in enumerate(nbits):
            if level < nb:
                order.append((ax, level))
        level += 1
    return order


def morton_encode(coords, dims):
    """Morton code of one cell (tuple of integer coordinates)."""
    code = 0
    for pos, (ax, bit) in enumerate(morton_bit_order(dims)):
        code |= ((coords[ax] >> bit) & 1) << pos
    return code


def morton_decode(code, dims):
    c = [0] * len(dims)
    for pos, (ax, bit) in enumerate(morton_bit_order(dims)):
        c[ax] |= ((code >> pos) & 1) << bit
    return tuple(c)


def lex_index(coords, dims):
    idx = 0
    stride = 1
    for ax, n in enumerate(dims):
        idx += coords[ax] * stride
        stride *= n
    return idx


def morton_perm(dims):
    """perm[m] = lexicographic index of the cell with Morton code m."""
    n = int(np.prod(dims))
    perm = np.empty(n, dtype=np.int64)
    for m in range(n):
        perm[m] = lex_index(morton_decode(m, dims), dims)
    return perm


def assemble(rho_lex, dims, bc="dirichlet", face="inv_rho"):
    """Assemble the 5/7-point operator in Morton order.

    Returns dict with float64 arrays ``diag[N]`` and ``wplus[D][N]`` where
    wplus[a][i] is the conductance of the +a face of cell i (0 on the boundary),
    plus ``perm`` (Morton -> lexicographic) and ``rho`` in Morton order.
    A_ii = diag[i], A_ij = -w_ij for face neighbours (Sec. 7.1).
    """
    dims = tuple(int(d) for d in dims)
    ndim = len(dims)
    n = int(np.prod(dims))
    perm = morton_perm(dims)
    rho = np.asarray(rho_lex, dtype=np.float64)[perm]
    # Morton index of each lexicographic cell
    lex_to_m = np.empty(n, dtype=np.int64)
    lex_to_m[perm] = np.arange(n)

    def weight(ri, rj):
        if face == "inv_rho":
            return 2.0 / (ri + rj)
        return 2.0 * ri * rj / (ri + rj)

    diag = np.zeros(n)
    wplus = np.zeros((ndim, n))
    for m in range(n):
        c = morton_decode(m, dims)
        acc = 0.0
        for ax in range(ndim):
            for step in (-1, +1):
                cn = list(c)
                cn[ax] += step
                if 0 <= cn[ax] < dims[ax]:
                    j = lex_to_m[lex_index(cn, dims)]
                    w = weight(rho[m], rho[j])
                    if step > 0:
                        wplus[ax][m] = w
                elif bc == "dirichlet":
                    w = 1.0 / rho[m]
                else:
                    w = 0.0
                acc = acc + w
        diag[m] = acc
    return dict(dims=dims, n=n, diag=diag, wplus=wplus, perm=perm, rho=rho)


def neighbours(dims):
    """nbr[i][2a + s] = Morton index of the -a (s=0) / +a (s=1) neighbour or -1."""
    n = int(np.prod(dims))
    ndim = len(dims)
    nbr = -np.ones((n, 2 * ndim), dtype=np.int64)
    for m in range(n):
        c = morton_decode(m, dims)
        for ax in range(ndim):
            for s, step in enumerate((-1, +1)):
                cn = list(c)
                cn[ax] += step
                if 0 <= cn[ax] < dims[ax]:
                    nbr[m][2 * ax + s] = morton_encode(tuple(cn), dims)
    return nbr


def dense_matrix(sys):
    """Dense A (N x N, float64) from an assembled system."""
    n = sys["n"]
    dims = sys["dims"]
    nbr = neighbours(dims)
    a = np.zeros((n, n))
    for i in range(n):
        a[i, i] = sys["diag"][i]
        for ax in range(len(dims)):
            j = nbr[i][2 * ax + 1]
            if j >= 0:
                w = sys["wplus"][ax][i]
                a[i, j] = -w
                a[j, i] = -w
    return a


def spmv(sys, x):
    """y = A x with the stencil written out face by face (float64)."""
    dims = sys["dims"]
    nbr = neighbours(dims) if "nbr" not in sys else sys["nbr"]
    y = sys["diag"] * x
    for ax in range(len(dims)):
        for i in range(sys["n"]):
            j = nbr[i][2 * ax + 1]
            if j >= 0:
                w = sys["wplus"][ax][i]
                y[i] -= w * x[j]
                y[j] -= w * x[i]
    return y


def sparse_matrix(sys):
    """scipy CSR form of A (for larger oracle solves)."""
    import scipy.sparse as sp
    n = sys["n"]
    nbr = neighbours(sys["dims"]) if "nbr" not in sys else sys["nbr"]
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [sys["diag"]]
    for ax in range(len(sys["dims"])):
        j = nbr[:, 2 * ax + 1]
        i = np.nonzero(j >= 0)[0]
        w = sys["wplus"][ax][i]
        rows += [i, j[i]]
        cols += [j[i], i]
        vals += [-w, -w]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))
