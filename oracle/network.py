"""The hierarchical transformer that emits the learned factors, FP64 (Sec. 4; Supp. B).

Plain PyTorch CPU ops in float64; gradients (for the training parity tests)
come from torch autograd on this forward.  One system at a time.

Readings of passages the paper leaves open (each also listed in the design notes):

* Features (Sec. 4.1, Supp. B "Encoder"): 8 node features [log rho - mean,
  centred x, y, z, boundary-face fraction, log diag - mean, interior coupling
  sum / diag, interface flag] and d_glob = 12 global statistics [log2 N / 16,
  3D flag, max/min/mean/std of log rho, heavy fraction, mean/std/max/min of
  log diag, boundary-cell fraction].  Pressure does not exist before the solve.
* Encoder MLP: Linear -> GELU -> Linear.  GCN (n_gcn = 2): h <- h + GELU(W (P h) + b)
  with P = D^-1 A, i.e. (P h)_i = h_i - sum_j (w_ij / d_i) h_j.
* Off-diagonal tokens (Sec. 4.2, Supp. B): token a of tile m is
  pool([mean of h over row chunk a of R_m ; mean over column chunk a of C_m]),
  chunks being S L / L_s consecutive nodes; pool is Linear(2d -> d).
* Edge descriptor (Supp. B): [dx, dy, dz, a] with d in units of the window's side
  (leaf side L^(1/D) for leaves, (S L)^(1/D) for tiles) and a = A_ij / sqrt(A_ii A_jj);
  tile pairs (a, b) use the centroid offset of row chunk a and column chunk b and
  the mean of a over all node pairs between them.  Per layer and stack an MLP
  4 -> 32 -> h (GELU) gives the per-head logit bias.
* Blocks: pre-norm; x += Attn(LN1 x) with the edge bias; then highways on
  y = LN2(x) of both stacks (Sec. 4.3): r_hw[i] = mean of y over the tokens whose
  rows cover i (the diagonal token i and, for each level where i's leaf is in a
  tile's row cluster, that tile's token whose row chunk holds i); c_hw likewise
  with column clusters; g = mean of y over all tokens of both stacks.  A diagonal
  token gathers [y, r_hw[i], c_hw[i], g]; a tile token gathers [y, mean of r_hw
  over its row chunk, mean of c_hw over its column chunk, g].  x += FFN(4d -> d_mlp -> d).
* Heads (Sec. 4.4): F rows = Linear(GELU(Linear(y))) (d -> d -> L); node head
  Linear(d -> 2 L_s + 1) gives U~, V~ and the gate logit; tile head Linear(d -> 2 L_s)
  gives U_m, V_m and B_m = U_m V_m^T.  lambda = softplus(logit).
* Units: every node row of F, U~, V~ is multiplied by diag(A)_i^-1/2 and the gate
  is stored as g_i = lambda_i / diag(A)_i, so M = D^-1/2 (learned) D^-1/2 and the
  gate term is the diag(lambda) diag(A)^-1 of Sec. 4.4.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import grid, hmatrix

TD = torch.float64


# ----------------------------------------------------------------- parameters
def unflatten(blob, layout):
    """Split the flat weight vector into named float64 tensors."""
    blob = torch.as_tensor(np.asarray(blob), dtype=TD)
    out = {}
    off = 0
    for name, shape in layout:
        n = int(np.prod(shape))
        out[name] = blob[off:off + n].reshape(shape).clone()
        off += n
    assert off == blob.numel()
    return out


def gelu(x):
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def linear(p, name, x):
    return x @ p[name + ".w"].T + p[name + ".b"]


def layer_norm(x, g, b, eps=1e-5):
    mu = x.mean(-1, keepdim=True)
    var = ((x - mu) ** 2).mean(-1, keepdim=True)
    return (x - mu) / torch.sqrt(var + eps) * g + b


# ----------------------------------------------------------------- geometry helpers
def coords(dims):
    n = int(np.prod(dims))
    c = np.zeros((n, 3))
    for m in range(n):
        cc = grid.morton_decode(m, dims)
        c[m, :len(dims)] = cc
    return c


def features(sys):
    """Per-node input features (N x 20), see the module docstring."""
    dims = sys["dims"]
    nd = len(dims)
    n = sys["n"]
    rho = sys["rho"]
    d = sys["diag"]
    nbr = grid.neighbours(dims)
    c = coords(dims)
    lr = np.log(rho)
    ld = np.log(d)
    nb = (nbr < 0).sum(1).astype(np.float64)
    off = np.zeros(n)
    iface = np.zeros(n)
    for i in range(n):
        for a in range(nd):
            jp = nbr[i][2 * a + 1]
            jm = nbr[i][2 * a]
            if jp >= 0:
                off[i] += sys["wplus"][a][i]
                if rho[jp] != rho[i]:
                    iface[i] = 1.0
            if jm >= 0:
                off[i] += sys["wplus"][a][jm]
                if rho[jm] != rho[i]:
                    iface[i] = 1.0
    g = np.zeros(12)
    g[0] = math.log2(n) / 16.0
    g[1] = 1.0 if nd == 3 else 0.0
    g[2], g[3], g[4] = lr.max(), lr.min(), lr.mean()
    g[5] = math.sqrt(((lr - g[4]) ** 2).mean())
    g[6] = float((lr > 0.5 * (g[2] + g[3])).mean())
    g[7] = ld.mean()
    g[8] = math.sqrt(((ld - g[7]) ** 2).mean())
    g[9], g[10] = ld.max(), ld.min()
    g[11] = float((nb > 0).mean())
    f = np.zeros((n, 20))
    f[:, 0] = lr - g[4]
    for a in range(nd):
        f[:, 1 + a] = (c[:, a] + 0.5) / dims[a] - 0.5
    f[:, 4] = nb / (2 * nd)
    f[:, 5] = ld - g[7]
    f[:, 6] = off / d
    f[:, 7] = iface
    f[:, 8:] = g[None, :]
    return f


def prop_matrix(sys):
    """P = D^-1 A as a dense-free list of (i, j, w_ij / d_i) couplings."""
    nbr = grid.neighbours(sys["dims"])
    rows, cols, vals = [], [], []
    d = sys["diag"]
    for i in range(sys["n"]):
        for a in range(len(sys["dims"])):
            jp = nbr[i][2 * a + 1]
            if jp >= 0:
                w = sys["wplus"][a][i]
                rows += [i, jp]
                cols += [jp, i]
                vals += [w / d[i], w / d[jp]]
    return (torch.tensor(rows), torch.tensor(cols), torch.tensor(vals, dtype=TD))


def apply_p(pm, h):
    rows, cols, vals = pm
    out = h.clone()
    out = out.index_add(0, rows, -(vals[:, None] * h[cols]))
    return out


def leaf_edges(sys, leaf):
    """Diagonal-window edge descriptors e[k, a, b, 4]."""
    dims = sys["dims"]
    nd = len(dims)
    n = sys["n"]
    k = n // leaf
    c = coords(dims)
    side = round(leaf ** (1.0 / nd))
    nbr = grid.neighbours(dims)
    d = sys["diag"]
    e = np.zeros((k, leaf, leaf, 4))
    for kk in range(k):
        base = kk * leaf
        cc = c[base:base + leaf]
        e[kk, :, :, :3] = (cc[None, :, :] - cc[:, None, :]) / side
        for a in range(leaf):
            e[kk, a, a, 3] = 1.0
            i = base + a
            for ax in range(nd):
                for s in (0, 1):
                    j = nbr[i][2 * ax + s]
                    if j >= 0 and base <= j < base + leaf:
                        w = sys["wplus"][ax][i] if s == 1 else sys["wplus"][ax][j]
                        e[kk, a, j - base, 3] = -w / math.sqrt(d[i] * d[j])
    return e


def tile_geometry(n, leaf, rank):
    """For each tile m: (level, S, row start node, column start node, chunk size)."""
    out = []
    for (m, lev, (r0, r1), (c0, c1)) in hmatrix.partition(n, leaf):
        s = r1 - r0
        out.append((lev, s, r0 * leaf, c0 * leaf, s * leaf // rank))
    return out


def tile_edges(sys, leaf, rank):
    """Off-diagonal-window edge descriptors e[m, a, b, 4] (chunk centroids, mean a_ij)."""
    dims = sys["dims"]
    nd = len(dims)
    n = sys["n"]
    c = coords(dims)
    d = sys["diag"]
    nbr = grid.neighbours(dims)
    geo = tile_geometry(n, leaf, rank)
    mh = len(geo)
    e = np.zeros((mh, rank, rank, 4))
    for m, (lev, s, r0, c0, ch) in enumerate(geo):
        side = (s * leaf) ** (1.0 / nd)
        cr = np.array([c[r0 + a * ch:r0 + (a + 1) * ch].mean(0) for a in range(rank)])
        cc = np.array([c[c0 + b * ch:c0 + (b + 1) * ch].mean(0) for b in range(rank)])
        e[m, :, :, :3] = (cc[None, :, :] - cr[:, None, :]) / side
        acc = np.zeros((rank, rank))
        for a in range(rank):
            for i in range(r0 + a * ch, r0 + (a + 1) * ch):
                for ax in range(nd):
                    j = nbr[i][2 * ax + 1]
                    if j >= c0 and j < c0 + rank * ch:
                        acc[a, (j - c0) // ch] += -sys["wplus"][ax][i] / math.sqrt(d[i] * d[j])
        e[m, :, :, 3] = acc / (ch * ch)
    return e


def edge_bias(p, prefix, e):
    """Per-head logit bias: Linear(GELU(Linear(e))) over the last axis, heads first."""
    x = gelu(linear(p, prefix + "edge1", e))
    b = linear(p, prefix + "edge2", x)            # (..., w, w, h)
    return b.movedim(-1, -3)                        # (..., h, w, w)


# ----------------------------------------------------------------- blocks
def attention(p, prefix, x, win, heads, bias):
    t, d = x.shape
    hd = d // heads
    y = layer_norm(x, p[prefix + "ln1.g"], p[prefix + "ln1.b"])
    qkv = linear(p, prefix + "qkv", y)
    q, k, v = qkv[:, :d], qkv[:, d:2 * d], qkv[:, 2 * d:]
    nw = t // win
    q = q.reshape(nw, win, heads, hd).transpose(1, 2)
    k = k.reshape(nw, win, heads, hd).transpose(1, 2)
    v = v.reshape(nw, win, heads, hd).transpose(1, 2)
    s = q @ k.transpose(-1, -2) / math.sqrt(hd) + bias
    pr = torch.softmax(s, dim=-1)
    o = (pr @ v).transpose(1, 2).reshape(t, d)
    return x + linear(p, prefix + "out", o), pr


def highways(yd, yo, n, leaf, rank):
    """Row/column axial buffers and the global token (Sec. 4.3) from y of both stacks."""
    d = yd.shape[1]
    geo = tile_geometry(n, leaf, rank)
    rsum = yd.clone()
    csum = yd.clone()
    rcnt = torch.ones(n, dtype=TD)
    ccnt = torch.ones(n, dtype=TD)
    for m, (lev, s, r0, c0, ch) in enumerate(geo):
        tok = yo[m * rank:(m + 1) * rank]                  # (rank, d)
        rep = tok.repeat_interleave(ch, dim=0)             # (S L, d)
        rsum = rsum.index_add(0, torch.arange(r0, r0 + rank * ch), rep)
        csum = csum.index_add(0, torch.arange(c0, c0 + rank * ch), rep)
        rcnt[r0:r0 + rank * ch] += 1
        ccnt[c0:c0 + rank * ch] += 1
    rhw = rsum / rcnt[:, None]
    chw = csum / ccnt[:, None]
    g = (yd.sum(0) + yo.sum(0)) / (yd.shape[0] + yo.shape[0])
    ud = torch.cat([yd, rhw, chw, g.expand(n, d)], dim=1)
    ro, co = [], []
    for m, (lev, s, r0, c0, ch) in enumerate(geo):
        ro.append(rhw[r0:r0 + rank * ch].reshape(rank, ch, d).mean(1))
        co.append(chw[c0:c0 + rank * ch].reshape(rank, ch, d).mean(1))
    uo = torch.cat([yo, torch.cat(ro), torch.cat(co), g.expand(yo.shape[0], d)], dim=1)
    return ud, uo


def pool_tokens(h, n, leaf, rank):
    """Pooled inputs of the off-diagonal tokens (Sec. 4.2; Supp. B "Off-diagonal tokens").

    Row a of tile m (in heap order, M_H * L_s rows in all) is [mean of h over row
    chunk a of R_m ; mean of h over column chunk a of C_m], a chunk being the
    S L / L_s consecutive nodes starting at r0 + a * chunk (resp. c0 + a * chunk).
    """
    pooled = []
    for (lev, s, r0, c0, ch) in tile_geometry(n, leaf, rank):
        pr = h[r0:r0 + rank * ch].reshape(rank, ch, -1).mean(1)
        pc = h[c0:c0 + rank * ch].reshape(rank, ch, -1).mean(1)
        pooled.append(torch.cat([pr, pc], dim=1))
    return torch.cat(pooled)


def ffn(p, prefix, x, u):
    return x + linear(p, prefix + "ffn2", gelu(linear(p, prefix + "ffn1", u)))


# ----------------------------------------------------------------- forward
def forward(p, sys, cfg, geom=None, highway=True):
    """Learned factors of one system as the oracle's factor dict (learned layout).

    cfg: dict(d, n_layers, n_heads, d_mlp, leaf, rank).  ``geom`` caches the
    A-dependent inputs (features, P, edge descriptors) across calls.
    """
    n = sys["n"]
    leaf, rank = cfg["leaf"], cfg["rank"]
    heads, nl = cfg["n_heads"], cfg["n_layers"]
    k = n // leaf
    if geom is None:
        geom = geometry(sys, leaf, rank)
    x = torch.as_tensor(geom["feat"], dtype=TD)
    h = linear(p, "enc2", gelu(linear(p, "enc1", x)))
    for g in range(2):
        h = h + gelu(linear(p, f"gcn{g}", apply_p(geom["P"], h)))
    xo = linear(p, "pool", pool_tokens(h, n, leaf, rank))
    xd = h
    ed = torch.as_tensor(geom["edge_leaf"], dtype=TD)
    eo = torch.as_tensor(geom["edge_tile"], dtype=TD)
    for l in range(nl):
        bd = edge_bias(p, f"diag{l}.", ed)
        bo = edge_bias(p, f"off{l}.", eo)
        xd, _ = attention(p, f"diag{l}.", xd, leaf, heads, bd)
        xo, _ = attention(p, f"off{l}.", xo, rank, heads, bo)
        yd = layer_norm(xd, p[f"diag{l}.ln2.g"], p[f"diag{l}.ln2.b"])
        yo = layer_norm(xo, p[f"off{l}.ln2.g"], p[f"off{l}.ln2.b"])
        if highway:
            ud, uo = highways(yd, yo, n, leaf, rank)
        else:
            z = torch.zeros_like
            ud = torch.cat([yd, z(yd), z(yd), z(yd)], 1)
            uo = torch.cat([yo, z(yo), z(yo), z(yo)], 1)
        xd = ffn(p, f"diag{l}.", xd, ud)
        xo = ffn(p, f"off{l}.", xo, uo)
    yd = layer_norm(xd, p["diag.lnf.g"], p["diag.lnf.b"])
    yo = layer_norm(xo, p["off.lnf.g"], p["off.lnf.b"])
    frow = linear(p, "leaf2", gelu(linear(p, "leaf1", yd)))          # (N, L)
    node = linear(p, "node", yd)                                      # (N, 2r + 1)
    offh = linear(p, "off", yo)                                       # (M_H r, 2r)
    dg = torch.as_tensor(sys["diag"], dtype=TD)
    s = 1.0 / torch.sqrt(dg)
    out = dict(layout="learned", n=n, leaf=leaf, rank=rank, K=k)
    out["leafblk"] = (frow * s[:, None]).reshape(k, leaf, leaf)
    out["U"] = node[:, :rank] * s[:, None]
    out["V"] = node[:, rank:2 * rank] * s[:, None]
    out["g"] = torch.nn.functional.softplus(node[:, 2 * rank]) / dg
    u = offh[:, :rank].reshape(k - 1, rank, rank)
    v = offh[:, rank:].reshape(k - 1, rank, rank)
    out["core"] = u @ v.transpose(1, 2)
    # |U_m| |V_m|^T: the scale of each core entry's dot product (a bound for its rounding error)
    out["core_scale"] = u.abs() @ v.abs().transpose(1, 2)
    return out


def geometry(sys, leaf, rank):
    return dict(feat=features(sys), P=prop_matrix(sys), edge_leaf=leaf_edges(sys, leaf),
                edge_tile=tile_edges(sys, leaf, rank))


def to_numpy_factors(f):
    g = dict(f)
    for key in ("leafblk", "U", "V", "g", "core", "core_scale"):
        if key in f:
            g[key] = f[key].detach().numpy()
    return g


# ----------------------------------------------------------------- apply in torch (for the loss)
def apply_torch(f, r):
    """z = M r in torch (same stages as hmatrix.apply), differentiable in the factors."""
    n, leaf, rank, k = f["n"], f["leaf"], f["rank"], f["K"]
    nr = r.shape[1]
    rk = r.reshape(k, leaf, nr)
    blk = f["leafblk"]
    z = blk @ (blk.transpose(1, 2) @ rk) + f["g"].reshape(k, leaf, 1) * rk
    z = z.reshape(n, nr)
    uh = (f["U"].reshape(k, leaf, rank).transpose(1, 2) @ rk)      # (k, r, nr)
    vh = (f["V"].reshape(k, leaf, rank).transpose(1, 2) @ rk)
    au = torch.zeros(k, rank, nr, dtype=r.dtype)
    av = torch.zeros(k, rank, nr, dtype=r.dtype)
    for (m, lev, (r0, r1), (c0, c1)) in hmatrix.partition(n, leaf):
        sr = uh[r0:r1].sum(0)
        sc = vh[c0:c1].sum(0)
        tr = f["core"][m] @ sc
        tc = f["core"][m].T @ sr
        au = au.index_add(0, torch.arange(r0, r1), tr.expand(r1 - r0, rank, nr))
        av = av.index_add(0, torch.arange(c0, c1), tc.expand(c1 - c0, rank, nr))
    dz = f["U"].reshape(k, leaf, rank) @ au + f["V"].reshape(k, leaf, rank) @ av
    return z + dz.reshape(n, nr)
