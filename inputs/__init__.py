"""Seeded synthetic workloads shared by the CUDA path's tests, the bench and the oracle.

This module only draws random inputs: per-cell density fields (in lexicographic
order, x fastest), zero-mean right-hand sides and seeded network weights.  It
holds none of the method's arithmetic (no ordering, no assembly, no
preconditioner), so importing it on either side couples nothing but the data.

Workload shapes follow the multiphase Poisson benchmark of Supp. D (density
contrast between a light phase rho=1 and heavy inclusions, b ~ N(0, I) projected
to zero mean).  Most frame families use discs (2D) and spheres (3D); the
paper's own rectangular-barrier generator is ``density_barriers`` (frame
families ``barriers2d_<N>``).
"""
from __future__ import annotations

import math
import numpy as np

__all__ = [
    "grid_centres", "density_discs", "density_spheres", "barrier_mask", "density_barriers",
    "BARRIER_GAPS", "rhs", "frame",
    "FRAMES", "batch_mixed_dims", "density_for_dims", "network_layout", "network_blob",
]


def grid_centres(dims):
    """Cell-centre coordinates (x, y[, z]) for a lexicographic grid, x fastest."""
    axes = [np.arange(n, dtype=np.float64) + 0.5 for n in dims]
    mesh = np.meshgrid(*axes, indexing="ij")
    # meshgrid with indexing='ij' gives shape (nx, ny[, nz]); lexicographic with x
    # fastest is Fortran order of that array.
    return [m.ravel(order="F") for m in mesh]


def density_discs(seed, dims=(32, 32), n_discs=1, r=(8.0, 8.0), rho_heavy=10.0,
                  centre_margin=True):
    """2D density: 1 outside, ``rho_heavy`` inside the union of ``n_discs`` discs.

    Radii are uniform in [r[0], r[1]] (a single value when equal); centres are
    uniform in [r, W - r] x [r, H - r] when ``centre_margin`` else in the box.
    A cell is heavy iff its centre lies within distance r of a disc centre
    (comparison in float64).
    """
    rng = np.random.default_rng(seed)
    cx, cy = grid_centres(dims)
    heavy = np.zeros(cx.shape, dtype=bool)
    for _ in range(n_discs):
        rad = float(rng.uniform(r[0], r[1])) if r[1] > r[0] else float(r[0])
        lo = rad if centre_margin else 0.0
        px = rng.uniform(lo, dims[0] - lo)
        py = rng.uniform(lo, dims[1] - lo)
        heavy |= (cx - px) ** 2 + (cy - py) ** 2 <= rad * rad
    rho = np.ones(cx.shape, dtype=np.float64)
    rho[heavy] = rho_heavy
    return rho


def density_spheres(seed, dims=(32, 16, 16), n_range=(5, 12), r=(2.0, 6.0),
                    rho_heavy=100.0):
    """3D density: 1 outside, ``rho_heavy`` inside the union of n spheres.

    n is uniform in {n_range[0], ..., n_range[1]}; radii uniform in [r0, r1];
    centres uniform in the box.  ``rho_heavy`` may be the string "loguniform"
    to draw the contrast log-uniformly in [1, 100] for this frame.
    """
    rng = np.random.default_rng(seed)
    if isinstance(rho_heavy, str):
        rho_heavy = float(math.exp(rng.uniform(0.0, math.log(100.0))))
    c = grid_centres(dims)
    heavy = np.zeros(c[0].shape, dtype=bool)
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    for _ in range(n):
        rad = float(rng.uniform(r[0], r[1]))
        ctr = [rng.uniform(0.0, d) for d in dims]
        d2 = sum((c[a] - ctr[a]) ** 2 for a in range(len(dims)))
        heavy |= d2 <= rad * rad
    rho = np.ones(c[0].shape, dtype=np.float64)
    rho[heavy] = rho_heavy
    return rho


BARRIER_GAPS = ("top", "bottom", "middle_hole", "closed")


def barrier_mask(dims, vertical, centre, thickness, gap_kind, gap=0.2):
    """Cells covered by one rectangular barrier of the 2D benchmark (Supp. D, "Density field").

    Coordinates are normalised cell centres u = (i + 1/2) / W, v = (j + 1/2) / H.  A vertical
    barrier covers the band |u - centre| <= thickness / 2 over the full height except its gap;
    a horizontal one swaps the axes.  The gap is a window of normalised length ``gap`` along the
    barrier: at its high end ("top"), its low end ("bottom"), centred ("middle_hole"), or absent
    ("closed").  Returns a boolean mask in lexicographic order (x fastest).
    """
    cx, cy = grid_centres(dims)
    u, v = cx / dims[0], cy / dims[1]
    across, along = (u, v) if vertical else (v, u)
    band = np.abs(across - centre) <= 0.5 * thickness
    if gap_kind == "top":
        hole = along > 1.0 - gap
    elif gap_kind == "bottom":
        hole = along < gap
    elif gap_kind == "middle_hole":
        hole = np.abs(along - 0.5) < 0.5 * gap
    elif gap_kind == "closed":
        hole = np.zeros_like(band)
    else:
        raise ValueError(gap_kind)
    return band & ~hole


def density_barriers(seed, dims=(32, 32), rho_range=(5.0, 100.0), jitter=0.05, gap=0.2,
                     return_params=False):
    """2D density of the paper's benchmark generator (Supp. D, "Density field").

    rho_heavy is log-uniform in ``rho_range``; light cells have density 1.  One to three
    barriers (uniform count), each with an equiprobable orientation, a centre U[0.2, 0.8] on
    the cross axis, a thickness U[0.05, 0.20] and a gap kind uniform over ``BARRIER_GAPS``
    (see ``barrier_mask``).  A cell is heavy iff any barrier covers it.  Every cell's density
    is then multiplied by 1 + N(0, jitter^2).
    """
    if len(dims) != 2:
        raise ValueError("the barrier generator is 2D")
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xBA55]))
    rho_heavy = float(math.exp(rng.uniform(math.log(rho_range[0]), math.log(rho_range[1]))))
    nb = int(rng.integers(1, 4))
    params = []
    heavy = np.zeros(dims[0] * dims[1], dtype=bool)
    for _ in range(nb):
        vertical = bool(rng.integers(0, 2))
        centre = float(rng.uniform(0.2, 0.8))
        thickness = float(rng.uniform(0.05, 0.20))
        kind = BARRIER_GAPS[int(rng.integers(0, len(BARRIER_GAPS)))]
        params.append(dict(vertical=vertical, centre=centre, thickness=thickness, gap_kind=kind))
        heavy |= barrier_mask(dims, vertical, centre, thickness, kind, gap)
    rho = np.where(heavy, rho_heavy, 1.0)
    rho = rho * (1.0 + jitter * rng.standard_normal(rho.shape))
    if return_params:
        return rho, dict(rho_heavy=rho_heavy, barriers=params, heavy=heavy)
    return rho


def rhs(seed, n):
    """b ~ N(0, I) of length n, projected onto the complement of the constant
    vector (Supp. D, right-hand side).  Drawn directly in solver order."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xB]))
    b = rng.standard_normal(n)
    return b - b.mean()


# Named frame families.  Each maps a seed to (dims, rho, b, hyper-parameters).
FRAMES = {
    # one disc of contrast 10 in a 32x32 square: the plain SVD-H workload
    "disc2d_1024": dict(dims=(32, 32), leaf=64, rank=16,
                        gen=lambda s: density_discs(s, (32, 32), 1, (8.0, 8.0), 10.0)),
    # 5-12 spheres of contrast 100 in a 32x16x16 box: the learned-inference workload
    "spheres3d_8192": dict(dims=(32, 16, 16), leaf=64, rank=16,
                           gen=lambda s: density_spheres(s, (32, 16, 16))),
    # training systems: 16^3 boxes, contrast log-uniform in [1, 100]
    "spheres3d_4096_lu": dict(dims=(16, 16, 16), leaf=64, rank=16,
                              gen=lambda s: density_spheres(s, (16, 16, 16),
                                                            rho_heavy="loguniform")),
    # 20 discs of contrast 100 in a 128x128 square: the precision sweep
    "discs2d_16384": dict(dims=(128, 128), leaf=64, rank=32,
                          gen=lambda s: density_discs(s, (128, 128), 20, (2.0, 8.0),
                                                      100.0, centre_margin=False)),
}
# the paper's own benchmark distribution (Supp. D): 1-3 barriers, contrast log-uniform in
# [5, 100], 5 % jitter, zero-flux boundaries, w = 2 rho_i rho_j / (rho_i + rho_j), rtol 1e-8;
# N from 1024 to 16384 on square-as-possible power-of-two grids
for _n, _d in ((1024, (32, 32)), (2048, (64, 32)), (4096, (64, 64)), (8192, (128, 64)),
               (16384, (128, 128))):
    FRAMES[f"barriers2d_{_n}"] = dict(dims=_d, leaf=64, rank=16, bc="neumann", face="rho", rtol=1e-8,
                                      gen=(lambda d: (lambda s: density_barriers(s, d)))(_d))
del _n, _d


def split_seeds(seed, n_train, n_test):
    """Disjoint frame seeds of one training/test split (Supp. D: 100 training and 20 test frames
    per scale): training seeds start at 100000 (seed + 1), test seeds 50000 above them."""
    base = 100000 * (seed + 1)
    return list(range(base, base + n_train)), list(range(base + 50000, base + 50000 + n_test))


def frame(family, seed):
    """Return dict(dims, rho, b, leaf, rank, bc, face, rtol) for one seeded frame of
    ``family`` (bc, face and rtol default to Dirichlet, 2/(rho_i+rho_j) and 1e-6)."""
    f = FRAMES[family]
    rho = f["gen"](seed)
    n = int(np.prod(f["dims"]))
    return dict(dims=tuple(f["dims"]), rho=rho, b=rhs(seed, n),
                leaf=f["leaf"], rank=f["rank"], bc=f.get("bc", "dirichlet"),
                face=f.get("face", "inv_rho"), rtol=f.get("rtol", 1e-6))


_MIXED_2D = {1024: (32, 32), 2048: (64, 32), 4096: (64, 64), 8192: (128, 64),
             16384: (128, 128)}
_MIXED_3D = {1024: (16, 8, 8), 2048: (16, 16, 8), 4096: (16, 16, 16),
             8192: (32, 16, 16), 16384: (32, 32, 16)}


def batch_mixed_dims(seed, count=64):
    """Grid shapes of a ragged batch: N uniform over {1024, ..., 16384},
    2D and 3D alternating by system index."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xBA7C]))
    sizes = rng.choice(sorted(_MIXED_2D), size=count)
    return [(_MIXED_2D if i % 2 == 0 else _MIXED_3D)[int(n)] for i, n in enumerate(sizes)]


def density_for_dims(seed, dims, rho_heavy=100.0):
    """1:rho_heavy density for an arbitrary grid: spheres (3D) or discs (2D)."""
    if len(dims) == 3:
        return density_spheres(seed, dims, rho_heavy=rho_heavy)
    n = max(1, (dims[0] * dims[1]) // 800)
    return density_discs(seed, dims, n, (2.0, 8.0), rho_heavy, centre_margin=False)


# ---------------------------------------------------------------- network weight layout
# The flat weight blob is an interface shared by both sides (like the packed
# factor layout): an ordered list of named float32 tensors.  Linear layers are
# stored as (out, in) followed by their bias.
N_NODE_FEATURES = 8
N_GLOBAL_FEATURES = 12
EDGE_HIDDEN = 32


def network_layout(d=128, n_layers=4, n_heads=4, d_mlp=512, leaf=64, rank=16):
    f_in = N_NODE_FEATURES + N_GLOBAL_FEATURES
    out = [("enc1.w", (d, f_in)), ("enc1.b", (d,)), ("enc2.w", (d, d)), ("enc2.b", (d,))]
    for g in range(2):
        out += [(f"gcn{g}.w", (d, d)), (f"gcn{g}.b", (d,))]
    out += [("pool.w", (d, 2 * d)), ("pool.b", (d,))]
    for s in ("diag", "off"):
        for l in range(n_layers):
            p = f"{s}{l}."
            out += [(p + "ln1.g", (d,)), (p + "ln1.b", (d,)),
                    (p + "qkv.w", (3 * d, d)), (p + "qkv.b", (3 * d,)),
                    (p + "out.w", (d, d)), (p + "out.b", (d,)),
                    (p + "ln2.g", (d,)), (p + "ln2.b", (d,)),
                    (p + "ffn1.w", (d_mlp, 4 * d)), (p + "ffn1.b", (d_mlp,)),
                    (p + "ffn2.w", (d, d_mlp)), (p + "ffn2.b", (d,)),
                    (p + "edge1.w", (EDGE_HIDDEN, 4)), (p + "edge1.b", (EDGE_HIDDEN,)),
                    (p + "edge2.w", (n_heads, EDGE_HIDDEN)), (p + "edge2.b", (n_heads,))]
        out += [(f"{s}.lnf.g", (d,)), (f"{s}.lnf.b", (d,))]
    out += [("leaf1.w", (d, d)), ("leaf1.b", (d,)), ("leaf2.w", (leaf, d)), ("leaf2.b", (leaf,)),
            ("node.w", (2 * rank + 1, d)), ("node.b", (2 * rank + 1,)),
            ("off.w", (2 * rank, d)), ("off.b", (2 * rank,))]
    return out


def network_init_rule(name):
    """Seeded init: truncated normal(0, 0.02) weights, zero biases, unit LayerNorm
    gains; the factor heads start 100x smaller so that M starts near the Jacobi
    gate; the gate bias starts at log(e - 1) so that softplus gives lambda = 1."""
    if name.endswith(".g"):
        return ("const", 1.0)
    if name == "node.b":
        return ("gate_bias", math.log(math.e - 1.0))
    if name.endswith(".b"):
        return ("const", 0.0)
    if name in ("leaf2.w", "node.w", "off.w"):
        return ("normal", 0.02 * 1e-2)
    return ("normal", 0.02)


def network_blob(seed, **cfg):
    """Flat float32 weight vector for ``network_layout(**cfg)``."""
    shapes = network_layout(**cfg)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x3E7]))
    parts = []
    for name, shape in shapes:
        kind, val = network_init_rule(name)
        size = int(np.prod(shape))
        if kind == "normal":
            x = np.clip(rng.standard_normal(size), -2.0, 2.0) * val
        elif kind == "gate_bias":
            x = np.zeros(size)
            x[-1] = val
        else:
            x = np.full(size, val)
        parts.append(x.astype(np.float32))
    return np.concatenate(parts)
