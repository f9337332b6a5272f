"""Pins for oracle.network (Sec. 4; Supp. B) and the loss through it (Sec. 6.1)."""
import math

import numpy as np
import pytest
import torch

import inputs
from oracle import grid, hmatrix, loss, network

TINY = dict(d=16, n_layers=1, n_heads=2, d_mlp=32, leaf=16, rank=4)


def _sys(dims=(16, 16), seed=1):
    rho = inputs.density_for_dims(seed, dims, rho_heavy=20.0)
    return grid.assemble(rho, dims)


def test_parameter_count_matches_paper():
    # Sec. 7.3: about 2.6M parameters at d=128, n_l=3, h=8, L=128, L_s=32, 4d FFN input
    lay = inputs.network_layout(d=128, n_layers=3, n_heads=8, d_mlp=512, leaf=128, rank=32)
    total = sum(int(np.prod(s)) for _, s in lay)
    assert abs(total - 2.6e6) / 2.6e6 < 0.05


def test_features_uniform_grid():
    s = grid.assemble(np.ones(64), (8, 8))
    f = network.features(s)
    assert np.allclose(f[:, 0], 0) and np.allclose(f[:, 7], 0)
    assert np.allclose(f[:, 8 + 2], 0) and np.allclose(f[:, 8 + 3], 0)
    # interior cells couple fully (off / diag = 1), corner cells 2 of 4 faces
    c = network.coords((8, 8))
    inner = (c[:, 0] > 0) & (c[:, 0] < 7) & (c[:, 1] > 0) & (c[:, 1] < 7)
    assert np.allclose(f[inner, 6], 1.0) and np.allclose(f[inner, 4], 0.0)
    assert math.isclose(f[0, 6], 0.5) and math.isclose(f[0, 4], 0.5)
    assert math.isclose(f[0, 8 + 11], 28 / 64)


def test_edge_descriptors_against_dense_a():
    s = _sys((16, 16), 3)
    a = grid.dense_matrix(s)
    dn = np.sqrt(np.diag(a))
    an = a / dn[:, None] / dn[None, :]
    e = network.leaf_edges(s, 16)
    for k in range(16):
        blk = an[k * 16:(k + 1) * 16, k * 16:(k + 1) * 16]
        assert np.allclose(e[k, :, :, 3], blk, atol=1e-15)
        assert np.allclose(e[k, :, :, :3], -e[k, :, :, :3].transpose(1, 0, 2))
    et = network.tile_edges(s, 16, 4)
    for m, (lev, ss, r0, c0, ch) in enumerate(network.tile_geometry(256, 16, 4)):
        for aa in range(4):
            for bb in range(4):
                blk = an[r0 + aa * ch:r0 + (aa + 1) * ch, c0 + bb * ch:c0 + (bb + 1) * ch]
                assert math.isclose(et[m, aa, bb, 3], blk.mean(), abs_tol=1e-15)


def test_attention_rows_sum_to_one_and_window_equivariance():
    torch.manual_seed(0)
    lay = inputs.network_layout(**TINY)
    p = network.unflatten(inputs.network_blob(3, **TINY), lay)
    x = torch.randn(32, 16, dtype=torch.float64)
    out, pr = network.attention(p, "diag0.", x, 16, 2, torch.zeros(2, 2, 16, 16, dtype=torch.float64))
    assert torch.allclose(pr.sum(-1), torch.ones_like(pr.sum(-1)), atol=1e-14)
    # without bias the block is permutation-equivariant within a window
    perm = torch.randperm(16)
    xp = x.clone()
    xp[:16] = x[:16][perm]
    outp, _ = network.attention(p, "diag0.", xp, 16, 2, torch.zeros(2, 2, 16, 16, dtype=torch.float64))
    assert torch.allclose(outp[:16], out[:16][perm], atol=1e-12)


def test_apply_torch_matches_structured_apply():
    rng = np.random.default_rng(0)
    n, leaf, rank = 256, 16, 4
    f = hmatrix.unpack(rng.standard_normal(hmatrix.packed_width(n, leaf, rank)), n, leaf, rank, "learned")
    ft = {k: (torch.as_tensor(v) if isinstance(v, np.ndarray) else v) for k, v in f.items()}
    r = rng.standard_normal((n, 3))
    got = network.apply_torch(ft, torch.as_tensor(r)).numpy()
    assert np.allclose(got, hmatrix.apply(f, r), atol=1e-12)


def test_init_is_near_jacobi_and_factors_finite():
    s = _sys((16, 16), 2)
    lay = inputs.network_layout(**TINY)
    p = network.unflatten(inputs.network_blob(0, **TINY), lay)
    f = network.to_numpy_factors(network.forward(p, s, TINY))
    m = hmatrix.dense_m(f)
    d = s["diag"]
    assert np.allclose(np.diag(m) * d, 1.0, atol=1e-3)
    off = m - np.diag(np.diag(m))
    assert np.abs(off * np.sqrt(d[:, None] * d[None, :])).max() < 1e-3


def test_loss_gradient_finite_differences():
    # central differences of the FP64 oracle (h = 1e-6) against autograd, tiny config
    s = _sys((16, 16), 4)
    lay = inputs.network_layout(**TINY)
    blob = inputs.network_blob(1, **TINY).astype(np.float64)
    geom = network.geometry(s, 16, 4)
    a = grid.sparse_matrix(s)
    z = loss.rademacher_probes(5, 0, 256, 8)
    w = torch.as_tensor(a @ z)
    # enlarge the heads so every parameter carries signal
    p0 = network.unflatten(blob, lay)
    for key in ("leaf2.w", "node.w", "off.w"):
        p0[key] = p0[key] * 100.0
    names = [k for k, _ in lay]
    flat = torch.cat([p0[k].reshape(-1) for k in names]).clone().requires_grad_(True)

    def lossf(vec):
        off = 0
        p = {}
        for k, shp in lay:
            nel = int(np.prod(shp))
            p[k] = vec[off:off + nel].reshape(shp)
            off += nel
        f = network.forward(p, s, TINY, geom=geom)
        y = network.apply_torch(f, w)
        zt = torch.as_tensor(z)
        return 1.0 - (zt * y).sum() / (zt.norm() * y.norm())

    l0 = lossf(flat)
    (g,) = torch.autograd.grad(l0, flat)
    rng = np.random.default_rng(2)
    idx = rng.choice(flat.numel(), 24, replace=False)
    offs = {}
    o = 0
    for k, shp in lay:
        offs[k] = o
        o += int(np.prod(shp))
    idx = list(idx) + [offs["leaf2.w"] + 3, offs["off.w"] + 5, offs["diag0.edge2.w"] + 1,
                       offs["off0.qkv.w"] + 7, offs["pool.w"] + 2, offs["node.b"] + 8]
    hstep = 1e-6
    with torch.no_grad():
        for i in idx:
            e = torch.zeros_like(flat)
            e[i] = hstep
            fd = (lossf(flat + e) - lossf(flat - e)) / (2 * hstep)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g).max()) + 1e-6 * abs(g[i]), (i, fd, g[i])
