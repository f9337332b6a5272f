"""Pins for oracle.adamw (against torch.optim.AdamW, a library routine) and oracle.train."""
import numpy as np
import torch

import inputs
from oracle import adamw, grid, loss, network, train


def test_adamw_matches_torch_over_ten_steps():
    rng = np.random.default_rng(0)
    p0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) * 3 for _ in range(10)]
    pt = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.AdamW([pt], lr=3e-3, weight_decay=1e-4)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for s, g in enumerate(grads, start=1):
        gc = adamw.clip_global(g, 1.0)
        opt.zero_grad()
        pt.grad = torch.tensor(g, dtype=torch.float64)
        torch.nn.utils.clip_grad_norm_([pt], 1.0)
        assert np.allclose(pt.grad.numpy(), gc, rtol=0, atol=1e-15)
        opt.step()
        p, m, v = adamw.adamw_step(p, gc, m, v, s, 3e-3)
        assert np.allclose(p, pt.detach().numpy(), rtol=0, atol=1e-12)


def test_batch_loss_gradient_is_mean_of_parts():
    cfg = dict(d=16, n_layers=1, n_heads=2, d_mlp=32, leaf=16, rank=4)
    lay = inputs.network_layout(**cfg)
    blob = inputs.network_blob(2, **cfg)
    systems = [grid.assemble(inputs.density_for_dims(s, (16, 16), 30.0), (16, 16)) for s in (1, 2)]
    l, g, parts = train.batch_loss(blob, lay, cfg, systems, 9, 4)
    assert abs(l - np.mean(parts)) < 1e-14
    # each system alone at the same probes (system index 0 / 1 keys the probes)
    l0, g0, _ = train.batch_loss(blob, lay, cfg, systems[:1], 9, 4)
    assert abs(l0 - parts[0]) < 1e-14
    assert 0.0 < l < 2.0 and np.isfinite(g).all()


def test_sai_scale_bounds_lambda_max():
    # Gershgorin: 2 max A_ii >= lambda_max(A); on a constant-coefficient grid the checkerboard
    # mode brings lambda_max to within a few per cent of it
    for seed, rho_heavy, lo in ((1, 30.0, 0.0), (2, 100.0, 0.0), (3, 1.0, 0.9)):
        dims = (16, 16)
        rho = inputs.density_for_dims(seed, dims, rho_heavy)
        if rho_heavy == 1.0:
            rho = np.ones_like(rho)
        s = grid.assemble(rho, dims)
        lmax = np.linalg.eigvalsh(grid.dense_matrix(s))[-1]
        c = train.sai_scale(s)
        assert c >= lmax * (1 - 1e-12)
        assert lmax >= lo * c


def test_sai_loss_is_the_probe_estimate_of_the_frobenius_distance():
    # E_z ||(M A / c - I) z||^2 = ||M A / c - I||_F^2 for unit-variance probes, and A M and M A
    # give the same expectation (transposes); a dense SPD M stands in for the network
    dims = (8, 8)
    s = grid.assemble(inputs.density_for_dims(4, dims, 20.0), dims)
    a = grid.dense_matrix(s)
    rng = np.random.default_rng(0)
    q = rng.standard_normal((64, 64))
    m = np.linalg.inv(a) + 1e-3 * q @ q.T / 64
    c = train.sai_scale(s)
    exact = np.linalg.norm(m @ a / c - np.eye(64)) ** 2
    z = rng.choice([-1.0, 1.0], size=(64, 20000))
    est_ma = np.sum((m @ (a @ z) / c - z) ** 2) / z.shape[1]
    est_am = loss.sai_loss(z, a @ (m @ z), c) / z.shape[1]
    assert abs(est_ma - exact) <= 0.03 * exact
    assert abs(est_am - exact) <= 0.03 * exact
    # M = c A^-1 zeroes it; doubling M does not keep it (not scale invariant, Prop. 1)
    zero = loss.sai_loss(z[:, :8], a @ (c * np.linalg.inv(a) @ z[:, :8]), c)
    assert zero <= 1e-20 * z[:, :8].size


def test_batch_loss_sai_is_scale_sensitive_and_highway_switch():
    cfg = dict(d=16, n_layers=1, n_heads=2, d_mlp=32, leaf=16, rank=4)
    lay = inputs.network_layout(**cfg)
    blob = inputs.network_blob(2, **cfg)
    systems = [grid.assemble(inputs.density_for_dims(s, (16, 16), 30.0), (16, 16)) for s in (1, 2)]
    l, g, parts = train.batch_loss(blob, lay, cfg, systems, 9, 4, loss_kind="sai")
    assert abs(l - np.mean(parts)) < 1e-14 and l > 0 and np.isfinite(g).all()
    # highway=False equals highway=True with the FFN columns that read the highway channels
    # zeroed (first FFN layer input is [y, r_hw, c_hw, g_hw], 4d wide)
    d = cfg["d"]
    b2 = blob.astype(np.float64).copy()
    off = 0
    for name, shp in lay:
        k = int(np.prod(shp))
        if name.endswith(".ffn1.w"):
            w = b2[off:off + k].reshape(shp)
            w[:, d:] = 0.0
        off += k
    assert any(name.endswith(".ffn1.w") for name, _ in lay)
    l_on, _, _ = train.batch_loss(b2, lay, cfg, systems, 9, 4, grad=False)
    l_off, _, _ = train.batch_loss(b2, lay, cfg, systems, 9, 4, grad=False, highway=False)
    assert abs(l_on - l_off) <= 1e-13
    l_full, _, _ = train.batch_loss(blob, lay, cfg, systems, 9, 4, grad=False)
    l_full_off, _, _ = train.batch_loss(blob, lay, cfg, systems, 9, 4, grad=False, highway=False)
    assert abs(l_full - l_full_off) > 1e-9
