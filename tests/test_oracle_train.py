"""Pins for oracle.adamw (against torch.optim.AdamW, a library routine) and oracle.train."""
import numpy as np
import torch

import inputs
from oracle import adamw, grid, network, train


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
