"""GPU training step against the FP64 oracle (loss, clipped gradient, AdamW update).

The GPU step runs the forward and every backward GEMM with BF16 operands and FP32
accumulation; the clipped gradient is compared with the oracle's (torch autograd
in FP64 on the same weights, systems and SplitMix64 probes, Rademacher or the
paper's smoothed Gaussian ones) by relative 2-norm error over the whole vector
and over each tensor that carries a share of it.
"""
import numpy as np
import pytest
import torch

import inputs
from oracle import adamw, grid, train

pytestmark = pytest.mark.gpu
h = pytest.importorskip("paper_2605_13343_gb300")

SMALL = dict(d=64, n_layers=1, n_heads=2, d_mlp=64, leaf=16, rank=16)
CFG3 = dict(d=128, n_layers=4, n_heads=4, d_mlp=512, leaf=64, rank=16)
# the paper's model size (Sec. 7.3): 8 heads of 16, 128-token leaf windows, rank 32
PAPER = dict(d=128, n_layers=3, n_heads=8, d_mlp=512, leaf=128, rank=32)


def _blob(cfg, seed, scale_heads=100.0):
    lay = inputs.network_layout(**cfg)
    w = inputs.network_blob(seed, **cfg)
    off = 0
    for name, shp in lay:
        k = int(np.prod(shp))
        if name in ("leaf2.w", "node.w", "off.w"):
            w[off:off + k] *= scale_heads
        off += k
    return w, lay


def _ctx(cfg, n, batch, w):
    return h.Context(max_n=n, leaf=cfg["leaf"], rank=cfg["rank"], d_model=cfg["d"], n_layers=cfg["n_layers"],
                     n_heads=cfg["n_heads"], d_mlp=cfg["d_mlp"], max_batch=batch, weights=w)


def _systems(dims, seeds):
    out_gpu, out_ref = [], []
    for s in seeds:
        rho = inputs.density_for_dims(s, dims, rho_heavy=float(np.exp(np.random.default_rng(s).uniform(0, np.log(100)))))
        sg = h.System(dims)
        h.assemble(torch.from_numpy(rho).cuda(), sg)
        out_gpu.append(sg)
        out_ref.append(grid.assemble(rho, dims))
    return out_gpu, out_ref


def _gpu_systems(dims, seeds):
    """Device systems only (the held-out test needs no oracle copies)."""
    out = []
    for s in seeds:
        rho = inputs.density_for_dims(s, dims, rho_heavy=float(np.exp(np.random.default_rng(s).uniform(0, np.log(100)))))
        sg = h.System(dims)
        h.assemble(torch.from_numpy(rho).cuda(), sg)
        out.append(sg)
    return out


# Relative 2-norm bounds of the clipped gradient against the FP64 oracle.  The GPU rounds every GEMM
# operand and stored activation to BF16 (unit roundoff u = 2^-9) on a path of about 60 roundings
# (forward and backward through 4 layers); independent errors add in quadrature, sqrt(60) u ~ 0.015,
# and the measured worst tensor on the GB300 was 0.023 (whole vector 0.018).  A tensor carrying at
# least 1% of the gradient norm (or 0.1% if it has >= 4096 entries) must be within 0.05, the whole
# vector within 0.04: a wrong sign, transposition or dropped term in any such tensor gives an error
# of order 1.  The bounds hold where the per-system loss is not small: near the minimum of Eq. 7
# dL/dY is a difference of two nearly equal terms and amplifies the BF16 error of Y by about
# 1 / L (on systems 7 and 8, with losses 0.14 and 0.08, the off-diagonal stack's tensors measured
# 0.03-0.09 on the GB300), so every case runs on systems whose loss at this initialisation is
# far from zero; the SAI and highway-off cases reuse systems 3 and 4 of the measured budget.
REL_TENSOR = 0.05
REL_ALL = 0.04
# The cosine loss is 1-Lipschitz in the unit vector Y / ||Y||, so |dL| <= 2 ||dY|| / ||Y||: the
# loss inherits the BF16 forward's error in M A Z, about 0.5 % per factor block (1 % with the
# paper's 8 heads and 128-token windows, whose loss measured 2.5e-3 off on the GB300; the
# benchmark network below 1e-3).  2 x 0.5 % bounds the loss error at 1e-2.
LOSS_TOL = 1e-2


@pytest.mark.parametrize("cfg,dims,seeds,nz,probes,loss_kind,highway", [
    (SMALL, (16, 16), [1, 2], 8, "rademacher", "cosine", True),
    (CFG3, (16, 16, 16), [3, 4], 16, "rademacher", "cosine", True),
    (CFG3, (16, 16, 16), [5, 6], 16, "gaussian", "cosine", True),
    (CFG3, (16, 16, 16), [3, 4], 16, "rademacher", "sai", True),
    (CFG3, (16, 16, 16), [3, 4], 16, "rademacher", "cosine", False),
    (PAPER, (64, 64), [3], 16, "rademacher", "cosine", True),
    # the paper's probe objective as printed: K_z = max(64, sqrt(4096)) = 64 smoothed Gaussian probes
    (CFG3, (16, 16, 16), [3, 4], 64, "gaussian", "cosine", True)])
def test_train_step_gradient_parity(cfg, dims, seeds, nz, probes, loss_kind, highway):
    # The paper-size network (rank 32) forms tile cores B_m = U_m V_m^T whose entries cancel: on
    # 2D frames the ratio ||(|U_m||V_m|^T)|| / ||U_m V_m^T|| is 4.3, 14.9 and 20.0 on systems 3, 4
    # and 5, and every gradient through a core inherits the BF16 error of U_m and V_m times that
    # ratio (the GB300 measured whole-vector errors 0.015, 0.045 and 0.117 on them).  Its case runs
    # on system 3, with heads scaled so that the loss stays near 1 (away from the minimum, where
    # Eq. 7's gradient adds its own amplification, see above).
    w, lay = _blob(cfg, 5, scale_heads=300.0 if cfg is PAPER else 100.0)
    n = int(np.prod(dims))
    ctx = _ctx(cfg, n, len(seeds), w)
    if probes == "gaussian":
        h.set_train_probes(ctx, h.PROBES_GAUSSIAN_SMOOTHED, 0.6, 2)
    if loss_kind == "sai":
        h.set_train_loss(ctx, h.LOSS_SAI)
    if not highway:
        h.set_highways(ctx, False)
    sg, sr = _systems(dims, seeds)
    loss_gpu = h.train_step(ctx, sg, nz, 0.0, 1234)
    g_gpu = h.get_grads(ctx, w.size).astype(np.float64)
    l_ref, g_ref, _ = train.batch_loss(w.astype(np.float64), lay, cfg, sr, 1234, nz, probes=probes,
                                       loss_kind=loss_kind, highway=highway)
    g_ref = adamw.clip_global(g_ref, 1.0)
    assert abs(loss_gpu - l_ref) <= LOSS_TOL, (loss_gpu, l_ref)
    tot = np.linalg.norm(g_ref)
    assert np.linalg.norm(g_gpu - g_ref) <= REL_ALL * tot, np.linalg.norm(g_gpu - g_ref) / tot
    off = 0
    for name, shp in lay:
        k = int(np.prod(shp))
        a, b = g_gpu[off:off + k], g_ref[off:off + k]
        off += k
        nb = np.linalg.norm(b)
        if nb >= 1e-2 * tot or (k >= 4096 and nb >= 1e-3 * tot):
            assert np.linalg.norm(a - b) <= REL_TENSOR * nb, (name, np.linalg.norm(a - b) / nb)
    # lr = 0 left the weights untouched
    assert np.array_equal(h.get_weights(ctx, w.size), w)
    ctx.close()


def test_adamw_update_matches_oracle():
    w, lay = _blob(SMALL, 6)
    ctx = _ctx(SMALL, 256, 2, w)
    sg, _ = _systems((16, 16), [7, 8])
    h.train_step(ctx, sg, 8, 1e-3, 99)
    g = h.get_grads(ctx, w.size).astype(np.float64)
    w1 = h.get_weights(ctx, w.size).astype(np.float64)
    p, m, v = adamw.adamw_step(w.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    assert np.abs(w1 - p).max() <= 1e-6
    ctx.close()


def test_training_lowers_heldout_loss():
    """Steps on fresh batches (new frames every step, new probes) lower the loss of a held-out
    batch of other frames with fixed probes (evaluated with lr = 0, which changes nothing): what
    the training learns carries over to systems it never saw."""
    w = inputs.network_blob(0, **CFG3)
    ctx = _ctx(CFG3, 4096, 4, w)
    held = _gpu_systems((16, 16, 16), [9100 + q for q in range(4)])
    before = h.train_step(ctx, held, 16, 0.0, 777)
    for step in range(STEPS_HELDOUT):
        sg = _gpu_systems((16, 16, 16), [20000 + 4 * step + q for q in range(4)])
        h.train_step(ctx, sg, 16, LR_HELDOUT, 5000 + step, want_loss=False)
    after = h.train_step(ctx, held, 16, 0.0, 777)
    assert after < before * (1.0 - DROP_HELDOUT), (before, after)
    ctx.close()


# 200 AdamW steps at the paper's learning rate 3e-4 (Supp. C) from the seeded initialisation; on
# the GB300 the held-out loss fell monotonically at every 25-step check, 0.0727 -> 0.0700 (3.7 %),
# so a 2 % drop is required.  (At 1e-3 the run is unstable: the loss first jumps to 0.116.)
STEPS_HELDOUT = 200
LR_HELDOUT = 3e-4
DROP_HELDOUT = 0.02
