"""GPU parity on the paper's own benchmark distribution (Supp. D; Supp. A): 2D barrier frames
with zero-flux boundaries, the face rule 2 rho_i rho_j / (rho_i + rho_j), zero-mean b and PCG to
rtol 1e-8.

A has the constant null space, so solutions are compared after removing their mean; the oracle's
pins for these frames live in test_oracle_barriers.py.  Parity: a true relative residual <= 1e-8
evaluated by the oracle in FP64, and the iteration count within 20 % of the FP64 oracle PCG on the
same preconditioner.  At rtol 1e-8 the FP32 vectors of the GPU iteration (Supp. G: FP32 apply path,
FP64 scalars) lose orthogonality over ~200 Jacobi iterations and converge later than FP64 CG: the
GB300 measured +12 % (199 vs 177) on one of these frames, where rtol 1e-6 frames stay within 2 %.
"""
import numpy as np
import pytest
import torch

import inputs
from oracle import grid, hmatrix, pcg

pytestmark = pytest.mark.gpu
h = pytest.importorskip("paper_2605_13343_gb300")


ITER_TOL = 0.20


@pytest.fixture(params=["cluster", "grid"])
def path(request, monkeypatch):
    monkeypatch.setenv("HMPCG_PCG_PATH", request.param)
    return request.param


@pytest.fixture(scope="module")
def ctx():
    c = h.Context(max_n=1 << 14, leaf=64, rank=16)
    yield c
    c.close()


def _frame(n, seed):
    fr = inputs.frame(f"barriers2d_{n}", seed)
    ref = grid.assemble(fr["rho"], fr["dims"], bc=fr["bc"], face=fr["face"])
    s = h.System(fr["dims"])
    h.assemble(torch.from_numpy(fr["rho"]).cuda(), s, bc=1, face=1)
    torch.cuda.synchronize()
    assert np.array_equal(s.diag.cpu().numpy(), ref["diag"])
    return fr, ref, s


def _check(info, out, a, fr, xg):
    assert info.status == h.OK and out["status"] == pcg.OK
    assert abs(info.iters - out["iters"]) <= max(2, ITER_TOL * out["iters"]), (info.iters, out["iters"])
    rel = np.linalg.norm(fr["b"] - a @ xg) / np.linalg.norm(fr["b"])
    assert rel <= fr["rtol"], rel


@pytest.mark.parametrize("n,seed", [(1024, 0), (1024, 1), (4096, 2), (16384, 3)])
def test_jacobi_pcg_rtol_1e8(ctx, path, n, seed):
    fr, ref, s = _frame(n, seed)
    a = grid.sparse_matrix(ref)
    out = pcg.pcg(lambda v: a @ v, lambda v: v / ref["diag"], fr["b"], rtol=fr["rtol"])
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    fac = h.Factors()
    fac.kind = h.PRE_JACOBI
    info = h.solve(ctx, s, fac, b, x, rtol=fr["rtol"])
    xg = x.cpu().numpy()
    _check(info, out, a, fr, xg)
    # the same solution up to the null space (a constant)
    d = (xg - xg.mean()) - (out["x"] - out["x"].mean())
    assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(out["x"] - out["x"].mean())


@pytest.mark.parametrize("seed", [0, 3])
def test_learned_pcg_rtol_1e8(path, seed):
    """The paper's method on its own frames: factors inferred on the GPU (seeded network with the
    benchmark configuration's sizes; heads scaled up so that the off-diagonal terms matter), PCG to
    rtol 1e-8 against the FP64 oracle PCG on the same packed factors."""
    from oracle import network  # noqa: F401  (the oracle side reads only the packed factors)
    cfg = dict(d=128, n_layers=4, n_heads=4, d_mlp=512, leaf=64, rank=16)
    lay = inputs.network_layout(**cfg)
    w = inputs.network_blob(21, **cfg)
    off = 0
    for name, shp in lay:
        k = int(np.prod(shp))
        if name in ("leaf2.w", "node.w", "off.w"):
            w[off:off + k] *= 10.0
        off += k
    fr, ref, s = _frame(1024, seed)
    ctx = h.Context(max_n=1024, leaf=64, rank=16, d_model=128, n_layers=4, n_heads=4, d_mlp=512, weights=w)
    P = h.packed_width(1024, 64, 16, h.PRE_LEARNED)
    packed = torch.empty(P, dtype=torch.float32, device="cuda")
    h.infer_factors(ctx, [s], packed)
    torch.cuda.synchronize()
    f = hmatrix.unpack(packed.cpu().numpy().astype(np.float64), 1024, 64, 16, "learned")
    a = grid.sparse_matrix(ref)
    out = pcg.pcg(lambda v: a @ v, lambda v: hmatrix.apply(f, v), fr["b"], rtol=fr["rtol"])
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    info = h.solve(ctx, s, h.factors(h.PRE_LEARNED, packed, 1024, 64, 16), b, x, rtol=fr["rtol"])
    _check(info, out, a, fr, x.cpu().numpy())
    ctx.close()


PAPER_CFG = dict(d=128, n_layers=3, n_heads=8, d_mlp=512, leaf=128, rank=32)


@pytest.mark.parametrize("n,seed", [(4096, 4), (8192, 5)])
def test_paper_size_network_on_barrier_frames(n, seed):
    """The paper's model size (Sec. 7.3: d 128, 3 layers, 8 heads of 16, leaf 128, rank 32;
    128-token diagonal windows, 32-token tile windows) on its own frames: GPU factors against the
    FP64 oracle forward element by element, then PCG to rtol 1e-8 on them against the FP64
    oracle PCG on the same packed factors."""
    from oracle import network
    cfg = PAPER_CFG
    lay = inputs.network_layout(**cfg)
    w = inputs.network_blob(22, **cfg)
    off = 0
    for name, shp in lay:
        k = int(np.prod(shp))
        if name in ("leaf2.w", "node.w", "off.w"):
            w[off:off + k] *= 10.0
        off += k
    fr, ref, s = _frame(n, seed)
    L, r = cfg["leaf"], cfg["rank"]
    ctx = h.Context(max_n=n, leaf=L, rank=r, d_model=cfg["d"], n_layers=cfg["n_layers"], n_heads=cfg["n_heads"],
                    d_mlp=cfg["d_mlp"], weights=w)
    P = h.packed_width(n, L, r, h.PRE_LEARNED)
    packed = torch.empty(P, dtype=torch.float32, device="cuda")
    h.infer_factors(ctx, [s], packed)
    torch.cuda.synchronize()
    got = hmatrix.unpack(packed.cpu().numpy().astype(np.float64), n, L, r, "learned")
    p = network.unflatten(w.astype(np.float64), lay)
    with torch.no_grad():
        f = network.to_numpy_factors(network.forward(p, ref, cfg))
    for key in ("leafblk", "U", "V"):
        g2 = got[key].reshape(got[key].shape[0], -1)
        r2 = f[key].reshape(f[key].shape[0], -1)
        sc = np.maximum(np.abs(r2).max(axis=1, keepdims=True), 1e-300)
        e = float((np.abs(g2 - r2) / sc).max())
        assert e <= 0.1, (key, e)
    ce = float((np.abs(got["core"] - f["core"]) / np.maximum(f["core_scale"], 1e-300)).max())
    assert ce <= 0.1, ce
    assert float(np.abs(got["g"] - f["g"]).max() / np.abs(f["g"]).max()) <= 0.1
    a = grid.sparse_matrix(ref)
    out = pcg.pcg(lambda v: a @ v, lambda v: hmatrix.apply(got, v), fr["b"], rtol=fr["rtol"])
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    info = h.solve(ctx, s, h.factors(h.PRE_LEARNED, packed, n, L, r), b, x, rtol=fr["rtol"])
    _check(info, out, a, fr, x.cpu().numpy())
    ctx.close()
