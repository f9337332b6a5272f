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
