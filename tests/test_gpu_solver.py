"""GPU parity of assembly, SpMV, H-apply and PCG against the FP64 oracle.

Tolerances (derivation in the design notes): FP32 accumulation of at most
n_t = L + 2 levels r products per output gives |err| <= n_t u |M| |r| with
u = 2^-24, so the apply is checked at 1e-5 relative in the 2-norm; PCG parity is
the iteration count within max(2, 2 %) of the FP64 oracle and a true relative
residual <= rtol evaluated by the oracle in FP64.
"""
import numpy as np
import pytest
import torch

import inputs
from oracle import grid, hmatrix, pcg

pytestmark = pytest.mark.gpu

h = pytest.importorskip("paper_2605_13343_gb300")


def _gpu_system(dims, rho, bc=0, face=0):
    s = h.System(dims)
    h.assemble(torch.from_numpy(rho).cuda(), s, bc=bc, face=face)
    return s


@pytest.fixture(params=["cluster", "grid"])
def path(request, monkeypatch):
    """Run a PCG test through the thread-block-cluster kernel and the grid-wide kernel."""
    monkeypatch.setenv("HMPCG_PCG_PATH", request.param)
    return request.param


@pytest.fixture(scope="module")
def ctx():
    c = h.Context(max_n=1 << 16, leaf=64, rank=16)
    yield c
    c.close()


# ------------------------------------------------------------------ assembly (bit-exact)
@pytest.mark.parametrize("family,seed,bc,face", [
    ("disc2d_1024", 0, 0, 0), ("spheres3d_8192", 1, 0, 0), ("spheres3d_4096_lu", 2, 1, 0),
    ("disc2d_1024", 3, 0, 1), ("discs2d_16384", 4, 0, 0)])
def test_assemble_bit_exact(family, seed, bc, face):
    fr = inputs.frame(family, seed)
    ref = grid.assemble(fr["rho"], fr["dims"], bc="dirichlet" if bc == 0 else "neumann",
                        face="inv_rho" if face == 0 else "rho")
    s = _gpu_system(fr["dims"], fr["rho"], bc, face)
    torch.cuda.synchronize()
    assert np.array_equal(s.perm.cpu().numpy(), ref["perm"].astype(np.int32))
    assert np.array_equal(s.rho.cpu().numpy(), ref["rho"])
    assert np.array_equal(s.diag.cpu().numpy(), ref["diag"])
    assert np.array_equal(s.diag32.cpu().numpy(), ref["diag"].astype(np.float32))
    for a in range(len(fr["dims"])):
        assert np.array_equal(s.wplus(a).cpu().numpy(), ref["wplus"][a])
        assert np.array_equal(s.wplus32(a).cpu().numpy(), ref["wplus"][a].astype(np.float32))


@pytest.mark.parametrize("dims", [(8, 8), (2, 2), (1024, 1024), (64, 64, 64)])
def test_assemble_edge_sizes(dims):
    n = int(np.prod(dims))
    rho = inputs.density_for_dims(5, dims) if n <= 4096 else np.ones(n)
    s = _gpu_system(dims, rho)
    torch.cuda.synchronize()
    perm = s.perm.cpu().numpy()
    # bijection at any size; sampled cells against the oracle's decode
    assert np.array_equal(np.sort(perm), np.arange(n, dtype=np.int32))
    for m in np.random.default_rng(0).integers(0, n, 50):
        c = grid.morton_decode(int(m), dims)
        assert perm[m] == grid.lex_index(c, dims)


# ------------------------------------------------------------------ SpMV
@pytest.mark.parametrize("family", ["disc2d_1024", "spheres3d_8192"])
def test_spmv(family):
    fr = inputs.frame(family, 0)
    ref = grid.assemble(fr["rho"], fr["dims"])
    s = _gpu_system(fr["dims"], fr["rho"])
    x = np.random.default_rng(1).standard_normal(s.n).astype(np.float32)
    y = torch.empty(s.n, dtype=torch.float32, device="cuda")
    h.spmv(s, torch.from_numpy(x).cuda(), y)
    want = grid.sparse_matrix(ref) @ x.astype(np.float64)
    absa = abs(grid.sparse_matrix(ref)) @ np.abs(x.astype(np.float64))
    err = np.abs(y.cpu().numpy() - want)
    assert (err <= 8 * 2.0 ** -24 * absa + 1e-30).all()


# ------------------------------------------------------------------ apply
def _learned_random(n, leaf, rank, seed, scale_off=1.0):
    rng = np.random.default_rng(seed)
    w = hmatrix.packed_width(n, leaf, rank, "learned")
    f = hmatrix.unpack(rng.standard_normal(w), n, leaf, rank, "learned")
    f["core"] *= scale_off
    return f


def _upload(f, dtype):
    p = hmatrix.pack(f)
    t = torch.from_numpy(p.astype(np.float32))
    if dtype == torch.float32:
        return t.cuda(), None, hmatrix.unpack(t.double().numpy(), f["n"], f["leaf"], f["rank"], f["layout"])
    if dtype == torch.bfloat16:
        q = t.to(torch.bfloat16)
        return q.cuda(), None, hmatrix.unpack(q.double().numpy(), f["n"], f["leaf"], f["rank"], f["layout"])
    raise ValueError


def _fp8_pack(f):
    """Per-block FP8-E4M3 quantisation; returns packed, scales and the dequantised factors."""
    n, L, r, K = f["n"], f["leaf"], f["rank"], f["K"]
    blocks = []   # (array view, scale index) in the scales layout order
    scales = []
    q = {}
    def quant(x):
        amax = float(np.abs(x).max()) or 1.0
        s = amax / 448.0
        xq = torch.from_numpy((x / s).astype(np.float32)).to(torch.float8_e4m3fn)
        return xq, s, xq.double().numpy() * s
    deq = dict(f)
    leafq, leafd, leafs = [], [], []
    for k in range(K):
        a, s, d = quant(f["leafblk"][k]); leafq.append(a); leafs.append(s); leafd.append(d)
    coreq, cored, cores = [], [], []
    for m in range(K - 1):
        a, s, d = quant(f["core"][m]); coreq.append(a); cores.append(s); cored.append(d)
    deq["leafblk"] = np.stack(leafd); deq["core"] = np.stack(cored)
    parts = [torch.cat([x.flatten() for x in leafq]), torch.cat([x.flatten() for x in coreq])]
    brs = []
    if f["layout"] == "learned":
        slots = [f["U"], f["V"]]
    else:
        slots = [f["W"][l] for l in range(f["W"].shape[0])]
    newslots = []
    for arr in slots:
        rows = []
        for k in range(K):
            a, s, d = quant(arr[k * L:(k + 1) * L]); rows.append((a, d)); brs.append(s)
        parts.append(torch.cat([a.flatten() for a, _ in rows]))
        newslots.append(np.vstack([d for _, d in rows]))
    gs = []
    if f["layout"] == "learned":
        deq["U"], deq["V"] = newslots
        gq, gd = [], []
        for k in range(K):
            a, s, d = quant(f["g"][k * L:(k + 1) * L]); gq.append(a); gd.append(d); gs.append(s)
        parts.append(torch.cat(gq))
        deq["g"] = np.concatenate(gd)
    else:
        deq["W"] = np.stack(newslots)
    packed = torch.cat(parts)
    sc = torch.tensor(leafs + cores + brs + gs, dtype=torch.float32)
    return packed.cuda(), sc.cuda(), deq


@pytest.mark.parametrize("n,leaf,rank", [(1024, 64, 16), (128, 64, 16), (8192, 64, 16),
                                         (4096, 128, 32), (512, 8, 8), (65536, 64, 16),
                                         (65536, 64, 8), (65536, 64, 32), (131072, 64, 16)])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_apply_learned_layout(ctx, n, leaf, rank, dtype):
    """Learned layout vs the oracle's structured apply; K >= 512 takes the blocked
    strip-sum path for rank <= 16 (two block levels at N = 131072) and the level tree
    for rank 32."""
    if leaf != 64 or rank != 16 or n > (1 << 16):
        c = h.Context(max_n=n, leaf=leaf, rank=rank)
    else:
        c = ctx
    f = _learned_random(n, leaf, rank, seed=n + leaf)
    if dtype == "fp8":
        packed, sc, deq = _fp8_pack(f)
    else:
        packed, sc, deq = _upload(f, torch.float32 if dtype == "f32" else torch.bfloat16)
    fac = h.factors(h.PRE_LEARNED, packed, n, leaf, rank, sc)
    r = np.random.default_rng(7).standard_normal(n).astype(np.float32)
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    h.apply(c, fac, torch.from_numpy(r).cuda(), z)
    want = hmatrix.apply(deq, r.astype(np.float64))
    got = z.cpu().numpy()
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_apply_svdh_layout_random_large(ctx, dtype):
    """SVD-H layout (one bridge per level) with random factors at K = 1024 leaves: the
    level-tree strip sums of the large-K path against the oracle's structured apply."""
    n, leaf, rank = 65536, 64, 16
    rng = np.random.default_rng(11)
    w = hmatrix.packed_width(n, leaf, rank, "svdh")
    f = hmatrix.unpack(rng.standard_normal(w), n, leaf, rank, "svdh")
    packed, sc, deq = _upload(f, torch.float32 if dtype == "f32" else torch.bfloat16)
    fac = h.factors(h.PRE_SVDH, packed, n, leaf, rank)
    r = np.random.default_rng(8).standard_normal(n).astype(np.float32)
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    h.apply(ctx, fac, torch.from_numpy(r).cuda(), z)
    want = hmatrix.apply(deq, r.astype(np.float64))
    assert np.linalg.norm(z.cpu().numpy() - want) <= 1e-5 * np.linalg.norm(want)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_apply_svdh_layout(ctx, dtype):
    fr = inputs.frame("disc2d_1024", 0)
    ref = grid.assemble(fr["rho"], fr["dims"])
    f = hmatrix.svdh_factors(grid.dense_matrix(ref), 64, 16)
    if dtype == "fp8":
        packed, sc, deq = _fp8_pack(f)
    else:
        packed, sc, deq = _upload(f, torch.float32 if dtype == "f32" else torch.bfloat16)
    fac = h.factors(h.PRE_SVDH, packed, 1024, 64, 16, sc)
    r = np.random.default_rng(8).standard_normal(1024).astype(np.float32)
    z = torch.empty(1024, dtype=torch.float32, device="cuda")
    h.apply(ctx, fac, torch.from_numpy(r).cuda(), z)
    want = hmatrix.apply(deq, r.astype(np.float64))
    assert np.linalg.norm(z.cpu().numpy() - want) <= 1e-5 * np.linalg.norm(want)


# ------------------------------------------------------------------ PCG
def _oracle_solve(ref, b, precond, rtol=1e-6):
    a = grid.sparse_matrix(ref)
    return pcg.pcg(lambda v: a @ v, precond, b, rtol=rtol), a


def _true_rel(a, b, x):
    return np.linalg.norm(b - a @ x) / np.linalg.norm(b)


@pytest.mark.parametrize("family,seed", [("disc2d_1024", 0), ("spheres3d_8192", 0),
                                         ("spheres3d_8192", 3), ("discs2d_16384", 1)])
def test_pcg_jacobi_parity(ctx, path, family, seed):
    fr = inputs.frame(family, seed)
    ref = grid.assemble(fr["rho"], fr["dims"])
    s = _gpu_system(fr["dims"], fr["rho"])
    out, a = _oracle_solve(ref, fr["b"], lambda v: v / ref["diag"])
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    fac = h.Factors(); fac.kind = h.PRE_JACOBI
    info = h.solve(ctx, s, fac, b, x, rtol=1e-6)
    assert info.status == h.OK
    assert abs(info.iters - out["iters"]) <= max(2, 0.02 * out["iters"])
    xg = x.cpu().numpy()
    assert _true_rel(a, fr["b"], xg) <= 1e-6
    assert abs(info.rel_res_true - _true_rel(a, fr["b"], xg)) <= 1e-9
    # agreement with the oracle's solution within the kappa-scaled bound
    assert np.linalg.norm(xg - out["x"]) <= 1e-3 * np.linalg.norm(out["x"])


def test_pcg_cg_and_iteration_cap(ctx, path):
    fr = inputs.frame("disc2d_1024", 2)
    ref = grid.assemble(fr["rho"], fr["dims"])
    s = _gpu_system(fr["dims"], fr["rho"])
    out, a = _oracle_solve(ref, fr["b"], lambda v: v.copy())
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    info = h.solve(ctx, s, None, b, x, rtol=1e-6)
    assert info.status == h.OK
    assert abs(info.iters - out["iters"]) <= max(2, 0.02 * out["iters"])
    info = h.solve(ctx, s, None, b, x, rtol=1e-6, max_iter=5)
    assert info.status == h.NOT_CONVERGED and info.iters == 5
    # b = 0 returns x = 0 with no iterations
    z = torch.zeros_like(b)
    info = h.solve(ctx, s, None, z, x, rtol=1e-6)
    assert info.status == h.OK and info.iters == 0 and float(x.abs().max()) == 0.0


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_pcg_svdh_parity(ctx, path, dtype):
    fr = inputs.frame("disc2d_1024", 0)
    ref = grid.assemble(fr["rho"], fr["dims"])
    ad = grid.dense_matrix(ref)
    f = hmatrix.svdh_factors(ad, 64, 16, leaves="inverse_block")
    packed, sc, deq = _upload(f, torch.float32 if dtype == "f32" else torch.bfloat16)
    out, a = _oracle_solve(ref, fr["b"], lambda v: hmatrix.apply(deq, v))
    assert out["status"] == pcg.OK
    s = _gpu_system(fr["dims"], fr["rho"])
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    info = h.solve(ctx, s, h.factors(h.PRE_SVDH, packed, 1024, 64, 16), b, x, rtol=1e-6)
    assert info.status == h.OK
    assert abs(info.iters - out["iters"]) <= max(2, 0.02 * out["iters"])
    assert _true_rel(a, fr["b"], x.cpu().numpy()) <= 1e-6


def test_pcg_exact_inverse_one_iteration(ctx, path):
    dims = (16, 16)
    rho = inputs.density_discs(3, dims, 1, (4.0, 4.0), 10.0)
    ref = grid.assemble(rho, dims)
    f = hmatrix.svdh_factors(grid.dense_matrix(ref), 64, 128, leaves="inverse_block")
    c = h.Context(max_n=256, leaf=64, rank=128)
    packed = torch.from_numpy(hmatrix.pack(f).astype(np.float32)).cuda()
    s = _gpu_system(dims, rho)
    b = torch.from_numpy(inputs.rhs(0, 256)).cuda()
    x = torch.empty_like(b)
    info = h.solve(c, s, h.factors(h.PRE_SVDH, packed, 256, 64, 128), b, x, rtol=1e-5)
    assert info.status == h.OK and info.iters <= 2


@pytest.mark.parametrize("how", ["negated", "block_inverse_leaves"])
def test_pcg_breakdown_indefinite(ctx, path, how):
    # (A_kk)^-1 leaves with truncated tiles are indefinite on this frame (the oracle breaks
    # down at the first iteration too); a negated M is indefinite by construction
    fr = inputs.frame("disc2d_1024", 0)
    ref = grid.assemble(fr["rho"], fr["dims"])
    f = hmatrix.svdh_factors(grid.dense_matrix(ref), 64, 16,
                             leaves="block_inverse" if how != "negated" else "inverse_block")
    if how == "negated":
        f["leafblk"] = -f["leafblk"]
        f["core"] = -f["core"]
    out, a = _oracle_solve(ref, fr["b"], lambda v: hmatrix.apply(f, v))
    assert out["status"] == pcg.BREAKDOWN
    packed = torch.from_numpy(hmatrix.pack(f).astype(np.float32)).cuda()
    s = _gpu_system(fr["dims"], fr["rho"])
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    info = h.solve(ctx, s, h.factors(h.PRE_SVDH, packed, 1024, 64, 16), b, x, rtol=1e-6,
                   allow=(h.E_BREAKDOWN,))
    assert info.status == h.E_BREAKDOWN


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_pcg_learned_layout_random_spd(ctx, path, dtype):
    # M = Jacobi gate + small PSD leaf term + small tiles: SPD, close to Jacobi
    fr = inputs.frame("spheres3d_8192", 2)
    ref = grid.assemble(fr["rho"], fr["dims"])
    n = ref["n"]
    f = _learned_random(n, 64, 16, seed=5)
    dinv = 1.0 / ref["diag"]
    f["g"] = dinv
    for k in range(n // 64):
        f["leafblk"][k] *= 0.02 * np.sqrt(dinv[k * 64:(k + 1) * 64])[:, None]
    f["U"] *= 0.3 * np.sqrt(dinv / n)[:, None]
    f["V"] *= 0.3 * np.sqrt(dinv / n)[:, None]
    f["core"] *= 0.3
    if dtype == "fp8":
        packed, sc, deq = _fp8_pack(f)
    else:
        packed, sc, deq = _upload(f, torch.float32 if dtype == "f32" else torch.bfloat16)
    out, a = _oracle_solve(ref, fr["b"], lambda v: hmatrix.apply(deq, v))
    assert out["status"] == pcg.OK
    s = _gpu_system(fr["dims"], fr["rho"])
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    info = h.solve(ctx, s, h.factors(h.PRE_LEARNED, packed, n, 64, 16, sc), b, x, rtol=1e-6)
    assert info.status == h.OK
    assert abs(info.iters - out["iters"]) <= max(2, 0.02 * out["iters"])
    assert _true_rel(a, fr["b"], x.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_pcg_learned_layout_n16384(ctx, path, dtype):
    """N = 16384 on one cluster: 16 leaves per CTA, so the BF16 leaf blocks live in shared memory
    without the bridges (swizzled rows, one warp per leaf) and the FP32 ones are read from L2."""
    fr = inputs.frame("discs2d_16384", 1)
    ref = grid.assemble(fr["rho"], fr["dims"])
    n = ref["n"]
    f = _learned_random(n, 64, 16, seed=9)
    dinv = 1.0 / ref["diag"]
    f["g"] = dinv
    for k in range(n // 64):
        f["leafblk"][k] *= 0.02 * np.sqrt(dinv[k * 64:(k + 1) * 64])[:, None]
    f["U"] *= 0.3 * np.sqrt(dinv / n)[:, None]
    f["V"] *= 0.3 * np.sqrt(dinv / n)[:, None]
    f["core"] *= 0.3
    packed, sc, deq = _upload(f, torch.float32 if dtype == "f32" else torch.bfloat16)
    out, a = _oracle_solve(ref, fr["b"], lambda v: hmatrix.apply(deq, v))
    assert out["status"] == pcg.OK
    s = _gpu_system(fr["dims"], fr["rho"])
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    info = h.solve(ctx, s, h.factors(h.PRE_LEARNED, packed, n, 64, 16, sc), b, x, rtol=1e-6)
    assert info.status == h.OK
    assert abs(info.iters - out["iters"]) <= max(2, 0.02 * out["iters"])
    assert _true_rel(a, fr["b"], x.cpu().numpy()) <= 1e-6
