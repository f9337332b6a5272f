"""GPU parity of the tcgen05 GEMM and of the hierarchical-transformer inference.

The GEMM is checked against a plain PyTorch FP32 matmul of the same BF16
operands (TF32 off).  The network forward runs BF16 GEMM operands with FP32
accumulation through ~30 dependent layers; its factors are checked against the
FP64 oracle forward on the same seeded weights at 3e-2 relative Frobenius
error per factor block (BF16 unit roundoff 3.9e-3 times the depth of the
residual stream, with margin).
"""
import numpy as np
import pytest
import torch

import inputs
from oracle import grid, hmatrix, network, pcg

pytestmark = pytest.mark.gpu
h = pytest.importorskip("paper_2605_13343_gb300")

CFG = dict(d=128, n_layers=4, n_heads=4, d_mlp=512, leaf=64, rank=16)


@pytest.mark.parametrize("m,n,k,bias,act", [(8192, 384, 128, True, 0), (2032, 128, 512, True, 1),
                                            (100, 64, 64, False, 0), (300, 32, 128, True, 1),
                                            (4096, 256, 256, False, 1), (128, 512, 512, True, 0),
                                            (32768, 512, 256, True, 1), (20000, 128, 512, False, 0)])
def test_gemm_tc_matches_torch(m, n, k, bias, act):
    torch.backends.cuda.matmul.allow_tf32 = False
    g = torch.Generator(device="cuda").manual_seed(m + n + k)
    a = torch.randn(m, k, device="cuda", generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, device="cuda", generator=g).to(torch.bfloat16)
    bb = torch.randn(n, device="cuda", generator=g) if bias else None
    c = h.gemm_bf16(a, b, bias=bb, act=act)
    ref = a.float() @ b.float().T
    if bias:
        ref = ref + bb
    if act:
        ref = torch.nn.functional.gelu(ref)
    torch.cuda.synchronize()
    err = (c - ref).abs().max().item()
    assert err <= 1e-4 * max(1.0, ref.abs().max().item()), err


def _blob(seed, scale_heads=100.0):
    lay = inputs.network_layout(**CFG)
    w = inputs.network_blob(seed, **CFG)
    off = 0
    for name, shp in lay:
        n = int(np.prod(shp))
        if name in ("leaf2.w", "node.w", "off.w"):
            w[off:off + n] *= scale_heads
        off += n
    return w, lay


def _ctx(max_n, weights, batch=1):
    return h.Context(max_n=max_n, leaf=64, rank=16, d_model=128, n_layers=4, n_heads=4, d_mlp=512,
                     max_batch=batch, weights=weights)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


# Element-wise bound: |got - ref| <= ELEM_TOL * max |ref| over each factor block (per leaf for F,
# per node row for U~ and V~, the gate over all nodes) and, for the tile cores B_m = U_m V_m^T,
# ELEM_TOL * (|U_m| |V_m|^T)_ij, the scale of that entry's dot product.  Both BF16 paths land
# near 0.02 (measured on the GB300); 0.1 leaves room for the ~30 BF16-rounded layers while a
# wrong row, tile or chunk (errors of order 1) still fails.
ELEM_TOL = 0.1


def _elem(got, ref):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))
    g2 = got.reshape(got.shape[0], -1)
    r2 = ref.reshape(ref.shape[0], -1)
    scale = np.maximum(np.abs(r2).max(axis=1, keepdims=True), 1e-300)
    return float((np.abs(g2 - r2) / scale).max())


def _gpu_system(fr):
    s = h.System(fr["dims"])
    h.assemble(torch.from_numpy(fr["rho"]).cuda(), s)
    return s


def test_weight_count_matches_layout():
    w, lay = _blob(0)
    c = h.Config(max_n=4096, max_batch=1, max_nrhs=1, leaf=64, rank=16, d_model=128, n_layers=4,
                 n_heads=4, d_mlp=512)
    import ctypes
    assert h.lib().hmpcg_weight_count(ctypes.byref(c)) == w.size


@pytest.mark.parametrize("family,seeds,highway", [("spheres3d_4096_lu", [0], True), ("spheres3d_4096_lu", [1, 2], True),
                                                  ("spheres3d_8192", [0], True), ("spheres3d_4096_lu", [5], False)])
def test_inference_parity(family, seeds, highway):
    w, lay = _blob(7)
    frs = [inputs.frame(family, s) for s in seeds]
    n = int(np.prod(frs[0]["dims"]))
    ctx = _ctx(n, w, batch=len(seeds))
    if not highway:
        h.set_highways(ctx, False)
    systems = [_gpu_system(fr) for fr in frs]
    P = h.packed_width(n, 64, 16, h.PRE_LEARNED)
    packed = torch.empty(len(seeds) * P, dtype=torch.float32, device="cuda")
    h.infer_factors(ctx, systems, packed)
    torch.cuda.synchronize()
    got_all = packed.cpu().numpy().astype(np.float64)
    p = network.unflatten(w, lay)
    for b, fr in enumerate(frs):
        ref = grid.assemble(fr["rho"], fr["dims"])
        with torch.no_grad():
            f = network.to_numpy_factors(network.forward(p, ref, CFG, highway=highway))
        got = hmatrix.unpack(got_all[b * P:(b + 1) * P], n, 64, 16, "learned")
        for key in ("leafblk", "U", "V"):
            assert _rel(got[key], f[key]) <= 3e-2, (key, _rel(got[key], f[key]))
        # the cores B_m = U_m V_m^T cancel (without highways their entries are nearly equal and
        # about 4x below |U_m||V_m|^T): their Frobenius error is measured against that scale
        cf = float(np.linalg.norm(got["core"] - f["core"]) / np.linalg.norm(f["core_scale"]))
        assert cf <= 3e-2, cf
        for key in ("leafblk", "U", "V"):
            # element by element: no entry off by more than ELEM_TOL of its block's scale
            assert _elem(got[key], f[key]) <= ELEM_TOL, (key, _elem(got[key], f[key]))
        # a core entry is a 16-term dot product that can cancel: its scale is (|U_m| |V_m|^T)_ij
        ce = float((np.abs(got["core"] - f["core"]) / np.maximum(f["core_scale"], 1e-300)).max())
        assert ce <= ELEM_TOL, ce
        assert _rel(got["g"], f["g"]) <= 1e-2
        assert _elem(got["g"], f["g"]) <= ELEM_TOL
        # the assembled preconditioners agree as operators too
        x = np.random.default_rng(b).standard_normal(n)
        assert _rel(hmatrix.apply(got, x), hmatrix.apply(f, x)) <= 3e-2
    ctx.close()


def test_learned_pcg_end_to_end():
    w, lay = _blob(3, scale_heads=10.0)
    fr = inputs.frame("spheres3d_8192", 4)
    n = 8192
    ctx = _ctx(n, w)
    s = _gpu_system(fr)
    P = h.packed_width(n, 64, 16, h.PRE_LEARNED)
    packed = torch.empty(P, dtype=torch.bfloat16, device="cuda")
    h.infer_factors(ctx, [s], packed)
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    info = h.solve(ctx, s, h.factors(h.PRE_LEARNED, packed, n, 64, 16), b, x, rtol=1e-6)
    assert info.status == h.OK
    ref = grid.assemble(fr["rho"], fr["dims"])
    a = grid.sparse_matrix(ref)
    rel = np.linalg.norm(fr["b"] - a @ x.cpu().numpy()) / np.linalg.norm(fr["b"])
    assert rel <= 1e-6
    # iteration count against the oracle PCG on the oracle's FP64 factors
    p = network.unflatten(w, lay)
    with torch.no_grad():
        f = network.to_numpy_factors(network.forward(p, ref, CFG))
    out = pcg.pcg(lambda v: a @ v, lambda v: hmatrix.apply(f, v), fr["b"], rtol=1e-6)
    assert out["status"] == pcg.OK
    assert abs(info.iters - out["iters"]) <= max(3, 0.05 * out["iters"])
    ctx.close()


@pytest.mark.parametrize("family,seeds", [("spheres3d_8192", [5]), ("spheres3d_4096_lu", [3, 4, 6])])
def test_fused_inference_matches_layered(family, seeds):
    """The fused layer kernels and the layered kernels compute the same network: factors of
    both modes agree block by block (both round GEMM operands and probabilities to BF16)."""
    w, lay = _blob(11)
    frs = [inputs.frame(family, s) for s in seeds]
    n = int(np.prod(frs[0]["dims"]))
    ctx = _ctx(n, w, batch=len(seeds))
    systems = [_gpu_system(fr) for fr in frs]
    P = h.packed_width(n, 64, 16, h.PRE_LEARNED)
    out = {}
    for mode in (h.INFER_LAYERED, h.INFER_FUSED):
        h.set_infer_mode(ctx, mode)
        packed = torch.empty(len(seeds) * P, dtype=torch.float32, device="cuda")
        h.infer_factors(ctx, systems, packed)
        torch.cuda.synchronize()
        out[mode] = packed.cpu().numpy().astype(np.float64)
    for b in range(len(seeds)):
        fu = hmatrix.unpack(out[h.INFER_FUSED][b * P:(b + 1) * P], n, 64, 16, "learned")
        la = hmatrix.unpack(out[h.INFER_LAYERED][b * P:(b + 1) * P], n, 64, 16, "learned")
        for key in ("leafblk", "U", "V", "core", "g"):
            assert np.isfinite(fu[key]).all()
            assert _rel(fu[key], la[key]) <= 3e-2, (key, _rel(fu[key], la[key]))
            if key != "core":
                assert _elem(fu[key], la[key]) <= ELEM_TOL, (key, _elem(fu[key], la[key]))
    ctx.close()


def test_fp8_inference_quantises_each_block():
    """FP8 factors from hmpcg_infer_factors: every block is the FP32 inference rounded to E4M3
    with scale max|block| / 448; the dequantised factors stay within the element bound of the
    FP64 oracle forward, and learned PCG on them matches the FP64 oracle PCG on the same
    (dequantised) preconditioner."""
    w, lay = _blob(3, scale_heads=10.0)
    fr = inputs.frame("spheres3d_8192", 6)
    n, L, r = 8192, 64, 16
    K = n // L
    ctx = _ctx(n, w)
    s = _gpu_system(fr)
    P = h.packed_width(n, L, r, h.PRE_LEARNED)
    p32 = torch.empty(P, dtype=torch.float32, device="cuda")
    h.infer_factors(ctx, [s], p32)
    p8 = torch.empty(P, dtype=torch.float8_e4m3fn, device="cuda")
    sc = torch.empty(4 * K + K - 1, dtype=torch.float32, device="cuda")
    h.infer_factors(ctx, [s], p8, scales=sc)
    torch.cuda.synchronize()
    f32 = p32.cpu().double().numpy()
    q = p8.cpu().float().double().numpy()
    scn = sc.cpu().double().numpy()
    # block boundaries in packed order (the scale order)
    offs, lens = [], []
    o = 0
    for cnt, ln in ((K, L * L), (K - 1, r * r), (K, L * r), (K, L * r), (K, L)):
        for _ in range(cnt):
            offs.append(o); lens.append(ln); o += ln
    assert o == P
    deq = np.empty(P)
    for j, (o, ln) in enumerate(zip(offs, lens)):
        blk = f32[o:o + ln]
        amax = np.abs(blk).max()
        assert abs(scn[j] - amax / 448.0) <= 1e-6 * amax / 448.0, j
        deq[o:o + ln] = q[o:o + ln] * scn[j]
        # E4M3: 3 mantissa bits, so rounding moves a normal value by <= 2^-4 of itself and a
        # subnormal one (|v| < 2^-6 scale) by <= 2^-10 scale; two FP32 runs of the network may
        # differ in the last bits, which can move a value to the neighbouring code: allow 2^-3
        assert np.all(np.abs(deq[o:o + ln] - blk) <= 2.0 ** -3 * np.abs(blk) + 2.0 ** -9 * scn[j]), j
    got = hmatrix.unpack(deq, n, L, r, "learned")
    ref = grid.assemble(fr["rho"], fr["dims"])
    p = network.unflatten(w, lay)
    with torch.no_grad():
        f = network.to_numpy_factors(network.forward(p, ref, CFG))
    for key in ("leafblk", "U", "V"):
        assert _elem(got[key], f[key]) <= ELEM_TOL, (key, _elem(got[key], f[key]))
    ce = float((np.abs(got["core"] - f["core"]) / np.maximum(f["core_scale"], 1e-300)).max())
    assert ce <= ELEM_TOL, ce
    assert _elem(got["g"], f["g"]) <= ELEM_TOL
    a = grid.sparse_matrix(ref)
    out = pcg.pcg(lambda v: a @ v, lambda v: hmatrix.apply(got, v), fr["b"], rtol=1e-6)
    assert out["status"] == pcg.OK
    b = torch.from_numpy(fr["b"]).cuda()
    x = torch.empty_like(b)
    info = h.solve(ctx, s, h.factors(h.PRE_LEARNED, p8, n, L, r, sc), b, x, rtol=1e-6)
    assert info.status == h.OK
    rel = np.linalg.norm(fr["b"] - a @ x.cpu().numpy()) / np.linalg.norm(fr["b"])
    assert rel <= 1e-6
    assert abs(info.iters - out["iters"]) <= max(2, 0.05 * out["iters"]), (info.iters, out["iters"])
    ctx.close()


def test_fp8_inference_argument_checks():
    w, _ = _blob(3)
    ctx = _ctx(4096, w)
    fr = inputs.frame("spheres3d_4096_lu", 0)
    s = _gpu_system(fr)
    P = h.packed_width(4096, 64, 16, h.PRE_LEARNED)
    p8 = torch.empty(P, dtype=torch.float8_e4m3fn, device="cuda")
    p32 = torch.empty(P, dtype=torch.float32, device="cuda")
    sc = torch.empty(4 * 64 + 63, dtype=torch.float32, device="cuda")
    arr = h.systems_array([s])
    lib = h.lib()
    assert lib.hmpcg_infer_factors(ctx.h, arr, 1, h.C.c_void_p(p8.data_ptr()), h.FP8E4M3, None, None) == h.E_INVALID
    assert lib.hmpcg_infer_factors(ctx.h, arr, 1, h.C.c_void_p(p32.data_ptr()), h.F32,
                                   h.C.c_void_p(sc.data_ptr()), None) == h.E_INVALID
    ctx.close()
