"""The allocation-free apply (hmpcg_apply_noalloc) against the context apply.

hmpcg_apply_noalloc serves callers that cannot call cudaMalloc (allocator
callbacks, real-time loops with a frozen memory budget, plug-ins whose host owns
all device memory): its scratch is a fixed device array inside the library.
This file runs last so that a failure here leaves every other result in place.
"""
import numpy as np
import pytest
import torch

from oracle import hmatrix

pytestmark = pytest.mark.gpu
h = pytest.importorskip("paper_2605_13343_gb300")


def _factors(n, leaf, rank, seed, dtype):
    rng = np.random.default_rng(seed)
    w = hmatrix.packed_width(n, leaf, rank, "learned")
    t = torch.from_numpy(rng.standard_normal(w).astype(np.float32)).to(dtype).cuda()
    return t


@pytest.mark.parametrize("n,dtype", [(8192, torch.bfloat16), (65536, torch.float32), (1024, torch.bfloat16)])
def test_noalloc_apply_matches_context_apply(n, dtype):
    packed = _factors(n, 64, 16, n, dtype)
    fac = h.factors(h.PRE_LEARNED, packed, n, 64, 16)
    ctx = h.Context(max_n=n, leaf=64, rank=16)
    g = torch.Generator(device="cuda").manual_seed(3)
    ref = torch.empty(n, dtype=torch.float32, device="cuda")
    for call in range(2):
        r = torch.randn(n, device="cuda", generator=g)
        h.apply(ctx, fac, r, ref)
        z = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        h.apply_noalloc(fac, r, z)
        torch.cuda.synchronize()
        err = torch.linalg.norm(z - ref).item()
        assert err <= 1e-5 * torch.linalg.norm(ref).item(), (call, err)
    ctx.close()


def test_noalloc_rejects_oversized_factors():
    n = 1 << 22   # needs n + 2 K r + 2 (K - 1) r floats > 4 Mi
    fac = h.Factors()
    fac.kind, fac.dtype, fac.leaf, fac.rank, fac.n = h.PRE_LEARNED, h.BF16, 64, 16, n
    dummy = torch.zeros(16, dtype=torch.bfloat16, device="cuda")
    fac.packed = dummy.data_ptr()
    r = torch.zeros(16, device="cuda")
    rc = h.lib().hmpcg_apply_noalloc(h.C.byref(fac), h.C.c_void_p(r.data_ptr()),
                                     h.C.c_void_p(r.data_ptr()), None)
    assert rc == h.E_SHAPE


def _compare(fac, n, rank, leaf=64):
    ctx = h.Context(max_n=n, leaf=leaf, rank=rank)
    g = torch.Generator(device="cuda").manual_seed(5)
    ref = torch.empty(n, dtype=torch.float32, device="cuda")
    for call in range(2):
        r = torch.randn(n, device="cuda", generator=g)
        h.apply(ctx, fac, r, ref)
        z = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        h.apply_noalloc(fac, r, z)
        torch.cuda.synchronize()
        err = torch.linalg.norm(z - ref).item()
        assert err <= 1e-5 * torch.linalg.norm(ref).item(), (call, err)
    ctx.close()


def test_noalloc_svdh_layout():
    # one bridge slot per level (nslot = levels = 6 at n = 4096): the scratch offsets depend on it
    n, leaf, rank = 4096, 64, 16
    rng = np.random.default_rng(11)
    packed = torch.from_numpy(rng.standard_normal(hmatrix.packed_width(n, leaf, rank, "svdh")).astype(np.float32)).cuda()
    _compare(h.factors(h.PRE_SVDH, packed, n, leaf, rank), n, rank)


def _fp8_blocks(x, rows):
    """FP8-E4M3 with one FP32 scale per block of `rows` values: (stored, scales)."""
    blk = x.reshape(-1, rows)
    sc = blk.abs().amax(dim=1).clamp_min(1e-30) / 448.0
    q = (blk / sc[:, None]).to(torch.float8_e4m3fn)
    return q.flatten(), sc


def test_noalloc_fp8_learned_with_scales():
    # scales in the documented order: leaf blocks, cores, bridges (slot-major, per leaf), gates
    n, leaf, rank = 8192, 64, 16
    k = n // leaf
    rng = np.random.default_rng(12)
    f = hmatrix.unpack(rng.standard_normal(hmatrix.packed_width(n, leaf, rank, "learned")), n, leaf, rank, "learned")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    lq, ls = _fp8_blocks(t(f["leafblk"]), leaf * leaf)
    cq, cs = _fp8_blocks(t(f["core"]), rank * rank)
    uq, us = _fp8_blocks(t(f["U"]), leaf * rank)
    vq, vs = _fp8_blocks(t(f["V"]), leaf * rank)
    gq, gs = _fp8_blocks(t(np.abs(f["g"])), leaf)
    packed = torch.cat([lq, cq, uq, vq, gq]).cuda()
    scales = torch.cat([ls, cs, us, vs, gs]).float().cuda()
    assert scales.numel() == k + (k - 1) + 2 * k + k
    _compare(h.factors(h.PRE_LEARNED, packed, n, leaf, rank, scales), n, rank)


def test_noalloc_at_the_documented_limit():
    # leaf 64, rank 16: n = 2^21 needs n + 2 K r + 2 (K - 1) r = 4 Mi - 32 floats, within the array
    n = 1 << 21
    packed = _factors(n, 64, 16, 13, torch.bfloat16)
    _compare(h.factors(h.PRE_LEARNED, packed, n, 64, 16), n, 16)
