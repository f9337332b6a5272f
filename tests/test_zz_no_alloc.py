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
